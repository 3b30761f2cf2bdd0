// The extern "C" boundary of the library: argument validation, lattice
// repacking into the four sweep orientations, the full / cluster / norm
// drivers (host-threaded lanes of streams; row passes that start as soon as
// their boundaries exist; cluster windows batched by shape), recorded plans
// (CUDA graphs) and their autotuner, the learned-closure calls, and
// kernel-class instrumentation.  No exception crosses this file.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <exception>
#include <thread>
#include <vector>

#include "aux.cuh"
#include "closure.cuh"
#include "engine.cuh"
#include "linalg.cuh"
#include "update.cuh"

using namespace peps;

// ---------------------------------------------------------------------------
// Instrumentation
// ---------------------------------------------------------------------------
namespace {

const char* kClassNames[K_NCLASS] = {"gemm_f64", "gemm_tc", "qr_f64", "svd_f64", "cu0", "observables", "aux", "pack"};

struct Prof {
  std::mutex mu;
  unsigned mask = 0;
  long long launches[K_NCLASS] = {};
  double flops[K_NCLASS] = {}, bytes[K_NCLASS] = {}, ms[K_NCLASS] = {};
  std::vector<cudaEvent_t> pool;
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> pending;

  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void drain() {
    for (auto& t : pending) {
      cudaEventSynchronize(std::get<2>(t));
      float m = 0.f;
      cudaEventElapsedTime(&m, std::get<1>(t), std::get<2>(t));
      ms[std::get<0>(t)] += m;
      pool.push_back(std::get<1>(t));
      pool.push_back(std::get<2>(t));
    }
    pending.clear();
  }
};

Prof& prof() {
  static Prof* p = new Prof();
  return *p;
}

// Start event of the launch in flight, per class and per host thread.
thread_local cudaEvent_t t_open_ev[K_NCLASS] = {};

// Counters of the graph being recorded (launch, flop and byte counts per
// class); while set, launches are counted there and not timed.
struct Counts {
  long long launches[K_NCLASS] = {};
  double flops[K_NCLASS] = {}, bytes[K_NCLASS] = {};
  // Timed classes: event pairs recorded as external event nodes of the graph,
  // read after every replay.
  std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> events;
};
std::atomic<Counts*> g_recording{nullptr};

thread_local std::string g_err;


int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

template <class F>
int guard(F&& f) {
  try {
    f();
    return PEPS_OK;
  } catch (const Error& e) {
    return fail(e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(PEPS_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(PEPS_ECUDA, e.what());
  }
}

}  // namespace

namespace peps {
std::atomic<int> g_fault_alloc{0};
std::atomic<int> g_cap_cu0{200}, g_cap_jacobi{60};

int fault_from_env() {
  const char* e = std::getenv("PEPS_FAULT");
  if (!e || !*e) return FAULT_NONE;
  const std::string v(e);
  if (v == "alloc") return FAULT_ALLOC;
  if (v == "nan") return FAULT_NAN;
  if (v == "converge") return FAULT_CONVERGE;
  return FAULT_NONE;
}
int cap_cu0_half_sweeps() { return g_cap_cu0.load(); }
int cap_jacobi_sweeps() { return g_cap_jacobi.load(); }

int peps_set_error(int code, const std::string& msg) { return fail(code, msg); }

void prof_launch(KClass c, cudaStream_t st, double flops, double bytes) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  if (Counts* rc = g_recording.load()) {
    rc->launches[c]++;
    rc->flops[c] += flops;
    rc->bytes[c] += bytes;
    if (p.mask & (1u << c)) {
      cudaEvent_t e = p.get();
      cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
      t_open_ev[c] = e;
    }
    return;
  }
  p.launches[c]++;
  p.flops[c] += flops;
  p.bytes[c] += bytes;
  if (p.mask & (1u << c)) {
    cudaEvent_t e = p.get();
    cudaEventRecord(e, st);
    t_open_ev[c] = e;
  }
}
void prof_more(KClass c, int kernels) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  if (Counts* rc = g_recording.load())
    rc->launches[c] += kernels;
  else
    p.launches[c] += kernels;
}
void prof_done(KClass c, cudaStream_t st) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  if (Counts* rc = g_recording.load()) {
    if ((p.mask & (1u << c)) && t_open_ev[c]) {
      cudaEvent_t e = p.get();
      cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
      rc->events.emplace_back(int(c), t_open_ev[c], e);
      t_open_ev[c] = nullptr;
    }
    return;
  }
  if ((p.mask & (1u << c)) && t_open_ev[c]) {
    cudaEvent_t e = p.get();
    cudaEventRecord(e, st);
    p.pending.emplace_back(int(c), t_open_ev[c], e);
    t_open_ev[c] = nullptr;
  }
}
bool prof_timing() { return prof().mask != 0; }
}  // namespace peps

// ---------------------------------------------------------------------------
// Env handle
// ---------------------------------------------------------------------------
struct peps_env {
  int device = 0;
  EnvData data;
  std::unique_ptr<Arena> arena;   // owns the device memory of this handle
  int kind = 0;                   // 0 full, 1 cluster
};

namespace {

// Launch configuration of one call: host lanes (0: PEPS_LANES or 4) and the
// largest thread-block cluster of a QR (0: PEPS_QR_CMAX or 16).
struct Tune {
  int lanes = 0;
  int qr_cmax = 0;
  int chunk = 0;   // cluster windows per batched chunk (0: 16)
};

// PEPS_FAULT=alloc for the lifetime of one call (set before the call's first
// allocation, cleared when the call ends, also by an exception).
struct FaultScope {
  int mode;
  FaultScope() : mode(fault_from_env()) {
    if (mode == FAULT_ALLOC) g_fault_alloc.fetch_add(1);
  }
  ~FaultScope() {
    if (mode == FAULT_ALLOC) g_fault_alloc.fetch_sub(1);
  }
};

struct Call {
  FaultScope fault;
  cudaStream_t st;
  Arena ws;
  Ctx cx;
  Tune tune;
  // persist: set while recording a graph; the status word and staged host
  // data then live in memory that outlives the recording.
  explicit Call(void* stream, Arena* persist = nullptr, Tune t = Tune())
      : st(static_cast<cudaStream_t>(stream)), ws(st), cx(st, &ws), tune(t) {
    cx.persist = persist;
    cx.svd_cap = fault.mode == FAULT_CONVERGE ? 1 : cap_jacobi_sweeps();
    cx.cu0_cap = fault.mode == FAULT_CONVERGE ? 1 : cap_cu0_half_sweeps();
    if (const char* e = std::getenv("PEPS_QR_CMAX")) cx.qr_cmax = std::atoi(e);
    if (tune.qr_cmax > 0) cx.qr_cmax = tune.qr_cmax;
    cx.flag = static_cast<int*>(persist ? persist->alloc(sizeof(int)) : ws.alloc(sizeof(int)));
    PEPS_CUDA(cudaMemsetAsync(cx.flag, 0, sizeof(int), st));
    cx.tmp = ws.dalloc(8);
  }
  // Synchronise and turn the device status word into a status code.
  void finish() { read_status(cx.flag, st); }
  static void read_status(const int* flag, cudaStream_t st) {
    int h = 0;
    PEPS_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    PEPS_CUDA(cudaStreamSynchronize(st));
    if (h & FLAG_SVD_NOCONV) throw Error(PEPS_ECONVERGE, "Jacobi SVD did not converge within its sweep cap");
    if (h & FLAG_CU0_NOCONV) throw Error(PEPS_ECONVERGE, "CU_0 separable boundary did not converge within its half-sweep cap");
    if (h & FLAG_BAD_VALUE) throw Error(PEPS_EINVAL, "zero or non-finite norm encountered (degenerate state)");
    if (h & FLAG_TIMEOUT) throw Error(PEPS_ETIMEOUT, "a device-side bounded wait ran out");
  }
};

void require_device() {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    throw Error(PEPS_ECUDA, "no CUDA device available (this library has no CPU path)");
  }
}

void check_lattice(const peps_lattice* lat) {
  PEPS_REQUIRE(lat != nullptr, "lattice is NULL");
  PEPS_REQUIRE(lat->Ly >= 1 && lat->Lx >= 1 && lat->Ly <= 4096 && lat->Lx <= 4096, "Ly, Lx must be in [1, 4096]");
  PEPS_REQUIRE(lat->d >= 1 && lat->d <= 4, "d must be in [1, 4]");
  PEPS_REQUIRE(lat->D >= 1 && lat->D <= 16, "D must be in [1, 16]");
  PEPS_REQUIRE(lat->dtype == PEPS_F64 || lat->dtype == PEPS_F32, "dtype must be PEPS_F64 or PEPS_F32");
  PEPS_REQUIRE(lat->A != nullptr, "A is NULL");
}

Opts check_opts(const peps_opts* o, bool cluster) {
  PEPS_REQUIRE(o != nullptr, "opts is NULL");
  PEPS_REQUIRE(o->chi >= 1 && o->chi <= 4096, "chi must be in [1, 4096]");
  PEPS_REQUIRE(o->mode == PEPS_SVD || o->mode == PEPS_VAR, "mode must be PEPS_SVD or PEPS_VAR");
  PEPS_REQUIRE(o->precision >= PEPS_PREC_FP64 && o->precision <= PEPS_PREC_BF16X3,
               "precision must be one of PEPS_PREC_FP64, _TF32, _BF16, _TF32X3, _BF16X3");
  if (o->precision != PEPS_PREC_FP64)
    PEPS_REQUIRE(tc_available(), "tensor-core precisions need an sm_103 (GB300) device");
  PEPS_REQUIRE(o->closure == PEPS_CLOSURE_PLAIN || o->closure == PEPS_CLOSURE_LEARNED,
               "closure must be PEPS_CLOSURE_PLAIN or PEPS_CLOSURE_LEARNED");
  PEPS_REQUIRE(o->closure == PEPS_CLOSURE_PLAIN || o->closure_weights != nullptr,
               "PEPS_CLOSURE_LEARNED needs closure_weights (device float*)");
  if (cluster) PEPS_REQUIRE(o->n >= 1, "cluster size n must be >= 1");
  Opts r;
  r.chi = o->chi;
  r.mode = o->mode;
  r.sweeps = o->sweeps <= 0 ? 2 : o->sweeps;
  r.precision = o->precision;
  r.seed = o->seed;
  return r;
}

long long obc_violations_host(const peps_lattice* L) {
  const int Ly = L->Ly, Lx = L->Lx, d = L->d, D = L->D;
  long long c = 0;
  const long long per = (long long)d * D * D * D * D;
  for (int y = 0; y < Ly; ++y)
    for (int x = 0; x < Lx; ++x)
      for (long long e = 0; e < per; ++e) {
        long long r = e;
        const int ri = int(r % D);
        r /= D;
        const int ni = int(r % D);
        r /= D;
        const int li = int(r % D);
        r /= D;
        const int ui = int(r % D);
        const bool out = (y == 0 && ui) || (x == 0 && li) || (y == Ly - 1 && ni) || (x == Lx - 1 && ri);
        if (!out) continue;
        const long long idx = ((long long)y * Lx + x) * per + e;
        const double v = L->dtype == PEPS_F32 ? double(static_cast<const float*>(L->A)[idx])
                                              : static_cast<const double*>(L->A)[idx];
        if (v != 0.0) ++c;
      }
  return c;
}

// The four sweep orientations of the full lattice (top-down, bottom-up,
// left-right, right-left), repacked with effective OBC dimensions.
struct Oriented {
  OLat o[4];
  double* one = nullptr;
  int Dmax = 0;
};

void build_orientations(Ctx& cx, const peps_lattice* in, Arena& keep, Oriented& out) {
  const int Ly = in->Ly, Lx = in->Lx, d = in->d, D = in->D;
  const size_t elems = size_t(Ly) * Lx * d * D * D * D * D;
  const size_t esz = in->dtype == PEPS_F32 ? 4 : 8;
  const void* src = in->A;
  const bool plant_nan = fault_from_env() == FAULT_NAN && !cx.persist;
  if (!in->on_device) {
    const long long bad = obc_violations_host(in);
    PEPS_REQUIRE(bad == 0, "A has " + std::to_string(bad) + " nonzero entries on outward (OBC) legs");
    void* dsrc = cx.ws->alloc(elems * esz);
    PEPS_CUDA(cudaMemcpyAsync(dsrc, in->A, elems * esz, cudaMemcpyHostToDevice, cx.st));
    src = dsrc;
  } else {
    cudaPointerAttributes at;
    PEPS_CUDA(cudaPointerGetAttributes(&at, in->A));
    PEPS_REQUIRE(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged,
                 "on_device is set but A is not a device pointer");
    if (plant_nan) {   // never write into the caller's buffer: plant into a copy
      void* dsrc = cx.ws->alloc(elems * esz);
      PEPS_CUDA(cudaMemcpyAsync(dsrc, in->A, elems * esz, cudaMemcpyDeviceToDevice, cx.st));
      src = dsrc;
    }
  }
  if (plant_nan) plant_nan_value(cx, const_cast<void*>(src), in->dtype == PEPS_F32);
  if (!cx.persist) {   // a recorded graph was validated by the plain call made before it
    const auto bad = input_violations_device(cx, src, in->dtype == PEPS_F32, Ly, Lx, d, D);
    PEPS_REQUIRE(bad.first == 0, "A has " + std::to_string(bad.first) + " nonzero entries on outward (OBC) legs");
    PEPS_REQUIRE(bad.second == 0, "A has " + std::to_string(bad.second) + " non-finite entries");
  }
  out.one = keep.dalloc(1);
  fill(cx, out.one, 1, 1.0);
  out.Dmax = D;
  const size_t per = size_t(d) * D * D * D * D;
  static const int perms[4][4] = {{0, 1, 2, 3}, {2, 1, 0, 3}, {1, 0, 3, 2}, {3, 0, 1, 2}};
  for (int o = 0; o < 4; ++o) {
    const int H = (o < 2) ? Ly : Lx, W = (o < 2) ? Lx : Ly;
    double* buf = keep.dalloc(per * H * W);
    std::vector<OrientSite> sites(size_t(H) * W);
    OLat& L = out.o[o];
    L.Ly = H;
    L.Lx = W;
    L.d = d;
    L.sites.resize(size_t(H) * W);
    for (int i = 0; i < H; ++i)
      for (int j = 0; j < W; ++j) {
        int y, x;
        if (o == 0) { y = i; x = j; }
        else if (o == 1) { y = Ly - 1 - i; x = j; }
        else if (o == 2) { y = j; x = i; }
        else { y = j; x = Lx - 1 - i; }
        const int od[4] = {y == 0 ? 1 : D, x == 0 ? 1 : D, y == Ly - 1 ? 1 : D, x == Lx - 1 ? 1 : D};
        OrientSite& s = sites[size_t(i) * W + j];
        s.dst = (long long)((size_t(i) * W + j) * per);
        s.y = y;
        s.x = x;
        for (int k = 0; k < 4; ++k) s.perm[k] = perms[o][k];
        s.du = od[s.perm[0]];
        s.dl = od[s.perm[1]];
        s.dn = od[s.perm[2]];
        s.dr = od[s.perm[3]];
        SiteT& t = L.sites[size_t(i) * W + j];
        t.p = buf + s.dst;
        t.d = d;
        t.du = s.du;
        t.dl = s.dl;
        t.dn = s.dn;
        t.dr = s.dr;
      }
    orient_lattice(cx, src, in->dtype == PEPS_F32, Ly, Lx, d, D, sites.data(), int(sites.size()), buf);
    const Mat one{out.one, 1};
    L.top.assign(W, one);
    L.bottom.assign(W, one);
    L.left.assign(H, one);
    L.right.assign(H, one);
  }
}

std::unique_ptr<peps_env> new_env(const peps_lattice* lat, int kind, cudaStream_t st) {
  auto env = std::make_unique<peps_env>();
  PEPS_CUDA(cudaGetDevice(&env->device));
  env->arena = std::make_unique<Arena>(st, size_t(64) << 20, /*async=*/false);
  env->kind = kind;
  EnvData& e = env->data;
  e.Ly = lat->Ly;
  e.Lx = lat->Lx;
  e.d = lat->d;
  e.D = lat->D;
  const size_t d2 = size_t(lat->d) * lat->d, d4 = d2 * d2;
  e.rho_site = env->arena->dalloc(size_t(e.Ly) * e.Lx * d2);
  e.rho_h = env->arena->dalloc(std::max<size_t>(1, size_t(e.Ly) * (e.Lx - 1) * d4));
  e.rho_v = env->arena->dalloc(std::max<size_t>(1, size_t(e.Ly - 1) * e.Lx * d4));
  e.lnnorm = env->arena->dalloc(2);
  // Quantities a cluster window cannot see (bonds when n = 1) stay zero.
  PEPS_CUDA(cudaMemsetAsync(e.rho_site, 0, sizeof(double) * size_t(e.Ly) * e.Lx * d2, st));
  PEPS_CUDA(cudaMemsetAsync(e.rho_h, 0, sizeof(double) * std::max<size_t>(1, size_t(e.Ly) * (e.Lx - 1) * d4), st));
  PEPS_CUDA(cudaMemsetAsync(e.rho_v, 0, sizeof(double) * std::max<size_t>(1, size_t(e.Ly - 1) * e.Lx * d4), st));
  return env;
}

// ---------------------------------------------------------------------------
// Lanes: independent work (the four sweeps, row passes, cluster windows) runs
// on a small pool of non-blocking streams, each with its own workspace and
// engine, forked from and joined back to the caller's stream with events.
// ---------------------------------------------------------------------------
// Number of lanes: PEPS_LANES (1..64) if set, else 4.
int lane_count() {
  static int n = [] {
    const char* e = std::getenv("PEPS_LANES");
    const int v = e ? std::atoi(e) : 4;
    return v < 1 ? 1 : (v > 64 ? 64 : v);
  }();
  return n;
}

int lanes_of(const Tune& t) { return t.lanes > 0 ? std::min(t.lanes, 64) : lane_count(); }

// Non-blocking streams of the lanes (set 0) and their second streams (set 1),
// created once per device and kept: a recorded graph may have used them.
std::vector<cudaStream_t>& lane_streams(int n, int set = 0) {
  static std::mutex mu;
  static std::vector<std::vector<cudaStream_t>> pool_sets[2];
  auto& pool = pool_sets[set];
  std::lock_guard<std::mutex> g(mu);
  int dev = 0;
  PEPS_CUDA(cudaGetDevice(&dev));
  if (int(pool.size()) <= dev) pool.resize(dev + 1);
  auto& v = pool[dev];
  while (int(v.size()) < n) {
    cudaStream_t s;
    PEPS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    v.push_back(s);
  }
  return v;
}

void stream_after(cudaStream_t waiter, cudaStream_t producer) {
  cudaEvent_t e;
  PEPS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  PEPS_CUDA(cudaEventRecord(e, producer));
  PEPS_CUDA(cudaStreamWaitEvent(waiter, e, 0));
  PEPS_CUDA(cudaEventDestroy(e));
}

struct Lane {
  cudaStream_t st;
  std::unique_ptr<Arena> ws;
  std::unique_ptr<Ctx> cx;
  std::unique_ptr<Engine> eng;
};

struct Lanes {
  cudaStream_t main;
  std::vector<Lane> l;
  // nb: problems each lane's engine runs in lockstep.
  Lanes(Call& c, const Opts& opt, int d, int D, int Lmax, int nb = 1) : main(c.st) {
    const int nl = lanes_of(c.tune);
    auto& pool = lane_streams(nl);
    l.resize(nl);
    for (int i = 0; i < int(l.size()); ++i) {
      Lane& a = l[i];
      a.st = pool[i];
      stream_after(a.st, main);
      a.ws = std::make_unique<Arena>(a.st);
      a.cx = std::make_unique<Ctx>(a.st, a.ws.get());
      a.cx->flag = c.cx.flag;
      a.cx->persist = c.cx.persist;
      a.cx->qr_cmax = c.cx.qr_cmax;
      a.cx->svd_cap = c.cx.svd_cap;
      a.cx->cu0_cap = c.cx.cu0_cap;
      a.cx->tmp = a.ws->dalloc(8);
      a.eng = std::make_unique<Engine>(*a.cx, opt, d, D, Lmax, nb);
      if (nb == 1) a.eng->enable_dual(lane_streams(nl, 1)[i]);
    }
  }
  // Fork: every lane waits for the caller's stream.
  void fork() {
    for (auto& a : l) stream_after(a.st, main);
  }
  // Join: the caller's stream waits for every lane.
  void join() {
    for (auto& a : l) stream_after(main, a.st);
  }
  ~Lanes() {
    // Lane workspaces are freed on their own streams after their work, and
    // the caller's stream waits for those frees too (a recorded graph must
    // end with every lane joined back).
    for (auto& a : l) {
      a.eng.reset();
      a.cx.reset();
      a.ws.reset();
      cudaEvent_t e;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(e, a.st);
        cudaStreamWaitEvent(main, e, 0);
        cudaEventDestroy(e);
      }
    }
  }
};

// Runs fn(lane, job) for every job in plan[lane] (by default lane i takes
// jobs i, i+n, ...); one host thread per lane, so every lane's stream is fed
// while the others block on a full launch queue.  The first exception of any
// lane is rethrown.
template <class F>
void run_lanes(Lanes& lanes, int njobs, F fn, const std::vector<std::vector<int>>* plan = nullptr) {
  const int nl = int(lanes.l.size());
  if (nl == 1) {
    for (int j = 0; j < njobs; ++j) fn(lanes.l[0], j);
    return;
  }
  int dev = 0;
  PEPS_CUDA(cudaGetDevice(&dev));
  std::vector<std::exception_ptr> errs(nl);
  std::vector<std::thread> th;
  for (int i = 0; i < nl; ++i)
    th.emplace_back([&, i] {
      try {
        PEPS_CUDA(cudaSetDevice(dev));
        if (plan)
          for (int j : (*plan)[i]) fn(lanes.l[i], j);
        else
          for (int j = i; j < njobs; j += nl) fn(lanes.l[i], j);
      } catch (...) {
        errs[i] = std::current_exception();
      }
    });
  for (auto& t : th) t.join();
  for (auto& e : errs)
    if (e) std::rethrow_exception(e);
}

// Boundaries published by the sweeps as they are produced: the host waits on
// the condition variable for the Mps, the device on the event recorded after it.
struct Published {
  std::mutex mu;
  std::condition_variable cv;
  std::vector<Mps> b[4];
  std::vector<cudaEvent_t> ev[4];
  std::vector<char> ready[4];
  std::exception_ptr failed;
  ~Published() {
    for (auto& v : ev)
      for (cudaEvent_t e : v)
        if (e) cudaEventDestroy(e);
  }
  void put(int o, int y, const Mps& m, cudaStream_t st) {
    cudaEvent_t e;
    PEPS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    PEPS_CUDA(cudaEventRecord(e, st));
    std::lock_guard<std::mutex> g(mu);
    b[o][y] = m;
    ev[o][y] = e;
    ready[o][y] = 1;
    cv.notify_all();
  }
  void fail(std::exception_ptr p) {
    std::lock_guard<std::mutex> g(mu);
    if (!failed) failed = p;
    cv.notify_all();
  }
  // Host: block until boundary (o, y) exists; device: make st wait for it.
  const Mps& get(int o, int y, cudaStream_t st) {
    std::unique_lock<std::mutex> g(mu);
    cv.wait(g, [&] { return ready[o][y] || failed; });
    if (!ready[o][y]) throw Error(PEPS_ECUDA, "a boundary sweep failed");
    PEPS_CUDA(cudaStreamWaitEvent(st, ev[o][y], 0));
    return b[o][y];
  }
};

void full_env(Call& c, const peps_lattice* lat, const Opts& opt, peps_env* env, Oriented& ori) {
  Ctx& cx = c.cx;
  Arena& keep = *env->arena;
  const int Ly = lat->Ly, Lx = lat->Lx, d = lat->d;
  double* lnacc = cx.ws->dalloc(4);
  fill(cx, lnacc, 4, 0.0);
  Lanes lanes(c, opt, d, lat->D, std::max(Ly, Lx));
  const int nl = int(lanes.l.size());
  // PEPS_VERBOSE (plain calls only): device time of the whole set
  cudaEvent_t ph[2] = {};
  const bool timed = std::getenv("PEPS_VERBOSE") && !cx.persist;
  if (timed) {
    for (auto& e : ph) PEPS_CUDA(cudaEventCreate(&e));
    PEPS_CUDA(cudaEventRecord(ph[0], c.st));
  }
  EnvData& e = env->data;
  const long long d2 = (long long)d * d, d4 = d2 * d2;
  const int ncol = Ly > 1 ? Lx : 0;
  // Jobs: 0..3 the four directional sweeps; then row passes (Ly), column
  // passes (ncol) and the norm.  A pass starts as soon as its two boundaries
  // exist (a wavefront: the middle rows first), overlapping the sweeps.
  Published pub;
  for (int o = 0; o < 4; ++o) {
    const int n = (o < 2 ? Ly : Lx);
    pub.b[o].resize(n);
    pub.ev[o].assign(n, nullptr);
    pub.ready[o].assign(n, 0);
  }
  const int njobs = 4 + Ly + ncol + 1;
  std::vector<std::vector<int>> plan(nl);
  {
    // Static plan: every lane runs its sweeps before any pass (so no pass
    // waits on work queued behind it).  Passes go, in order of readiness, to
    // the lane free earliest; a sweep costs ~8 passes, a pass is ready when
    // the later of its two boundaries is (fraction of a sweep).
    const double S = 8.0;
    std::vector<double> avail(nl, 0.0);
    for (int o = 0; o < 4; ++o) {
      plan[o % nl].push_back(o);
      avail[o % nl] += S;
    }
    std::vector<std::pair<double, int>> passes;
    for (int y = 0; y < Ly; ++y)
      passes.push_back({S * std::max(y, Ly - 1 - y) / std::max(1, Ly - 1), 4 + y});
    for (int x = 0; x < ncol; ++x)
      passes.push_back({S * std::max(x, Lx - 1 - x) / std::max(1, Lx - 1), 4 + Ly + x});
    passes.push_back({S, 4 + Ly + ncol});
    std::stable_sort(passes.begin(), passes.end());
    for (auto& pj : passes) {
      int best = 0;
      double bt = 1e300;
      for (int li = 0; li < nl; ++li) {
        const double t = std::max(avail[li], pj.first) + 1.0;
        if (t < bt) {
          bt = t;
          best = li;
        }
      }
      plan[best].push_back(pj.second);
      avail[best] = bt;
    }
  }
  run_lanes(lanes, njobs, [&](Lane& L, int job) {
    if (job < 4) {
      const int o = job;
      try {
        L.eng->sweep(ori.o[o], o, (o < 2 ? Ly : Lx) - 1, lnacc + o, keep,
                     [&](int y, const Mps& m) { pub.put(o, y, m, L.st); });
      } catch (...) {
        pub.fail(std::current_exception());
        throw;
      }
    } else if (job < 4 + Ly) {
      const int y = job - 4;
      const Mps& T = pub.get(0, y, L.st);
      const Mps& B = pub.get(1, Ly - 1 - y, L.st);
      Engine::Targets ts, tb;
      for (int x = 0; x < Lx; ++x) ts.push_back({x, e.rho_site + ((long long)y * Lx + x) * d2});
      for (int x = 0; x + 1 < Lx; ++x) tb.push_back({x, e.rho_h + ((long long)y * (Lx - 1) + x) * d4});
      L.eng->row_rhos(ori.o[0], T, B, y, ts, tb);
    } else if (job < 4 + Ly + ncol) {
      // row x of the transposed lattice holds the vertical bonds (y,x)-(y+1,x) at its column y
      const int x = job - 4 - Ly;
      const Mps& T = pub.get(2, x, L.st);
      const Mps& B = pub.get(3, Lx - 1 - x, L.st);
      Engine::Targets tb;
      for (int y = 0; y + 1 < Ly; ++y) tb.push_back({y, e.rho_v + ((long long)y * Lx + x) * d4});
      L.eng->row_rhos(ori.o[2], T, B, x, {}, tb);
    } else {
      const Mps& T = pub.get(0, Ly - 1, L.st);
      L.eng->norm_from_top(ori.o[0], T, lnacc, e.lnnorm);
    }
  }, &plan);
  lanes.join();
  if (timed) {
    PEPS_CUDA(cudaEventRecord(ph[1], c.st));
    PEPS_CUDA(cudaEventSynchronize(ph[1]));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ph[0], ph[1]);
    std::fprintf(stderr, "[peps] full env: %.2f ms on the device\n", ms);
    for (auto& ev : ph) cudaEventDestroy(ev);
  }
  e.has_norm = true;
}

// Window of the cluster scheme (Section 5.3): n x n around (i) clipped at [0, L).
std::pair<int, int> window(int L, int i, int n) {
  const int h = (n + 1) / 2;
  const int lo = i - h + 1;
  return {std::max(lo, 0), std::min(lo + n - 1, L - 1)};
}

OLat sub(const OLat& f, int r0, int r1, int c0, int c1) {
  OLat s;
  s.Ly = r1 - r0 + 1;
  s.Lx = c1 - c0 + 1;
  s.d = f.d;
  for (int r = r0; r <= r1; ++r)
    for (int c = c0; c <= c1; ++c) s.sites.push_back(f.at(r, c));
  return s;
}

// CU_0 separable boundaries from all four sides (one CTA per side): sig[o] is
// [L_o][W_o][D*D], matrix (r, x) on the up legs of row r of orientation o.
void cu0_all_sides(Ctx& cx, const peps_lattice* lat, Oriented& ori, Arena& keep, double* sig[4]) {
  const int Ly = lat->Ly, Lx = lat->Lx, d = lat->d, D = lat->D, DM2 = D * D;
  Cu0Lattice cl[4];
  std::vector<std::vector<long long>> offs(4);
  std::vector<std::vector<int>> dims(4);
  double* closure_ones = cx.ws->dalloc(size_t(std::max(Ly, Lx)) * DM2);
  fill(cx, closure_ones, (long long)std::max(Ly, Lx) * DM2, 1.0);   // 1x1 closures read entry 0
  for (int o = 0; o < 4; ++o) {
    const OLat& L = ori.o[o];
    sig[o] = keep.dalloc(size_t(L.Ly) * L.Lx * DM2);
    offs[o].resize(size_t(L.Ly) * L.Lx);
    dims[o].resize(size_t(L.Ly) * L.Lx * 4);
    const double* base = L.sites[0].p.d(0);
    for (size_t i = 0; i < L.sites.size(); ++i) {
      offs[o][i] = L.sites[i].p.d(0) - base;
      dims[o][4 * i + 0] = L.sites[i].du;
      dims[o][4 * i + 1] = L.sites[i].dl;
      dims[o][4 * i + 2] = L.sites[i].dn;
      dims[o][4 * i + 3] = L.sites[i].dr;
    }
    auto* doff = static_cast<const long long*>(stage(cx, offs[o].data(), sizeof(long long) * offs[o].size()));
    auto* ddim = static_cast<const int*>(stage(cx, dims[o].data(), sizeof(int) * dims[o].size()));
    Cu0Lattice& q = cl[o];
    q.Ly = L.Ly;
    q.Lx = L.Lx;
    q.d = d;
    q.Dmax = D;
    q.A = base;
    q.off = doff;
    q.dims = ddim;
    q.top = closure_ones;
    q.left = closure_ones;
    q.right = closure_ones;
    q.out = sig[o];
    q.work = cx.ws->dalloc(cu0_work_size(L.Lx, d, D));
    q.max_half = std::max(1, cx.cu0_cap);
    q.tol = 1e-13;
  }
  cu0_launch(cx, cl, 4);
}

// ln|<P|Q>| and its sign into out[0], out[1] (device, FP64): transfer
// matrices from the left, each rescaled to unit norm with the logs summed.
void mps_ln_overlap(Ctx& cx, const Mps& P, const Mps& Q, double* out) {
  const int L = int(P.p.size());
  PEPS_REQUIRE(L == int(Q.p.size()) && L >= 1, "internal: overlap of MPS of different lengths");
  size_t maxE = 1, maxT = 1;
  for (int x = 0; x < L; ++x) {
    maxE = std::max(maxE, size_t(P.dims[x][3]) * Q.dims[x][3]);
    maxT = std::max(maxT, size_t(Q.dims[x][0]) * P.dims[x][1] * P.dims[x][2] * P.dims[x][3]);
  }
  double* lnacc = cx.ws->dalloc(2);
  fill(cx, lnacc, 2, 0.0);
  double* E = cx.ws->dalloc(maxE);
  double* E2 = cx.ws->dalloc(maxE);
  double* T = cx.ws->dalloc(maxT);
  fill(cx, E, 1, 1.0);
  Dims ed = {1, 1};
  for (int x = 0; x < L; ++x) {
    PEPS_REQUIRE(P.dims[x][1] == Q.dims[x][1] && P.dims[x][2] == Q.dims[x][2], "internal: overlap legs");
    const Dims td = ein_dims("ab,auvc->buvc", ed, P.dims[x]);
    ein(cx, "ab,auvc->buvc", E, ed, P.p[x], P.dims[x], T);
    const Dims nd = ein_dims("buvc,buvd->cd", td, Q.dims[x]);
    ein(cx, "buvc,buvd->cd", T, td, Q.p[x], Q.dims[x], E2);
    if (x + 1 < L) normalize(cx, E2, (long long)numel(nd), lnacc, lnacc + 1);
    std::swap(E, E2);
    ed = nd;
  }
  finish_norm(cx, lnacc, 1, nullptr, E, out, out + 1);
}

// Rim positions (orientation o, cut r >= 1, column x), in that order.
std::vector<RimSite> rim_sites(const Oriented& ori, double* const sig[4], int D) {
  std::vector<RimSite> v;
  for (int o = 0; o < 4; ++o) {
    const OLat& L = ori.o[o];
    for (int r = 1; r < L.Ly; ++r)
      for (int x = 0; x < L.Lx; ++x) {
        const SiteT& t = L.at(r - 1, x);
        v.push_back(RimSite{t.p.d(0), t.du, t.dl, t.dn, t.dr, sig[o] + ((long long)r * L.Lx + x) * D * D});
      }
  }
  return v;
}

// Windows of the anchors with row-major index in [a0, a1) (a1 < 0: all).
// Tensor update of a set of bonds (Section 2: the gate's action refit by ALS
// on the reduced tensors), every bond from the full environment of the input
// state -- the bonds of one Trotter set updated independently, the parallel
// schedule of Sections 4.4 and 5.2.  Horizontal bonds use the row sweeps,
// vertical bonds the column sweeps (rows of the transposed lattice); only the
// boundaries the bonds' rows need are computed.
// delta < 0: the full environment (FU).  delta >= 0: the cluster update
// CU_delta (Section 5): a row's bonds see the exact contraction of the rows
// within distance delta of it (all columns), closed above and below by the
// CU_0 separable boundaries of Section 5.1; a column's bonds likewise.
void bond_update(Call& c, const peps_lattice* lat, const Opts& opt, const double* gate_host, const int* bonds,
                 int nb, int iters, void* out, double* cost_host, Oriented& ori, int delta = -1) {
  Ctx& cx = c.cx;
  const int Ly = lat->Ly, Lx = lat->Lx, d = lat->d, D = lat->D;
  struct Job {
    int o = 0, r = 0, c = 0, y1 = 0, x1 = 0, y2 = 0, x2 = 0;
    int kl = 0, kr = 0, Do = 0, Dn = 0, ml = 0, mr = 0;
    SiteT L, R;
    Engine::BondNorm bn;
    double *al_new = nullptr, *ar_new = nullptr, *q = nullptr, *nl = nullptr, *nr = nullptr;
  };
  std::vector<Job> jobs(nb);
  int up[4] = {-1, -1, -1, -1};
  std::map<std::pair<int, int>, std::vector<int>> rows;
  for (int i = 0; i < nb; ++i) {
    Job& j = jobs[i];
    const int kind = bonds[3 * i], y = bonds[3 * i + 1], x = bonds[3 * i + 2];
    j.o = kind == 0 ? 0 : 2;
    j.r = kind == 0 ? y : x;
    j.c = kind == 0 ? x : y;
    j.y1 = y;
    j.x1 = x;
    j.y2 = kind == 0 ? y : y + 1;
    j.x2 = kind == 0 ? x + 1 : x;
    const OLat& ol = ori.o[j.o];
    j.L = ol.at(j.r, j.c);
    j.R = ol.at(j.r, j.c + 1);
    j.ml = j.L.du * j.L.dl * j.L.dn;
    j.mr = j.R.du * j.R.dn * j.R.dr;
    j.kl = std::min(j.ml, d * j.L.dr);
    j.kr = std::min(j.mr, d * j.R.dl);
    j.Do = j.L.dr;
    j.Dn = std::min({D, j.kl * d, j.kr * d});
    PEPS_REQUIRE(j.kl * j.Dn <= kCholMax && j.kr * j.Dn <= kCholMax,
                 "bond update: a reduced system has more than " + std::to_string(kCholMax) +
                     " unknowns per physical value (d*D*D too large)");
    Engine::BondNorm& b = j.bn;
    b.x = j.c;
    b.ml = cx.ws->dalloc(size_t(j.ml) * d * j.L.dr);
    b.mr = cx.ws->dalloc(size_t(j.mr) * d * j.R.dl);
    b.xl = cx.ws->dalloc(size_t(j.kl) * j.ml);
    b.xr = cx.ws->dalloc(size_t(j.kr) * j.mr);
    b.al = cx.ws->dalloc(size_t(j.kl) * d * j.L.dr);
    b.ar = cx.ws->dalloc(size_t(j.kr) * d * j.R.dl);
    b.N = cx.ws->dalloc(size_t(j.kl) * j.kr * j.kl * j.kr);
    j.al_new = cx.ws->dalloc(size_t(j.kl) * d * j.Dn);
    j.ar_new = cx.ws->dalloc(size_t(j.Dn) * d * j.kr);
    j.q = cx.ws->dalloc(2);
    j.nl = cx.ws->dalloc(size_t(d) * j.ml * j.Dn);
    j.nr = cx.ws->dalloc(size_t(d) * j.R.du * j.Dn * j.R.dn * j.R.dr);
    const int H = j.o == 0 ? Ly : Lx;
    up[j.o] = std::max(up[j.o], j.r);
    up[j.o + 1] = std::max(up[j.o + 1], H - 1 - j.r);
    rows[{j.o, j.r}].push_back(i);
  }
  double* gate = static_cast<double*>(stage(cx, gate_host, sizeof(double) * d * d * d * d));
  double* lnacc = cx.ws->dalloc(4);
  fill(cx, lnacc, 4, 0.0);
  Arena keep(c.st, size_t(64) << 20, /*async=*/false);
  if (delta >= 0) {
    // CU_delta: one strip per row (orientation 0) or column (orientation 2)
    // holding bonds, each with its own two short sweeps, on the lanes
    double* sig[4];
    cu0_all_sides(cx, lat, ori, keep, sig);
    const int DM2 = D * D;
    auto S = [&](int o, int r, int x, int dim) {
      const OLat& L = ori.o[o];
      return Mat{TP(sig[o] + ((long long)r * L.Lx + x) * DM2), dim};
    };
    std::vector<std::pair<int, int>> row_keys;
    for (auto& kv : rows) row_keys.push_back(kv.first);
    Lanes lanes(c, opt, d, D, std::max(Ly, Lx));
    const int nl = int(lanes.l.size());
    double* lnj = cx.ws->dalloc(size_t(nl) * 64);
    run_lanes(lanes, int(row_keys.size()), [&](Lane& L, int job) {
      const int o = row_keys[job].first, r = row_keys[job].second;
      const int H = o == 0 ? Ly : Lx, W = o == 0 ? Lx : Ly;
      const int r0 = std::max(0, r - delta), r1 = std::min(H - 1, r + delta), h = r1 - r0 + 1, rr = r - r0;
      OLat S0 = sub(ori.o[o], r0, r1, 0, W - 1);
      OLat S1 = sub(ori.o[o + 1], H - 1 - r1, H - 1 - r0, 0, W - 1);
      for (int j = 0; j < W; ++j) {
        S0.top.push_back(S(o, r0, j, S0.at(0, j).du));
        S0.bottom.push_back(S(o + 1, H - 1 - r1, j, S0.at(h - 1, j).dn));
      }
      for (int i = 0; i < h; ++i) {
        S0.left.push_back(ori.o[o].left[r0 + i]);
        S0.right.push_back(ori.o[o].right[r0 + i]);
      }
      S1.top = S0.bottom;
      S1.bottom = S0.top;
      for (int i = 0; i < h; ++i) {
        S1.left.push_back(S0.left[h - 1 - i]);
        S1.right.push_back(S0.right[h - 1 - i]);
      }
      const int li = int(&L - lanes.l.data());
      double* lj = lnj + size_t(li) * 64;
      fill(*L.cx, lj, 2, 0.0);
      auto bt = L.eng->sweep(S0, o, rr, TP(lj), keep);
      auto bb = L.eng->sweep(S1, o + 1, h - 1 - rr, TP(lj + 1), keep);
      std::vector<Engine::BondNorm> bn;
      for (int i : rows[row_keys[job]]) bn.push_back(jobs[i].bn);
      L.eng->row_bond_norms(S0, bt[rr], bb[h - 1 - rr], rr, bn);
    });
    lanes.join();
  } else {
    Lanes lanes(c, opt, d, D, std::max(Ly, Lx));
    const int nl = int(lanes.l.size());
    Published pub;
    for (int o = 0; o < 4; ++o) {
      const int n = (o < 2 ? Ly : Lx);
      pub.b[o].resize(n);
      pub.ev[o].assign(n, nullptr);
      pub.ready[o].assign(n, 0);
    }
    // jobs: the needed sweeps first on every lane, then one job per row
    std::vector<int> sweeps;
    for (int o = 0; o < 4; ++o)
      if (up[o] >= 0) sweeps.push_back(o);
    std::vector<std::pair<int, int>> row_keys;
    for (auto& kv : rows) row_keys.push_back(kv.first);
    const int njobs = int(sweeps.size() + row_keys.size());
    std::vector<std::vector<int>> plan(nl);
    for (int i = 0; i < njobs; ++i) plan[i % nl].push_back(i);
    run_lanes(lanes, njobs, [&](Lane& L, int job) {
      if (job < int(sweeps.size())) {
        const int o = sweeps[job];
        try {
          L.eng->sweep(ori.o[o], o, up[o], lnacc + o, keep, [&](int y, const Mps& m) { pub.put(o, y, m, L.st); });
        } catch (...) {
          pub.fail(std::current_exception());
          throw;
        }
        return;
      }
      const auto key = row_keys[job - sweeps.size()];
      const int o = key.first, r = key.second, H = o == 0 ? Ly : Lx;
      const Mps& T = pub.get(o, r, L.st);
      const Mps& B = pub.get(o + 1, H - 1 - r, L.st);
      std::vector<Engine::BondNorm> bn;
      for (int i : rows[key]) bn.push_back(jobs[i].bn);
      L.eng->row_bond_norms(ori.o[o], T, B, r, bn);
    }, &plan);
    lanes.join();
  }
  // ALS per shape group (one batched sequence per group)
  std::map<std::array<int, 4>, std::vector<BondAls>> groups;
  for (auto& j : jobs) {
    BondAls a;
    a.N = j.bn.N;
    a.al = j.bn.al;
    a.ar = j.bn.ar;
    a.al_new = j.al_new;
    a.ar_new = j.ar_new;
    a.q = j.q;
    groups[{j.kl, j.kr, j.Do, j.Dn}].push_back(a);
  }
  for (auto& kv : groups)
    bond_als(cx, d, kv.first[0], kv.first[1], kv.first[2], kv.first[3], gate, kv.second, iters);
  // new site tensors A = X a, unit Frobenius norm, into the output lattice
  static const int perms[4][4] = {{0, 1, 2, 3}, {2, 1, 0, 3}, {1, 0, 3, 2}, {3, 0, 1, 2}};
  std::vector<SiteStore> st;
  for (auto& j : jobs) {
    ein(cx, "km,ksr->smr", TP(j.bn.xl), {j.kl, j.ml}, TP(j.al_new), {j.kl, d, j.Dn}, TP(j.nl));
    ein(cx, "kunr,ltk->tulnr", TP(j.bn.xr), {j.kr, j.R.du, j.R.dn, j.R.dr}, TP(j.ar_new), {j.Dn, d, j.kr},
        TP(j.nr));
    normalize(cx, TP(j.nl), (long long)d * j.ml * j.Dn, TP());
    normalize(cx, TP(j.nr), (long long)d * j.R.du * j.Dn * j.R.dn * j.R.dr, TP());
    SiteStore a, b;
    a.src = j.nl;
    a.y = j.y1;
    a.x = j.x1;
    const int da[5] = {d, j.L.du, j.L.dl, j.L.dn, j.Dn};
    const int db[5] = {d, j.R.du, j.Dn, j.R.dn, j.R.dr};
    std::memcpy(a.dims, da, sizeof(da));
    std::memcpy(a.perm, perms[j.o], sizeof(a.perm));
    b.src = j.nr;
    b.y = j.y2;
    b.x = j.x2;
    std::memcpy(b.dims, db, sizeof(db));
    std::memcpy(b.perm, perms[j.o], sizeof(b.perm));
    st.push_back(a);
    st.push_back(b);
  }
  const size_t bytes = size_t(Ly) * Lx * d * D * D * D * D * (lat->dtype == PEPS_F32 ? 4 : 8);
  if (out != lat->A) PEPS_CUDA(cudaMemcpyAsync(out, lat->A, bytes, cudaMemcpyDeviceToDevice, c.st));
  store_sites(cx, out, lat->dtype == PEPS_F32, Lx, d, D, st);
  if (cost_host) {
    std::vector<double> qh(size_t(2) * nb);
    for (int i = 0; i < nb; ++i)
      PEPS_CUDA(cudaMemcpyAsync(&qh[2 * i], jobs[i].q, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    PEPS_CUDA(cudaStreamSynchronize(c.st));
    for (int i = 0; i < nb; ++i) cost_host[i] = qh[2 * i + 1] > 0 ? qh[2 * i] / qh[2 * i + 1] : 0.0;
  }
}

void cluster_env(Call& c, const peps_lattice* lat, const Opts& opt, int n, peps_env* env, Oriented& ori,
                 const float* closure_w, long long a0 = 0, long long a1 = -1) {
  Ctx& cx = c.cx;
  const int Ly = lat->Ly, Lx = lat->Lx, d = lat->d, D = lat->D, DM2 = D * D;
  double* sig[4];
  cu0_all_sides(cx, lat, ori, *env->arena, sig);
  if (closure_w) {
    // learned closure: predict every rim matrix, keep CU_0 where the prediction is unusable
    MlpDims m;
    m.d = d;
    m.D = D;
    m.W = PEPS_CLOSURE_WIDTH;
    const std::vector<RimSite> rs = rim_sites(ori, sig, D);
    const long long ne = (long long)rs.size();
    float* X = cx.ws->falloc(size_t(ne) * m.F());
    float* P = cx.ws->falloc(size_t(ne) * m.out());
    closure_features(cx, m, rs.data(), ne, X);
    mlp_predict(cx, m, closure_w, X, ne, P);
    std::vector<double*> tg(ne);
    for (long long e = 0; e < ne; ++e) tg[e] = const_cast<double*>(rs[e].sigma);
    closure_apply(cx, D, P, tg.data(), ne);
  }
  auto S = [&](int o, int r, int x, int dim) {
    const OLat& L = ori.o[o];
    return Mat{TP(sig[o] + ((long long)r * L.Lx + x) * DM2), dim};
  };
  // Windows of one shape signature -- size, anchor position inside, and which
  // lattice edges they touch (which fixes every site's leg dimensions) -- run
  // as the problems of one engine, in chunks that fit the memory budget.
  struct Win {
    int y, x, r0, r1, c0, c1;
  };
  std::map<std::array<int, 8>, std::vector<Win>> groups;
  for (int y = 0; y < Ly; ++y)
    for (int x = 0; x < Lx; ++x) {
      const long long a = (long long)y * Lx + x;
      if (a < a0 || (a1 >= 0 && a >= a1)) continue;
      const auto rr = window(Ly, y, n), cc = window(Lx, x, n);
      const Win wv{y, x, rr.first, rr.second, cc.first, cc.second};
      const std::array<int, 8> key{wv.r1 - wv.r0, wv.c1 - wv.c0, y - wv.r0, x - wv.c0,
                                   int(wv.r0 == 0), int(wv.r1 == Ly - 1), int(wv.c0 == 0), int(wv.c1 == Lx - 1)};
      groups[key].push_back(wv);
    }
  const int nl = lanes_of(c.tune);
  const int Lwin = std::min(n, std::max(Ly, Lx));
  const size_t per = Engine::footprint(opt, d, D, Lwin) * sizeof(double);
  size_t free_b = 0, total_b = 0;
  PEPS_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const size_t budget = std::min<size_t>(free_b * 2 / 5, size_t(96) << 30);
  // Up to 16 windows per chunk by default (the autotuner also tries 8 and 32):
  // beyond that a launch gains little (its work is already bandwidth-bound)
  // while smaller chunks balance the lanes.
  const int cap = c.tune.chunk > 0 ? std::min(c.tune.chunk, MAXB) : 16;
  const int bmax = int(std::max<size_t>(1, std::min<size_t>(size_t(cap), budget / (per * nl))));
  std::vector<std::vector<Win>> chunks;
  for (auto& kv : groups) {
    const auto& v = kv.second;
    const int nch = int((v.size() + bmax - 1) / bmax);
    const int sz = int((v.size() + nch - 1) / nch);
    for (size_t i0 = 0; i0 < v.size(); i0 += sz)
      chunks.emplace_back(v.begin() + i0, v.begin() + std::min(v.size(), i0 + size_t(sz)));
  }
  // Longest chunk first onto the least-loaded lane.  Estimated device time of
  // a chunk: (window sites)^1.6 x (3 + B) / 4, fitted to measured chunk times
  // (one window pays the latency of every step; extra windows ride along).
  auto cost = [](const std::vector<Win>& v) {
    const double area = double(v[0].r1 - v[0].r0 + 1) * double(v[0].c1 - v[0].c0 + 1);
    return std::pow(area, 1.6) * (3.0 + double(v.size())) / 4.0;
  };
  std::stable_sort(chunks.begin(), chunks.end(),
                   [&](const std::vector<Win>& a, const std::vector<Win>& b) { return cost(a) > cost(b); });
  std::vector<std::vector<int>> plan(nl);
  {
    std::vector<double> load(nl, 0.0);
    for (int j = 0; j < int(chunks.size()); ++j) {
      const int li = int(std::min_element(load.begin(), load.end()) - load.begin());
      plan[li].push_back(j);
      load[li] += cost(chunks[j]);
    }
  }
  int bl = 1;
  for (auto& c : chunks) bl = std::max(bl, int(c.size()));
  Lanes lanes(c, opt, d, D, Lwin, bl);
  double* junk = cx.ws->dalloc(size_t(lanes.l.size()) * 4 * 32 * MAXB);
  EnvData& e = env->data;
  const long long d2 = (long long)d * d, d4 = d2 * d2;
  // Merge per-window lattices (identical shapes) into one lattice of pointer sets.
  auto merge = [](const std::vector<OLat>& ws) {
    OLat m = ws[0];
    const int B = int(ws.size());
    auto set = [&](TP& t, auto get) {
      t.n = B;
      for (int b = 0; b < B; ++b) t.p[b] = get(b).p[0];
    };
    for (size_t i = 0; i < m.sites.size(); ++i) set(m.sites[i].p, [&](int b) { return ws[b].sites[i].p; });
    for (size_t i = 0; i < m.top.size(); ++i) set(m.top[i].p, [&](int b) { return ws[b].top[i].p; });
    for (size_t i = 0; i < m.bottom.size(); ++i) set(m.bottom[i].p, [&](int b) { return ws[b].bottom[i].p; });
    for (size_t i = 0; i < m.left.size(); ++i) set(m.left[i].p, [&](int b) { return ws[b].left[i].p; });
    for (size_t i = 0; i < m.right.size(); ++i) set(m.right[i].p, [&](int b) { return ws[b].right[i].p; });
    return m;
  };
  run_lanes(lanes, int(chunks.size()), [&](Lane& lane, int job) {
    const std::vector<Win>& ch = chunks[job];
    const int B = int(ch.size());
    const int li = int(&lane - lanes.l.data());
    Engine& eng = *lane.eng;
    eng.use(B);
    const TP lj = strided(junk + size_t(li) * 4 * 32 * MAXB, B, 1);
    std::vector<OLat> w0(B), w1(B), w2(B), w3(B);
    TP t_site, t_h, t_v;
    t_site.n = t_h.n = t_v.n = B;
    for (int b = 0; b < B; ++b) {
      const Win& wv = ch[b];
      const int r0 = wv.r0, r1 = wv.r1, c0 = wv.c0, c1 = wv.c1;
      const int h = r1 - r0 + 1, w = c1 - c0 + 1;
      // window in the four orientations (sub-blocks of the oriented full lattice)
      OLat W0 = sub(ori.o[0], r0, r1, c0, c1);
      OLat W1 = sub(ori.o[1], Ly - 1 - r1, Ly - 1 - r0, c0, c1);
      OLat W2 = sub(ori.o[2], c0, c1, r0, r1);
      OLat W3 = sub(ori.o[3], Lx - 1 - c1, Lx - 1 - c0, r0, r1);
      for (int j = 0; j < w; ++j) {
        W0.top.push_back(S(0, r0, c0 + j, W0.at(0, j).du));
        W0.bottom.push_back(S(1, Ly - 1 - r1, c0 + j, W0.at(h - 1, j).dn));
      }
      for (int i = 0; i < h; ++i) {
        W0.left.push_back(S(2, c0, r0 + i, W0.at(i, 0).dl));
        W0.right.push_back(S(3, Lx - 1 - c1, r0 + i, W0.at(i, w - 1).dr));
      }
      W1.top = W0.bottom;
      W1.bottom = W0.top;
      for (int i = 0; i < h; ++i) {
        W1.left.push_back(W0.left[h - 1 - i]);
        W1.right.push_back(W0.right[h - 1 - i]);
      }
      W2.top = W0.left;
      W2.bottom = W0.right;
      W2.left = W0.top;
      W2.right = W0.bottom;
      W3.top = W0.right;
      W3.bottom = W0.left;
      for (int j = 0; j < w; ++j) {
        W3.left.push_back(W0.top[w - 1 - j]);
        W3.right.push_back(W0.bottom[w - 1 - j]);
      }
      w0[b] = std::move(W0);
      w1[b] = std::move(W1);
      w2[b] = std::move(W2);
      w3[b] = std::move(W3);
      t_site.p[b] = e.rho_site + ((long long)wv.y * Lx + wv.x) * d2;
      t_h.p[b] = e.rho_h + ((long long)wv.y * (Lx - 1) + wv.x) * d4;
      t_v.p[b] = e.rho_v + ((long long)wv.y * Lx + wv.x) * d4;
    }
    const Win& w_ = ch[0];
    const int h = w_.r1 - w_.r0 + 1, w = w_.c1 - w_.c0 + 1, yw = w_.y - w_.r0, xw = w_.x - w_.c0;
    const OLat W0 = merge(w0), W1 = merge(w1), W2 = merge(w2), W3 = merge(w3);
    // PEPS_VERBOSE (plain calls only): device time of every chunk
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    const bool timed = std::getenv("PEPS_VERBOSE") && !cx.persist;
    if (timed) {
      PEPS_CUDA(cudaEventCreate(&ev0));
      PEPS_CUDA(cudaEventCreate(&ev1));
      PEPS_CUDA(cudaEventRecord(ev0, lane.st));
    }
    Arena keep(lane.st);
    auto bt = eng.sweep(W0, 0, yw, lj, keep);
    auto bb = eng.sweep(W1, 1, h - 1 - yw, lj, keep);
    Engine::Targets ts{{xw, t_site}}, tb;
    if (xw + 1 < w) tb.push_back({xw, t_h});
    eng.row_rhos(W0, bt[yw], bb[h - 1 - yw], yw, ts, tb);
    if (yw + 1 < h) {
      auto bl = eng.sweep(W2, 2, xw, lj, keep);
      auto br = eng.sweep(W3, 3, w - 1 - xw, lj, keep);
      eng.row_rhos(W2, bl[xw], br[w - 1 - xw], xw, {}, {{yw, t_v}});
    }
    if (timed) {
      PEPS_CUDA(cudaEventRecord(ev1, lane.st));
      PEPS_CUDA(cudaEventSynchronize(ev1));
      float ms = 0.f;
      PEPS_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
      std::fprintf(stderr, "[peps] chunk %d: %d windows %dx%d anchor (%d,%d), lane %d, %.2f ms\n", job, B, h, w, yw,
                   xw, li, ms);
      cudaEventDestroy(ev0);
      cudaEventDestroy(ev1);
    }
  }, &plan);
  lanes.join();
  e.has_norm = false;
}

// The whole environment computation of one call, enqueued on c's stream.
void compute(Call& c, const peps_lattice* lat, const peps_opts* opts, const Opts& o, bool cluster, peps_env* env,
             long long a0 = 0, long long a1 = -1) {
  Oriented ori;
  build_orientations(c.cx, lat, *env->arena, ori);
  if (cluster)
    cluster_env(c, lat, o, opts->n, env, ori,
                opts->closure == PEPS_CLOSURE_LEARNED ? static_cast<const float*>(opts->closure_weights) : nullptr,
                a0, a1);
  else
    full_env(c, lat, o, env, ori);
}

int run_env(const peps_lattice* lat, const peps_opts* opts, peps_env** out, void* stream, bool cluster,
            long long a0 = 0, long long a1 = -1) {
  if (out) *out = nullptr;
  return guard([&] {
    PEPS_REQUIRE(out != nullptr, "out is NULL");
    require_device();
    check_lattice(lat);
    const Opts o = check_opts(opts, cluster);
    if (cluster && a1 >= 0)
      PEPS_REQUIRE(a0 >= 0 && a0 <= a1 && a1 <= (long long)lat->Ly * lat->Lx,
                   "anchor range must satisfy 0 <= begin <= end <= Ly*Lx");
    Call c(stream);
    auto env = new_env(lat, cluster ? 1 : 0, c.st);
    const auto t0 = std::chrono::steady_clock::now();
    compute(c, lat, opts, o, cluster, env.get(), a0, a1);
    const auto t1 = std::chrono::steady_clock::now();
    c.finish();
    if (std::getenv("PEPS_VERBOSE")) {
      const auto t2 = std::chrono::steady_clock::now();
      std::fprintf(stderr, "[peps] env: host enqueue %.1f ms, then device drain %.1f ms\n",
                   std::chrono::duration<double, std::milli>(t1 - t0).count(),
                   std::chrono::duration<double, std::milli>(t2 - t1).count());
    }
    *out = env.release();
  });
}

}  // namespace

// A recorded environment computation: the CUDA graph, the memory it writes
// its results and status into, and the kernel counts of one replay.
struct peps_plan {
  int device = 0;
  std::unique_ptr<Arena> persist;   // status word and staged shape data (outlives the recording)
  std::unique_ptr<peps_env> env;    // results, rewritten by every replay
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int* flag = nullptr;
  long long nodes = 0;
  long long kernels = 0;            // kernel nodes of the graph: kernels one replay launches
  int lanes = 0, qr_cmax = 0;       // launch configuration it was recorded with
  Counts counts;                    // kernel launches (and their flops) in one replay
};

namespace {

struct PlanDel {
  void operator()(peps_plan* p) const { peps_plan_free(p); }
};
using PlanPtr = std::unique_ptr<peps_plan, PlanDel>;

Opts plan_checks(const peps_lattice* lat, const peps_opts* opts, bool cl) {
  require_device();
  check_lattice(lat);
  PEPS_REQUIRE(lat->on_device, "a plan reads its lattice from device memory (on_device = 1)");
  return check_opts(opts, cl);
}

// One plain call validates the input and performs every one-time set-up
// (kernel attributes, cluster occupancy queries) outside any recording.
void validate_by_running(const peps_lattice* lat, const peps_opts* opts, bool cl, void* stream) {
  peps_env* probe = nullptr;
  const int rc = run_env(lat, opts, &probe, stream, cl);
  peps_env_free(probe);
  if (rc != PEPS_OK) throw Error(rc, g_err);
}

// Records the whole computation of one call, with launch configuration t, as a CUDA graph.
PlanPtr record_plan(const peps_lattice* lat, const peps_opts* opts, const Opts& o, bool cl, const Tune& t) {
  static std::mutex record_mu;   // one recording at a time (shared lane streams)
  std::lock_guard<std::mutex> lk(record_mu);
  PlanPtr plan(new peps_plan());
  PEPS_CUDA(cudaGetDevice(&plan->device));
  plan->lanes = lanes_of(t);
  plan->qr_cmax = t.qr_cmax;
  plan->persist = std::make_unique<Arena>(nullptr, size_t(1) << 20, /*async=*/false);
  cudaStream_t cs = nullptr;
  PEPS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  struct Cleanup {
    cudaStream_t s;
    ~Cleanup() {
      g_recording.store(nullptr);
      cudaStreamDestroy(s);
    }
  } cleanup{cs};
  g_recording.store(&plan->counts);
  PEPS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  try {
    Call c(cs, plan->persist.get(), t);
    plan->flag = c.cx.flag;
    plan->env = new_env(lat, cl ? 1 : 0, cs);
    compute(c, lat, opts, o, cl, plan->env.get());
  } catch (...) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(cs, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    throw;
  }
  PEPS_CUDA(cudaStreamEndCapture(cs, &plan->graph));
  g_recording.store(nullptr);
  size_t nodes = 0;
  PEPS_CUDA(cudaGraphGetNodes(plan->graph, nullptr, &nodes));
  plan->nodes = (long long)nodes;
  {
    std::vector<cudaGraphNode_t> all(nodes);
    size_t got = nodes;
    if (nodes) PEPS_CUDA(cudaGraphGetNodes(plan->graph, all.data(), &got));
    for (size_t i = 0; i < got; ++i) {
      cudaGraphNodeType ty;
      PEPS_CUDA(cudaGraphNodeGetType(all[i], &ty));
      if (ty == cudaGraphNodeTypeKernel) ++plan->kernels;
    }
  }
  const auto t0 = std::chrono::steady_clock::now();
  PEPS_CUDA(cudaGraphInstantiate(&plan->exec, plan->graph, 0));
  if (std::getenv("PEPS_VERBOSE"))
    std::fprintf(stderr, "[peps] plan: %zu graph nodes (%lld kernels), instantiated in %.1f ms\n", nodes,
                 plan->kernels,
                 std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
  return plan;
}

// Device time of one replay: one warm replay, then the best of `reps` (CUDA events on st).
double time_plan(peps_plan* p, cudaStream_t st, int reps) {
  cudaEvent_t e0, e1;
  PEPS_CUDA(cudaEventCreate(&e0));
  PEPS_CUDA(cudaEventCreate(&e1));
  double best = 1e300;
  cudaError_t err = cudaGraphLaunch(p->exec, st);
  for (int r = 0; r < reps && err == cudaSuccess; ++r) {
    cudaEventRecord(e0, st);
    err = cudaGraphLaunch(p->exec, st);
    cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) best = std::min(best, double(ms));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  PEPS_CUDA(err);
  Call::read_status(p->flag, st);
  return best;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace {

int bond_update_call(const peps_lattice* lat, const peps_opts* opts, int delta, const double* gate, const int* bonds,
                     int nbonds, int als_iters, void* A_out, double* cost, void* cuda_stream) {
  return guard([&] {
    require_device();
    check_lattice(lat);
    const Opts o = check_opts(opts, false);
    PEPS_REQUIRE(lat->on_device, "the bond update reads and writes device lattices (on_device = 1)");
    PEPS_REQUIRE(gate != nullptr && bonds != nullptr && A_out != nullptr, "gate, bonds and A_out must be non-NULL");
    PEPS_REQUIRE(nbonds >= 1, "nbonds must be >= 1");
    PEPS_REQUIRE(als_iters >= 1 && als_iters <= 1000, "als_iters must be in [1, 1000]");
    const int d = lat->d, d4 = d * d * d * d;
    for (int i = 0; i < d4; ++i) PEPS_REQUIRE(std::isfinite(gate[i]), "the gate has a non-finite entry");
    std::vector<char> used(size_t(lat->Ly) * lat->Lx, 0);
    for (int i = 0; i < nbonds; ++i) {
      const int kind = bonds[3 * i], y = bonds[3 * i + 1], x = bonds[3 * i + 2];
      PEPS_REQUIRE(kind == 0 || kind == 1, "bond kind must be 0 (horizontal) or 1 (vertical)");
      const int y2 = kind == 0 ? y : y + 1, x2 = kind == 0 ? x + 1 : x;
      PEPS_REQUIRE(y >= 0 && x >= 0 && y2 < lat->Ly && x2 < lat->Lx, "bond outside the lattice");
      char& a = used[size_t(y) * lat->Lx + x];
      char& b = used[size_t(y2) * lat->Lx + x2];
      PEPS_REQUIRE(!a && !b, "two bonds of one call share a site");
      a = b = 1;
    }
    cudaPointerAttributes at;
    PEPS_CUDA(cudaPointerGetAttributes(&at, A_out));
    PEPS_REQUIRE(at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged, "A_out is not a device pointer");
    Call c(cuda_stream);
    Arena keep(c.st, size_t(64) << 20, /*async=*/false);
    Oriented ori;
    build_orientations(c.cx, lat, keep, ori);
    bond_update(c, lat, o, gate, bonds, nbonds, als_iters, A_out, cost, ori, delta);
    c.finish();
  });
}
}  // namespace

namespace {

// Checkpoint files: one JSON header line padded with spaces to kCkptHeader
// bytes, then the arrays as raw little-endian values.
constexpr size_t kCkptHeader = 512;

void ckpt_write(const char* path, const std::string& json, const std::vector<std::pair<const void*, size_t>>& parts) {
  PEPS_REQUIRE(path != nullptr, "path is NULL");
  PEPS_REQUIRE(json.size() + 1 <= kCkptHeader, "internal: checkpoint header too long");
  std::string hdr = json;
  hdr.resize(kCkptHeader - 1, ' ');
  hdr.push_back('\n');
  FILE* f = std::fopen(path, "wb");
  PEPS_REQUIRE(f != nullptr, std::string("cannot open ") + path + " for writing");
  bool ok = std::fwrite(hdr.data(), 1, hdr.size(), f) == hdr.size();
  for (auto& p : parts) ok = ok && (p.second == 0 || std::fwrite(p.first, 1, p.second, f) == p.second);
  ok = (std::fclose(f) == 0) && ok;
  PEPS_REQUIRE(ok, std::string("writing ") + path + " failed");
}

struct CkptIn {
  std::string hdr;
  std::vector<char> body;
};

CkptIn ckpt_read(const char* path, const char* format) {
  PEPS_REQUIRE(path != nullptr, "path is NULL");
  FILE* f = std::fopen(path, "rb");
  PEPS_REQUIRE(f != nullptr, std::string("cannot open ") + path);
  CkptIn c;
  c.hdr.resize(kCkptHeader);
  const bool ok = std::fread(&c.hdr[0], 1, kCkptHeader, f) == kCkptHeader;
  if (ok) {
    char buf[1 << 16];
    size_t r;
    while ((r = std::fread(buf, 1, sizeof(buf), f)) > 0) c.body.insert(c.body.end(), buf, buf + r);
  }
  std::fclose(f);
  PEPS_REQUIRE(ok, std::string(path) + " is shorter than a checkpoint header");
  PEPS_REQUIRE(c.hdr.find(std::string("\"format\":\"") + format + "\"") != std::string::npos,
               std::string(path) + " is not a " + format + " checkpoint");
  return c;
}

long long ckpt_int(const std::string& hdr, const char* key) {
  const std::string k = std::string("\"") + key + "\":";
  const size_t at = hdr.find(k);
  PEPS_REQUIRE(at != std::string::npos, std::string("checkpoint header lacks ") + key);
  char* end = nullptr;
  const long long v = std::strtoll(hdr.c_str() + at + k.size(), &end, 10);
  PEPS_REQUIRE(end != hdr.c_str() + at + k.size(), std::string("checkpoint header: bad value for ") + key);
  return v;
}

}  // namespace

extern "C" {

int peps_env_full(const peps_lattice* lat, const peps_opts* opts, peps_env** out, void* cuda_stream) {
  return run_env(lat, opts, out, cuda_stream, false);
}

int peps_env_cluster(const peps_lattice* lat, const peps_opts* opts, peps_env** out, void* cuda_stream) {
  return run_env(lat, opts, out, cuda_stream, true);
}

int peps_env_cluster_range(const peps_lattice* lat, const peps_opts* opts, long long anchor_begin,
                           long long anchor_end, peps_env** out, void* cuda_stream) {
  if (anchor_end < 0) {
    if (out) *out = nullptr;
    return fail(PEPS_EINVAL, "anchor range must satisfy 0 <= begin <= end <= Ly*Lx");
  }
  return run_env(lat, opts, out, cuda_stream, true, anchor_begin, anchor_end);
}

int peps_ipeps_cluster(const double* A, int d, int D, int on_device, const peps_opts* opts, double* rho_site,
                       double* rho_h, double* rho_v, double* sigma, void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(A != nullptr && rho_site != nullptr && rho_h != nullptr && rho_v != nullptr, "NULL argument");
    PEPS_REQUIRE(d >= 1 && d <= 4 && D >= 1 && D <= 16, "d must be in [1, 4] and D in [1, 16]");
    require_device();
    const Opts o = check_opts(opts, true);
    PEPS_REQUIRE(opts->closure == PEPS_CLOSURE_PLAIN, "the infinite lattice uses the plain CU_0 closure");
    PEPS_REQUIRE(opts->n <= 64, "window size n must be <= 64");
    const int n = opts->n;
    Call c(cuda_stream);
    Arena keep(c.st);
    // The tensor at the centre of a 3x3 OBC lattice has every leg of dimension
    // D in all four orientations: its oriented copies are the window's sites.
    const size_t per = size_t(d) * D * D * D * D;
    double* dense = keep.dalloc(9 * per);
    PEPS_CUDA(cudaMemsetAsync(dense, 0, 9 * per * sizeof(double), c.st));
    PEPS_CUDA(cudaMemcpyAsync(dense + 4 * per, A, per * sizeof(double),
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c.st));
    const peps_lattice l3{3, 3, d, D, PEPS_F64, dense, 1};
    Oriented ori;
    build_orientations(c.cx, &l3, keep, ori);
    const SiteT* ctr[4];
    const double* ca[4];
    for (int k = 0; k < 4; ++k) {
      ctr[k] = &ori.o[k].at(1, 1);
      ca[k] = ctr[k]->p.d(0);
    }
    double* sig = keep.dalloc(size_t(4) * D * D);
    cu0_infinite(c.cx, ca, d, D, sig, 25 * c.cx.cu0_cap);
    // n x n window of copies, closed by the four boundaries (corners dropped);
    // orientation k sees side s of the window as side map[k][s] of W0
    auto side = [&](int s) { return Mat{TP(sig + size_t(s) * D * D), D}; };
    static const int map[4][4] = {{0, 1, 2, 3}, {1, 0, 2, 3}, {2, 3, 0, 1}, {3, 2, 0, 1}};
    OLat W[4];
    for (int k = 0; k < 4; ++k) {
      W[k].Ly = W[k].Lx = n;
      W[k].d = d;
      W[k].sites.assign(size_t(n) * n, *ctr[k]);
      W[k].top.assign(n, side(map[k][0]));
      W[k].bottom.assign(n, side(map[k][1]));
      W[k].left.assign(n, side(map[k][2]));
      W[k].right.assign(n, side(map[k][3]));
    }
    const int a = (n + 1) / 2 - 1;
    const long long d2 = (long long)d * d, d4 = d2 * d2;
    double* out = keep.dalloc(size_t(d2 + 2 * d4));
    fill(c.cx, out, d2 + 2 * d4, 0.0);
    double* lnj = keep.dalloc(4);
    fill(c.cx, lnj, 4, 0.0);
    {
      Engine eng(c.cx, o, d, D, n);
      auto bt = eng.sweep(W[0], 0, a, TP(lnj), keep);
      auto bb = eng.sweep(W[1], 1, n - 1 - a, TP(lnj), keep);
      Engine::Targets tb;
      if (a + 1 < n) tb.push_back({a, TP(out + d2)});
      eng.row_rhos(W[0], bt[a], bb[n - 1 - a], a, {{a, TP(out)}}, tb);
      if (a + 1 < n) {
        auto bl = eng.sweep(W[2], 2, a, TP(lnj), keep);
        auto br = eng.sweep(W[3], 3, n - 1 - a, TP(lnj), keep);
        eng.row_rhos(W[2], bl[a], br[n - 1 - a], a, {}, {{a, TP(out + d2 + d4)}});
      }
    }
    PEPS_CUDA(cudaMemcpyAsync(rho_site, out, sizeof(double) * d2, cudaMemcpyDeviceToHost, c.st));
    PEPS_CUDA(cudaMemcpyAsync(rho_h, out + d2, sizeof(double) * d4, cudaMemcpyDeviceToHost, c.st));
    PEPS_CUDA(cudaMemcpyAsync(rho_v, out + d2 + d4, sizeof(double) * d4, cudaMemcpyDeviceToHost, c.st));
    if (sigma)
      PEPS_CUDA(cudaMemcpyAsync(sigma, sig, sizeof(double) * 4 * D * D, cudaMemcpyDeviceToHost, c.st));
    c.finish();
  });
}

int peps_set_iteration_caps(int cu0_half_sweeps, int jacobi_sweeps) {
  return guard([&] {
    PEPS_REQUIRE(cu0_half_sweeps >= 0 && cu0_half_sweeps <= 1000000 && jacobi_sweeps >= 0 &&
                     jacobi_sweeps <= 1000000,
                 "iteration caps must be in [0, 1e6] (0 restores the default)");
    g_cap_cu0.store(cu0_half_sweeps == 0 ? 200 : cu0_half_sweeps);
    g_cap_jacobi.store(jacobi_sweeps == 0 ? 60 : jacobi_sweeps);
  });
}

int peps_wait_selftest(int budget_us, void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(budget_us >= 1 && budget_us <= 1000000, "budget_us must be in [1, 1e6]");
    require_device();
    Call c(cuda_stream);
    wait_unset_flag(c.cx, (long long)budget_us * 1000);
    c.finish();
  });
}


int peps_bond_update(const peps_lattice* lat, const peps_opts* opts, const double* gate, const int* bonds,
                     int nbonds, int als_iters, void* A_out, double* cost, void* cuda_stream) {
  return bond_update_call(lat, opts, -1, gate, bonds, nbonds, als_iters, A_out, cost, cuda_stream);
}

int peps_bond_update_cluster(const peps_lattice* lat, const peps_opts* opts, int delta, const double* gate,
                             const int* bonds, int nbonds, int als_iters, void* A_out, double* cost,
                             void* cuda_stream) {
  if (delta < 0) return peps_set_error(PEPS_EINVAL, "delta must be >= 0");
  return bond_update_call(lat, opts, delta, gate, bonds, nbonds, als_iters, A_out, cost, cuda_stream);
}

int peps_boundary_fidelity(const peps_lattice* lat, const peps_opts* opts, int delta, int chi_ref,
                           double* one_minus_f, void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(one_minus_f != nullptr, "NULL argument");
    PEPS_REQUIRE(delta >= 1, "delta must be >= 1");
    PEPS_REQUIRE(chi_ref >= 1 && chi_ref <= 4096, "chi_ref must be in [1, 4096]");
    require_device();
    check_lattice(lat);
    const Opts o = check_opts(opts, false);
    PEPS_REQUIRE(lat->Lx >= 2, "the left-most column's environment needs Lx >= 2");
    Call c(cuda_stream);
    Arena keep(c.st);
    Oriented ori;
    build_orientations(c.cx, lat, keep, ori);
    const OLat& o3 = ori.o[3];   // right-left sweep: rows are the columns from the right
    const int L = o3.Ly, W = o3.Lx, D = lat->D;
    double* ln = c.ws.dalloc(2);
    fill(c.cx, ln, 2, 0.0);
    Opts oref = o;
    oref.chi = chi_ref;
    Mps ref, rho;
    {
      Engine e(c.cx, oref, lat->d, D, W);
      ref = e.sweep(o3, 3, L - 1, TP(ln), keep).back();
    }
    if (delta >= L - 1) {
      Engine e(c.cx, o, lat->d, D, W);
      rho = e.sweep(o3, 3, L - 1, TP(ln + 1), keep).back();
    } else {
      double* sig[4];
      cu0_all_sides(c.cx, lat, ori, keep, sig);
      const int r0 = L - 1 - delta;
      OLat part;
      part.Ly = delta + 1;
      part.Lx = W;
      part.d = o3.d;
      part.sites.assign(o3.sites.begin() + size_t(r0) * W, o3.sites.end());
      for (int x = 0; x < W; ++x)
        part.top.push_back(Mat{TP(sig[3] + ((long long)r0 * W + x) * D * D), o3.at(r0, x).du});
      part.bottom = o3.bottom;
      part.left.assign(o3.left.begin() + r0, o3.left.end());
      part.right.assign(o3.right.begin() + r0, o3.right.end());
      Engine e(c.cx, o, lat->d, D, W);
      rho = e.sweep(part, 3, delta, TP(ln + 1), keep).back();
    }
    double* ov = c.ws.dalloc(6);
    mps_ln_overlap(c.cx, ref, rho, ov);
    mps_ln_overlap(c.cx, ref, ref, ov + 2);
    mps_ln_overlap(c.cx, rho, rho, ov + 4);
    double h[6];
    PEPS_CUDA(cudaMemcpyAsync(h, ov, sizeof(h), cudaMemcpyDeviceToHost, c.st));
    c.finish();
    PEPS_REQUIRE(h[3] > 0 && h[5] > 0, "zero boundary (degenerate state)");
    *one_minus_f = 1.0 - std::exp(h[0] - 0.5 * (h[2] + h[4]));
  });
}

static int count_of(const EnvData& e, int kind) {
  if (kind == PEPS_SITE) return e.Ly * e.Lx;
  if (kind == PEPS_HBOND) return e.Ly * (e.Lx - 1);
  if (kind == PEPS_VBOND) return (e.Ly - 1) * e.Lx;
  return -1;
}

int peps_expect_local(const peps_env* env, const peps_lattice* lat, int kind, const double* op, double* out,
                      void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(env != nullptr && op != nullptr && out != nullptr, "NULL argument");
    const EnvData& e = env->data;
    const int count = count_of(e, kind);
    PEPS_REQUIRE(count >= 0, "kind must be PEPS_SITE, PEPS_HBOND or PEPS_VBOND");
    if (lat) PEPS_REQUIRE(lat->Ly == e.Ly && lat->Lx == e.Lx && lat->d == e.d, "lattice does not match env");
    if (count == 0) return;
    Call c(cuda_stream);
    const int k = kind == PEPS_SITE ? e.d : e.d * e.d;
    double* dop = c.ws.dalloc(size_t(k) * k);
    double* dout = c.ws.dalloc(count);
    PEPS_CUDA(cudaMemcpyAsync(dop, op, sizeof(double) * k * k, cudaMemcpyHostToDevice, c.st));
    const double* rho = kind == PEPS_SITE ? e.rho_site : (kind == PEPS_HBOND ? e.rho_h : e.rho_v);
    expect_batch(c.cx, rho, count, k, dop, dout);
    PEPS_CUDA(cudaMemcpyAsync(out, dout, sizeof(double) * count, cudaMemcpyDeviceToHost, c.st));
    c.finish();
  });
}

int peps_env_rho(const peps_env* env, int kind, double* out, void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(env != nullptr && out != nullptr, "NULL argument");
    const EnvData& e = env->data;
    const int count = count_of(e, kind);
    PEPS_REQUIRE(count >= 0, "kind must be PEPS_SITE, PEPS_HBOND or PEPS_VBOND");
    const int k = kind == PEPS_SITE ? e.d : e.d * e.d;
    const double* rho = kind == PEPS_SITE ? e.rho_site : (kind == PEPS_HBOND ? e.rho_h : e.rho_v);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (count > 0)
      PEPS_CUDA(cudaMemcpyAsync(out, rho, sizeof(double) * size_t(count) * k * k, cudaMemcpyDeviceToHost, st));
    PEPS_CUDA(cudaStreamSynchronize(st));
  });
}

int peps_norm(const peps_lattice* lat, const peps_opts* opts, double* ln_norm, int* sign, void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(ln_norm != nullptr && sign != nullptr, "NULL argument");
    require_device();
    check_lattice(lat);
    const Opts o = check_opts(opts, false);
    Call c(cuda_stream);
    Arena keep(c.st);
    Oriented ori;
    build_orientations(c.cx, lat, keep, ori);
    Engine eng(c.cx, o, lat->d, lat->D, std::max(lat->Ly, lat->Lx));
    double* acc = c.ws.dalloc(4);
    fill(c.cx, acc, 1, 0.0);
    auto bt = eng.sweep(ori.o[0], 0, lat->Ly - 1, acc, keep);
    eng.norm_from_top(ori.o[0], bt[lat->Ly - 1], acc, acc + 2);
    double h[2];
    PEPS_CUDA(cudaMemcpyAsync(h, acc + 2, sizeof(h), cudaMemcpyDeviceToHost, c.st));
    c.finish();
    *ln_norm = h[0];
    *sign = int(h[1]);
  });
}

int peps_env_ln_norm(const peps_env* env, double* ln_norm, int* sign, void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(env != nullptr && ln_norm != nullptr && sign != nullptr, "NULL argument");
    PEPS_REQUIRE(env->data.has_norm, "this env holds no norm (cluster envs do not)");
    double h[2];
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    PEPS_CUDA(cudaMemcpyAsync(h, env->data.lnnorm, sizeof(h), cudaMemcpyDeviceToHost, st));
    PEPS_CUDA(cudaStreamSynchronize(st));
    *ln_norm = h[0];
    *sign = int(h[1]);
  });
}

int peps_closure_data(const peps_lattice* lat, const peps_opts* opts, float* X, float* Y, long long capacity,
                      long long* count, void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(count != nullptr, "count is NULL");
    require_device();
    check_lattice(lat);
    const Opts o = check_opts(opts, false);
    PEPS_REQUIRE(lat->D <= 8, "learned closure supports D <= 8");
    long long ne = 0;
    ne += (long long)(lat->Ly - 1) * lat->Lx * 2 + (long long)(lat->Lx - 1) * lat->Ly * 2;
    *count = ne;
    if (X == nullptr && Y == nullptr) return;
    PEPS_REQUIRE(X != nullptr && Y != nullptr && capacity >= ne, "X, Y must hold count examples");
    Call c(cuda_stream);
    Arena keep(c.st, size_t(64) << 20, false);
    Oriented ori;
    build_orientations(c.cx, lat, keep, ori);
    // full boundaries at bond chi from all four sides
    Lanes lanes(c, o, lat->d, lat->D, std::max(lat->Ly, lat->Lx));
    double* lnacc = c.ws.dalloc(4);
    fill(c.cx, lnacc, 4, 0.0);
    std::vector<Mps> b[4];
    lanes.join();
    lanes.fork();
    run_lanes(lanes, 4, [&](Lane& L, int oi) {
      b[oi] = L.eng->sweep(ori.o[oi], oi, ori.o[oi].Ly - 1, lnacc + oi, keep);
    });
    lanes.join();
    double* sig[4];
    cu0_all_sides(c.cx, lat, ori, keep, sig);
    MlpDims m;
    m.d = lat->d;
    m.D = lat->D;
    const std::vector<RimSite> rs = rim_sites(ori, sig, lat->D);
    closure_features(c.cx, m, rs.data(), ne, X);
    // labels: best product approximation of each full boundary (one job per cut)
    std::vector<Rank1Job> jobs;
    std::vector<std::vector<const double*>> ptrs;
    std::vector<std::vector<int>> bonds;
    long long e0 = 0;
    int maxchi = 1, maxL = 1;
    for (int oi = 0; oi < 4; ++oi) {
      const OLat& L = ori.o[oi];
      for (int r = 1; r < L.Ly; ++r) {
        const Mps& T = b[oi][r];
        std::vector<const double*> pp;
        for (const TP& t : T.p) pp.push_back(t.d(0));
        std::vector<int> bd;
        for (int x = 0; x < L.Lx; ++x) bd.push_back(T.dims[x][0]);
        bd.push_back(T.dims[L.Lx - 1][3]);
        for (int v : bd) maxchi = std::max(maxchi, v);
        maxL = std::max(maxL, L.Lx);
        auto* dp = static_cast<const double* const*>(stage(c.cx, pp.data(), sizeof(double*) * pp.size()));
        auto* db = static_cast<const int*>(stage(c.cx, bd.data(), sizeof(int) * bd.size()));
        jobs.push_back(Rank1Job{dp, db, L.Lx, Y + e0 * m.out()});
        e0 += L.Lx;
      }
    }
    rank1_labels(c.cx, lat->D, maxchi, maxL, jobs.data(), int(jobs.size()));
    c.finish();
  });
}

long long peps_mlp_param_count(int d, int D, int width) {
  MlpDims m;
  m.d = d;
  m.D = D;
  m.W = width;
  return m.params();
}

static MlpDims mlp_dims(int d, int D, int width) {
  PEPS_REQUIRE(d >= 1 && d <= 4 && D >= 1 && D <= 8 && width >= 16 && width <= 4096, "bad MLP dims");
  MlpDims m;
  m.d = d;
  m.D = D;
  m.W = width;
  return m;
}

int peps_mlp_init(float* w, int d, int D, int width, unsigned long long seed, void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(w != nullptr, "w is NULL");
    require_device();
    const MlpDims m = mlp_dims(d, D, width);
    Call c(cuda_stream);
    mlp_init(c.cx, m, w, seed);
    c.finish();
  });
}

int peps_mlp_loss_grad(const float* w, const float* X, const float* Y, long long n, int d, int D, int width,
                       double* loss, float* grad, void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(w && X && Y && loss && grad && n > 0, "NULL argument or empty batch");
    require_device();
    PEPS_REQUIRE(tc_available(), "the learned closure runs on sm_103 tensor cores");
    const MlpDims m = mlp_dims(d, D, width);
    Call c(cuda_stream);
    double* dl = c.ws.dalloc(1);
    mlp_loss_grad(c.cx, m, w, X, Y, n, dl, grad);
    PEPS_CUDA(cudaMemcpyAsync(loss, dl, sizeof(double), cudaMemcpyDeviceToHost, c.st));
    c.finish();
  });
}

int peps_mlp_train(float* w, const float* X, const float* Y, long long n, int d, int D, int width, int steps,
                   int batch, float lr, float weight_decay, unsigned long long seed, double* final_loss,
                   void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(w && X && Y && n > 0, "NULL argument or empty training set");
    require_device();
    PEPS_REQUIRE(tc_available(), "the learned closure runs on sm_103 tensor cores");
    const MlpDims m = mlp_dims(d, D, width);
    Call c(cuda_stream);
    mlp_train(c.cx, m, w, X, Y, n, steps, batch, lr, weight_decay, seed, final_loss);
    c.finish();
  });
}

int peps_mlp_train_state(float* w, float* adam_m, float* adam_v, long long* step, const float* X, const float* Y,
                         long long n, int d, int D, int width, int steps, int batch, float lr, float weight_decay,
                         unsigned long long seed, double* final_loss, void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(w && adam_m && adam_v && step && X && Y && n > 0, "NULL argument or empty training set");
    PEPS_REQUIRE(*step >= 0, "step must be >= 0");
    require_device();
    PEPS_REQUIRE(tc_available(), "the learned closure runs on sm_103 tensor cores");
    const MlpDims m = mlp_dims(d, D, width);
    Call c(cuda_stream);
    mlp_train(c.cx, m, w, X, Y, n, steps, batch, lr, weight_decay, seed, final_loss, adam_m, adam_v, *step);
    c.finish();
    *step += steps;
  });
}

int peps_mlp_save(const char* path, const float* w, const float* adam_m, const float* adam_v, long long step, int d,
                  int D, int width, void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(w != nullptr, "w is NULL");
    PEPS_REQUIRE((adam_m == nullptr) == (adam_v == nullptr), "pass both AdamW moments or neither");
    require_device();
    const MlpDims m = mlp_dims(d, D, width);
    const size_t P = size_t(m.params());
    const bool state = adam_m != nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<float> hw(P), hm(state ? P : 0), hv(state ? P : 0);
    PEPS_CUDA(cudaMemcpyAsync(hw.data(), w, P * sizeof(float), cudaMemcpyDeviceToHost, st));
    if (state) {
      PEPS_CUDA(cudaMemcpyAsync(hm.data(), adam_m, P * sizeof(float), cudaMemcpyDeviceToHost, st));
      PEPS_CUDA(cudaMemcpyAsync(hv.data(), adam_v, P * sizeof(float), cudaMemcpyDeviceToHost, st));
    }
    PEPS_CUDA(cudaStreamSynchronize(st));
    const std::string json = "{\"format\":\"peps-mlp\",\"version\":1,\"d\":" + std::to_string(d) +
                             ",\"D\":" + std::to_string(D) + ",\"width\":" + std::to_string(width) +
                             ",\"params\":" + std::to_string(P) + ",\"state\":" + std::to_string(state ? 1 : 0) +
                             ",\"step\":" + std::to_string(step) + ",\"dtype\":\"f32\"}";
    ckpt_write(path, json, {{hw.data(), P * sizeof(float)}, {hm.data(), hm.size() * sizeof(float)},
                            {hv.data(), hv.size() * sizeof(float)}});
  });
}

int peps_mlp_load(const char* path, float* w, float* adam_m, float* adam_v, long long* step, int d, int D, int width,
                  void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(w != nullptr, "w is NULL");
    PEPS_REQUIRE((adam_m == nullptr) == (adam_v == nullptr), "pass both AdamW moments or neither");
    require_device();
    const MlpDims m = mlp_dims(d, D, width);
    const size_t P = size_t(m.params());
    const CkptIn c = ckpt_read(path, "peps-mlp");
    PEPS_REQUIRE(ckpt_int(c.hdr, "d") == d && ckpt_int(c.hdr, "D") == D && ckpt_int(c.hdr, "width") == width &&
                     ckpt_int(c.hdr, "params") == (long long)P,
                 "the checkpoint holds a network of another shape");
    const bool state = ckpt_int(c.hdr, "state") != 0;
    PEPS_REQUIRE(c.body.size() == (state ? 3 : 1) * P * sizeof(float), "checkpoint body has the wrong size");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    PEPS_CUDA(cudaMemcpyAsync(w, c.body.data(), P * sizeof(float), cudaMemcpyHostToDevice, st));
    if (adam_m) {
      if (state) {
        PEPS_CUDA(cudaMemcpyAsync(adam_m, c.body.data() + P * sizeof(float), P * sizeof(float),
                                  cudaMemcpyHostToDevice, st));
        PEPS_CUDA(cudaMemcpyAsync(adam_v, c.body.data() + 2 * P * sizeof(float), P * sizeof(float),
                                  cudaMemcpyHostToDevice, st));
      } else {
        PEPS_CUDA(cudaMemsetAsync(adam_m, 0, P * sizeof(float), st));
        PEPS_CUDA(cudaMemsetAsync(adam_v, 0, P * sizeof(float), st));
      }
    }
    if (step) *step = state ? ckpt_int(c.hdr, "step") : 0;
    PEPS_CUDA(cudaStreamSynchronize(st));
  });
}

int peps_env_save(const peps_env* env, const char* path, void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(env != nullptr, "env is NULL");
    require_device();
    const EnvData& e = env->data;
    const size_t d2 = size_t(e.d) * e.d, d4 = d2 * d2;
    const size_t ns = size_t(e.Ly) * e.Lx * d2, nh = std::max<size_t>(1, size_t(e.Ly) * (e.Lx - 1) * d4),
                 nv = std::max<size_t>(1, size_t(e.Ly - 1) * e.Lx * d4);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<double> hs(ns), hh(nh), hv(nv), hl(2);
    PEPS_CUDA(cudaMemcpyAsync(hs.data(), e.rho_site, ns * sizeof(double), cudaMemcpyDeviceToHost, st));
    PEPS_CUDA(cudaMemcpyAsync(hh.data(), e.rho_h, nh * sizeof(double), cudaMemcpyDeviceToHost, st));
    PEPS_CUDA(cudaMemcpyAsync(hv.data(), e.rho_v, nv * sizeof(double), cudaMemcpyDeviceToHost, st));
    PEPS_CUDA(cudaMemcpyAsync(hl.data(), e.lnnorm, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    PEPS_CUDA(cudaStreamSynchronize(st));
    const std::string json = "{\"format\":\"peps-env\",\"version\":1,\"kind\":" + std::to_string(env->kind) +
                             ",\"Ly\":" + std::to_string(e.Ly) + ",\"Lx\":" + std::to_string(e.Lx) +
                             ",\"d\":" + std::to_string(e.d) + ",\"D\":" + std::to_string(e.D) +
                             ",\"has_norm\":" + std::to_string(e.has_norm ? 1 : 0) + ",\"n_site\":" +
                             std::to_string(ns) + ",\"n_h\":" + std::to_string(nh) + ",\"n_v\":" +
                             std::to_string(nv) + ",\"dtype\":\"f64\"}";
    ckpt_write(path, json, {{hs.data(), ns * sizeof(double)}, {hh.data(), nh * sizeof(double)},
                            {hv.data(), nv * sizeof(double)}, {hl.data(), 2 * sizeof(double)}});
  });
}

int peps_env_load(const char* path, peps_env** out, void* cuda_stream) {
  if (out) *out = nullptr;
  return guard([&] {
    PEPS_REQUIRE(out != nullptr, "out is NULL");
    require_device();
    const CkptIn c = ckpt_read(path, "peps-env");
    peps_lattice shape{};
    shape.Ly = int(ckpt_int(c.hdr, "Ly"));
    shape.Lx = int(ckpt_int(c.hdr, "Lx"));
    shape.d = int(ckpt_int(c.hdr, "d"));
    shape.D = int(ckpt_int(c.hdr, "D"));
    PEPS_REQUIRE(shape.Ly >= 1 && shape.Lx >= 1 && shape.Ly <= 4096 && shape.Lx <= 4096 && shape.d >= 1 &&
                     shape.d <= 4 && shape.D >= 1 && shape.D <= 16,
                 "checkpoint header: lattice shape out of range");
    const int kind = int(ckpt_int(c.hdr, "kind"));
    const size_t d2 = size_t(shape.d) * shape.d, d4 = d2 * d2;
    const size_t ns = size_t(shape.Ly) * shape.Lx * d2, nh = std::max<size_t>(1, size_t(shape.Ly) * (shape.Lx - 1) * d4),
                 nv = std::max<size_t>(1, size_t(shape.Ly - 1) * shape.Lx * d4);
    PEPS_REQUIRE(ckpt_int(c.hdr, "n_site") == (long long)ns && ckpt_int(c.hdr, "n_h") == (long long)nh &&
                     ckpt_int(c.hdr, "n_v") == (long long)nv,
                 "checkpoint header: array sizes do not match the lattice shape");
    PEPS_REQUIRE(c.body.size() == (ns + nh + nv + 2) * sizeof(double), "checkpoint body has the wrong size");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    auto env = new_env(&shape, kind, st);
    EnvData& e = env->data;
    e.has_norm = ckpt_int(c.hdr, "has_norm") != 0;
    const char* b = c.body.data();
    PEPS_CUDA(cudaMemcpyAsync(e.rho_site, b, ns * sizeof(double), cudaMemcpyHostToDevice, st));
    PEPS_CUDA(cudaMemcpyAsync(e.rho_h, b + ns * sizeof(double), nh * sizeof(double), cudaMemcpyHostToDevice, st));
    PEPS_CUDA(cudaMemcpyAsync(e.rho_v, b + (ns + nh) * sizeof(double), nv * sizeof(double), cudaMemcpyHostToDevice,
                              st));
    PEPS_CUDA(cudaMemcpyAsync(e.lnnorm, b + (ns + nh + nv) * sizeof(double), 2 * sizeof(double),
                              cudaMemcpyHostToDevice, st));
    PEPS_CUDA(cudaStreamSynchronize(st));
    *out = env.release();
  });
}

int peps_mlp_predict(const float* w, const float* X, long long n, int d, int D, int width, float* sigma,
                     void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(w && X && sigma, "NULL argument");
    require_device();
    PEPS_REQUIRE(tc_available(), "the learned closure runs on sm_103 tensor cores");
    const MlpDims m = mlp_dims(d, D, width);
    Call c(cuda_stream);
    mlp_predict(c.cx, m, w, X, n, sigma);
    c.finish();
  });
}

void peps_env_free(peps_env* env) {
  if (!env) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(env->device);
  cudaDeviceSynchronize();
  env->arena.reset();
  cudaDeviceSynchronize();
  cudaSetDevice(cur);
  delete env;
}

const char* peps_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------
// Recorded plans (CUDA graphs)
// ---------------------------------------------------------------------------
int peps_plan_create(const peps_lattice* lat, const peps_opts* opts, int cluster, peps_plan** out,
                     void* cuda_stream) {
  if (out) *out = nullptr;
  return guard([&] {
    PEPS_REQUIRE(out != nullptr, "out is NULL");
    const Opts o = plan_checks(lat, opts, cluster != 0);
    validate_by_running(lat, opts, cluster != 0, cuda_stream);
    *out = record_plan(lat, opts, o, cluster != 0, Tune()).release();
  });
}

int peps_plan_tune(const peps_lattice* lat, const peps_opts* opts, int cluster, peps_plan** out, int* lanes,
                   int* qr_cluster, void* cuda_stream) {
  if (out) *out = nullptr;
  return guard([&] {
    PEPS_REQUIRE(out != nullptr, "out is NULL");
    const bool cl = cluster != 0;
    const Opts o = plan_checks(lat, opts, cl);
    validate_by_running(lat, opts, cl, cuda_stream);
    const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    PlanPtr best;
    double tbest = 1e300;
    Tune tb;
    auto consider = [&](const Tune& t) {
      PlanPtr p(record_plan(lat, opts, o, cl, t).release());
      const double ms = time_plan(p.get(), st, 2);
      if (std::getenv("PEPS_VERBOSE"))
        std::fprintf(stderr, "[peps] tune: lanes %d, qr cluster <= %d, chunk %d: %.3f ms\n", lanes_of(t),
                     t.qr_cmax > 0 ? t.qr_cmax : 16, t.chunk > 0 ? t.chunk : 16, ms);
      if (ms < tbest) {
        tbest = ms;
        tb = t;
        best.swap(p);
      }
    };
    // Coordinate search: lanes first (QR clusters by the model), then (cluster
    // scheme) the windows per batched chunk, then the QR cluster cap.
    for (int nl : {2, 4, 8}) consider(Tune{nl, 0, 0});
    if (cl)
      for (int ch : {8, 32}) consider(Tune{tb.lanes, 0, ch});
    const Tune base = tb;
    for (int qc : {8, 4}) consider(Tune{base.lanes, qc, base.chunk});
    if (lanes) *lanes = lanes_of(tb);
    if (qr_cluster) *qr_cluster = tb.qr_cmax > 0 ? tb.qr_cmax : 16;
    *out = best.release();
  });
}

int peps_plan_run(peps_plan* plan, void* cuda_stream) {
  return guard([&] {
    PEPS_REQUIRE(plan != nullptr && plan->exec != nullptr, "plan is NULL");
    int cur = 0;
    PEPS_CUDA(cudaGetDevice(&cur));
    PEPS_REQUIRE(cur == plan->device, "the plan was recorded on another device");
    const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    PEPS_CUDA(cudaGraphLaunch(plan->exec, st));
    Call::read_status(plan->flag, st);
    Prof& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    for (int i = 0; i < K_NCLASS; ++i) {
      p.launches[i] += plan->counts.launches[i];
      p.flops[i] += plan->counts.flops[i];
      p.bytes[i] += plan->counts.bytes[i];
    }
    for (auto& t : plan->counts.events) {   // classes timed when the plan was recorded
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, std::get<1>(t), std::get<2>(t)) == cudaSuccess) p.ms[std::get<0>(t)] += ms;
    }
    cudaGetLastError();
  });
}

const peps_env* peps_plan_env(const peps_plan* plan) { return plan ? plan->env.get() : nullptr; }

long long peps_plan_launches(const peps_plan* plan) { return plan ? plan->kernels : 0; }

void peps_plan_free(peps_plan* plan) {
  if (!plan) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(plan->device);
  cudaDeviceSynchronize();
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  for (auto& t : plan->counts.events) {
    cudaEventDestroy(std::get<1>(t));
    cudaEventDestroy(std::get<2>(t));
  }
  plan->exec = nullptr;
  plan->graph = nullptr;
  plan->env.reset();
  plan->persist.reset();
  cudaDeviceSynchronize();
  cudaSetDevice(cur);
  delete plan;
}

void peps_profile_enable(int mask) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.mask = unsigned(mask);
}

void peps_profile_reset(void) {
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.drain();
  for (int i = 0; i < K_NCLASS; ++i) {
    p.launches[i] = 0;
    p.flops[i] = p.bytes[i] = p.ms[i] = 0.0;
  }
}

int peps_profile_count(void) { return K_NCLASS; }

const char* peps_profile_name(int cls) { return (cls >= 0 && cls < K_NCLASS) ? kClassNames[cls] : ""; }

int peps_profile_read(int cls, long long* launches, double* ms, double* flops, double* bytes) {
  if (cls < 0 || cls >= K_NCLASS) return fail(PEPS_EINVAL, "bad kernel class");
  Prof& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.drain();
  if (launches) *launches = p.launches[cls];
  if (ms) *ms = p.ms[cls];
  if (flops) *flops = p.flops[cls];
  if (bytes) *bytes = p.bytes[cls];
  return PEPS_OK;
}

}  // extern "C"
