// Boundary-MPS sweeps, one-site ALS compression, row environments and local
// density matrices (Sections 2, 5.1-5.3), orchestrated on the host, executed
// on the device.  No host synchronisation happens inside a sweep: bond
// dimensions depend on shapes only, and every data-dependent quantity (norms,
// log-scales, convergence) stays on the device.
#include <algorithm>
#include <cmath>
#include <map>
#include <set>

#include "aux.cuh"
#include "engine.cuh"
#include "linalg.cuh"
#include "update.cuh"

namespace peps {

std::vector<int> bond_caps(const std::vector<int>& phys, const std::vector<long long>& prod, int chi) {
  const int Lx = int(phys.size());
  std::vector<int> caps(std::max(0, Lx - 1));
  const long long big = 1LL << 40;
  for (int k = 0; k + 1 < Lx; ++k) {
    long long lp = 1, rp = 1;
    for (int x = 0; x <= k; ++x) lp = std::min(lp * phys[x], big);
    for (int x = k + 1; x < Lx; ++x) rp = std::min(rp * phys[x], big);
    caps[k] = int(std::min<long long>({(long long)chi, lp, rp, prod[k]}));
  }
  for (int k = 1; k + 1 < Lx; ++k) caps[k] = std::min<long long>(caps[k], (long long)caps[k - 1] * phys[k]);
  for (int k = Lx - 3; k >= 0; --k) caps[k] = std::min<long long>(caps[k], (long long)caps[k + 1] * phys[k + 1]);
  return caps;
}

Engine::Engine(Ctx& c, const Opts& o, int d, int Dmax, int Lmax, int nb)
    : cx(c), opt(o), d_(d), Dmax_(Dmax), Lmax_(Lmax), nb_(nb), cap_(nb) {
  PEPS_REQUIRE(nb >= 1 && nb <= MAXB, "internal: problems per engine");
  const size_t chi = size_t(o.chi), D2 = size_t(Dmax) * Dmax, dd = size_t(d) * d;
  bigN_ = chi * chi * D2 * D2;
  // X1: chain stage 1 (chi^2 D^4; room for a padded tensor-core operand);
  // X2: ket stage (d chi^2 D^4); X3: bra stage with the physical pair open
  // (d^2 chi^2 D^4).  The largest intermediates of an environment set.
  X1_ = alloc(*cx.ws, bigN_ * dd);
  X2_ = alloc(*cx.ws, bigN_ * dd * d);
  x1per_ = (bigN_ * dd + 31) / 32 * 32;
  x2per_ = (bigN_ * dd * d + 31) / 32 * 32;
  X3_ = alloc(*cx.ws, bigN_ * dd);
  envN_ = chi * D2 * chi * dd;
  bb_ = alloc(*cx.ws, envN_);
  vv_ = alloc(*cx.ws, envN_);
  Lmax = std::max(Lmax, 2);
  Lenv_.resize(Lmax);
  Renv_.resize(Lmax);
  for (int i = 0; i < Lmax; ++i) {
    Lenv_[i] = alloc(*cx.ws, envN_);
    Renv_[i] = alloc(*cx.ws, envN_);
  }
  one_ = TP(cx.ws->dalloc(1));
  fill(cx, one_, 1, 1.0);
  tmp0_ = alloc(*cx.ws, 1);
  tmp1_ = alloc(*cx.ws, 1);
  tc_ = o.precision != PEPS_PREC_FP64;
  x64_ = !tc_;
  site_packs_ = std::make_unique<PackCache>(cx.ws);
  main_ = Side{&cx, X1_, X2_, X3_, tmp0_, site_packs_.get(), x1per_ * nb_, x2per_ * nb_};
}

Engine::~Engine() {
  if (!dual_) return;
  aux_.cx = nullptr;
  cache2_.reset();
  cx2_.reset();
  ws2_.reset();   // frees on the second stream ...
  cudaEvent_t e;   // ... which the main stream then waits for (required while recording a graph)
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
    cudaEventRecord(e, ws2_stream_);
    cudaStreamWaitEvent(cx.st, e, 0);
    cudaEventDestroy(e);
  }
}

void Engine::enable_dual(cudaStream_t st2) {
  const size_t dd = size_t(d_) * d_;
  const size_t set = (bigN_ * dd + bigN_ * dd * d_ + bigN_ * dd) * 8;
  if (dual_ || nb_ != 1 || set > (size_t(512) << 20)) return;
  ws2_stream_ = st2;
  {
    cudaEvent_t e;   // the second stream starts after everything enqueued so far
    PEPS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    PEPS_CUDA(cudaEventRecord(e, cx.st));
    PEPS_CUDA(cudaStreamWaitEvent(st2, e, 0));
    PEPS_CUDA(cudaEventDestroy(e));
  }
  ws2_ = std::make_unique<Arena>(st2);
  cx2_ = std::make_unique<Ctx>(st2, ws2_.get());
  cx2_->flag = cx.flag;
  cx2_->persist = cx.persist;
  cx2_->qr_cmax = cx.qr_cmax;
  cx2_->svd_cap = cx.svd_cap;
  cx2_->cu0_cap = cx.cu0_cap;
  cx2_->tmp = ws2_->dalloc(8);
  cache2_ = std::make_unique<PackCache>(ws2_.get());
  const size_t x1 = bigN_ * dd;
  aux_ = Side{cx2_.get(), strided(ws2_->dalloc((x1 + 31) / 32 * 32), 1, x1),
              strided(ws2_->dalloc((bigN_ * dd * d_ + 31) / 32 * 32), 1, bigN_ * dd * d_),
              strided(ws2_->dalloc((bigN_ * dd + 31) / 32 * 32), 1, bigN_ * dd),
              strided(ws2_->dalloc(32), 1, 1), cache2_.get(), (x1 + 31) / 32 * 32,
              (bigN_ * dd * d_ + 31) / 32 * 32};
  dual_ = true;
}

size_t Engine::footprint(const Opts& o, int d, int Dmax, int Lmax) {
  const size_t chi = size_t(o.chi), D2 = size_t(Dmax) * Dmax, dd = size_t(d) * d;
  const size_t big = chi * chi * D2 * D2, env = chi * D2 * chi * dd;
  return big * dd + big * dd * d + big * dd + 2 * env + 2 * size_t(std::max(Lmax, 2)) * env + 7 * 32;
}

void Engine::use(int B) {
  PEPS_REQUIRE(B >= 1 && B <= cap_, "internal: more problems than the engine holds");
  nb_ = B;
  for (TP* t : {&X1_, &X2_, &X3_, &bb_, &vv_, &tmp0_, &tmp1_}) t->n = B;
  for (auto& t : Lenv_) t.n = B;
  for (auto& t : Renv_) t.n = B;
  main_ = Side{&cx, X1_, X2_, X3_, tmp0_, site_packs_.get(), x1per_ * B, x2per_ * B};   // the helpers' view
}

TP Engine::alloc(Arena& a, size_t per) const {
  const size_t stride = (per + 31) / 32 * 32;
  return strided(a.dalloc(stride * nb_), nb_, per);
}

void Engine::con(const char* spec, const TP& A, bool a64, const Dims& ad, const TP& B, bool b64,
                 const Dims& bd, const TP& C, bool c64, bool b_site) {
  Ctx& c = *side_->cx;
  if (!tc_) {
    ein(c, spec, A, ad, B, bd, C);
    return;
  }
  ein_tc(c, spec, A, a64 ? 1 : 0, ad, B, b64 ? 1 : 0, bd, C, c64 ? 1 : 0, opt.precision, 1.0, TP(),
         b_site ? side_->cache : nullptr);
}

Mps Engine::closure_mps(const std::vector<Mat>& mats, Arena&) {
  Mps T;
  for (const Mat& m : mats) {
    T.p.push_back(m.p);
    T.dims.push_back({1, m.n, m.n, 1});
  }
  return T;
}

// Tensor-core chains.  The three GEMMs of an absorb chain hand their results
// over in the next GEMM's operand layout (TcChain), so the intermediates are
// written once, already rounded and split, and never repacked.  The output
// letter orders of the first two contractions are chosen for that hand-over:
// the next contraction's K letters are contiguous in its operand, so the
// epilogue writes runs along them.  The first two contractions sum over the same
// letters as the plain form; the third one takes its K letters in the order
// (s, then the bra leg pair) so that the second GEMM's rows write contiguous
// runs, which changes only the FP32 summation order.  Falls back to the plain
// form where the chain buffers are too small for a padded operand (tiny bonds).
Dims Engine::chain_left_tc(const TP& L, const Dims& ld, const TP& M, const Dims& md, const SiteT& A,
                           const TP& X3, bool open) {
  static const char* s1 = "clma,auvb->clmbvu";
  static const char* s2 = "clmbvu,sulnr->cbsmvnr";
  // bra stage: s traced, or kept open next to the bra's t (a site's density matrix)
  const char* s3 = open ? "cbsmvnr,tvmoq->cbsnrtoq" : "cbsmvnr,svmoq->cbnroq";
  Ctx& c = *side_->cx;
  const Dims ad = A.dims();
  const Dims x1 = ein_dims(s1, ld, md), x2 = ein_dims(s2, x1, ad), x3 = ein_dims(s3, x2, ad);
  const int np = ::peps::problems({&L, &M, &A.p, &X3});
  if (tc_operand_words(s2, x1, ad, np, opt.precision) > side_->x1n ||
      tc_operand_words(s3, x2, ad, np, opt.precision) > side_->x2n)
    return Dims();
  TcOperand o1, o2;
  TcChain c1, c2, c3;
  c1.next = s2;
  c1.next_bd = ad;
  c1.next_mem = side_->X1.d(0);
  c1.next_cap = side_->x1n;
  c1.next_out = &o1;
  ein_tc(c, s1, L, 1, ld, M, 1, md, TP(), 0, opt.precision, 1.0, TP(), nullptr, &c1);
  c2.a_pre = &o1;
  c2.next = s3;
  c2.next_bd = ad;
  c2.next_mem = side_->X2.d(0);
  c2.next_cap = side_->x2n;
  c2.next_out = &o2;
  ein_tc(c, s2, TP(), 0, x1, A.p, 1, ad, TP(), 0, opt.precision, 1.0, TP(), side_->cache, &c2);
  c3.a_pre = &o2;
  ein_tc(c, s3, TP(), 0, x2, A.p, 1, ad, X3, 0, opt.precision, 1.0, TP(), side_->cache, &c3);
  return x3;
}

Dims Engine::chain_right_tc(const TP& R, const Dims& rd, const TP& M, const Dims& md, const SiteT& A,
                            const TP& Y3, bool open) {
  static const char* s1 = "auvb,brqc->auvcqr";
  static const char* s2 = "auvcqr,sulnr->acsvqln";
  const char* s3 = open ? "acsvqln,tvmoq->acslntmo" : "acsvqln,svmoq->aclnmo";
  Ctx& c = *side_->cx;
  const Dims ad = A.dims();
  const Dims y1 = ein_dims(s1, md, rd), y2 = ein_dims(s2, y1, ad), y3 = ein_dims(s3, y2, ad);
  const int np = ::peps::problems({&R, &M, &A.p, &Y3});
  if (tc_operand_words(s2, y1, ad, np, opt.precision) > side_->x1n ||
      tc_operand_words(s3, y2, ad, np, opt.precision) > side_->x2n)
    return Dims();
  TcOperand o1, o2;
  TcChain c1, c2, c3;
  c1.next = s2;
  c1.next_bd = ad;
  c1.next_mem = side_->X1.d(0);
  c1.next_cap = side_->x1n;
  c1.next_out = &o1;
  ein_tc(c, s1, M, 1, md, R, 1, rd, TP(), 0, opt.precision, 1.0, TP(), nullptr, &c1);
  c2.a_pre = &o1;
  c2.next = s3;
  c2.next_bd = ad;
  c2.next_mem = side_->X2.d(0);
  c2.next_cap = side_->x2n;
  c2.next_out = &o2;
  ein_tc(c, s2, TP(), 0, y1, A.p, 1, ad, TP(), 0, opt.precision, 1.0, TP(), side_->cache, &c2);
  c3.a_pre = &o2;
  ein_tc(c, s3, TP(), 0, y2, A.p, 1, ad, Y3, 0, opt.precision, 1.0, TP(), side_->cache, &c3);
  return y3;
}

Dims Engine::chain_left(const TP& L, const Dims& ld, const TP& M, const Dims& md, const SiteT& A,
                        const TP& X3) {
  if (tc_) {
    const Dims r = chain_left_tc(L, ld, M, md, A, X3, false);
    if (!r.empty()) return r;
  }
  const Dims ad = A.dims();
  const Dims x1 = ein_dims("clma,auvb->clmuvb", ld, md);
  con("clma,auvb->clmuvb", L, true, ld, M, true, md, side_->X1, x64_);
  const Dims x2 = ein_dims("clmuvb,sulnr->cmvbsnr", x1, ad);
  con("clmuvb,sulnr->cmvbsnr", side_->X1, x64_, x1, A.p, true, ad, side_->X2, x64_, true);
  const Dims x3 = ein_dims("cmvbsnr,svmoq->cbnroq", x2, ad);
  con("cmvbsnr,svmoq->cbnroq", side_->X2, x64_, x2, A.p, true, ad, X3, x64_, true);
  return x3;
}

Dims Engine::chain_right(const TP& R, const Dims& rd, const TP& M, const Dims& md, const SiteT& A,
                         const TP& Y3) {
  if (tc_) {
    const Dims r = chain_right_tc(R, rd, M, md, A, Y3, false);
    if (!r.empty()) return r;
  }
  const Dims ad = A.dims();
  const Dims y1 = ein_dims("auvb,brqc->auvrqc", md, rd);
  con("auvb,brqc->auvrqc", M, true, md, R, true, rd, side_->X1, x64_);
  const Dims y2 = ein_dims("auvrqc,sulnr->avqcsln", y1, ad);
  con("auvrqc,sulnr->avqcsln", side_->X1, x64_, y1, A.p, true, ad, side_->X2, x64_, true);
  const Dims y3 = ein_dims("avqcsln,svmoq->aclnmo", y2, ad);
  con("avqcsln,svmoq->aclnmo", side_->X2, x64_, y2, A.p, true, ad, Y3, x64_, true);
  return y3;
}

Mps Engine::product_mps(const Mps& T, const OLat& lat, int y, Arena& step) {
  const int Lx = lat.Lx;
  Mps P;
  for (int x = 0; x < Lx; ++x) {
    const SiteT& A = lat.at(y, x);
    const Dims ad = A.dims();
    const Dims t1 = ein_dims("auvb,sulnr->avbslnr", T.dims[x], ad);
    con("auvb,sulnr->avbslnr", T.p[x], true, T.dims[x], A.p, true, ad, X2_, x64_, true);
    const Dims t2 = ein_dims("avbslnr,svmoq->almnobrq", t1, ad);
    TP cur = alloc(step, numel(t2));
    con("avbslnr,svmoq->almnobrq", X2_, x64_, t1, A.p, true, ad, cur, true, true);
    Dims cd = t2;
    if (x == 0) {
      const Mat& c = lat.left[y];
      const Dims nd = ein_dims("lm,almnobrq->anobrq", {c.n, c.n}, cd);
      TP nx = alloc(step, numel(nd));
      ein(cx, "lm,almnobrq->anobrq", c.p, {c.n, c.n}, cur, cd, nx);
      cur = nx;
      cd = nd;
    }
    if (x == Lx - 1) {
      const Mat& c = lat.right[y];
      const char* spec = (x == 0) ? "anobrq,rq->anob" : "almnobrq,rq->almnob";
      const Dims nd = ein_dims(spec, cd, {c.n, c.n});
      TP nx = alloc(step, numel(nd));
      ein(cx, spec, cur, cd, c.p, {c.n, c.n}, nx);
      cur = nx;
      cd = nd;
    }
    Dims pd;
    if (x == 0) {
      pd = {cd[0], cd[1], cd[2], 1};
      for (size_t i = 3; i < cd.size(); ++i) pd[3] *= cd[i];
    } else {
      pd = {cd[0] * cd[1] * cd[2], cd[3], cd[4], 1};
      for (size_t i = 5; i < cd.size(); ++i) pd[3] *= cd[i];
    }
    P.p.push_back(cur);
    P.dims.push_back(pd);
  }
  return P;
}

void Engine::left_canonicalize(Mps& P, Arena& step) {
  const int Lx = int(P.p.size());
  for (int x = 0; x + 1 < Lx; ++x) {
    const Dims pd = P.dims[x];
    const int m = pd[0] * pd[1] * pd[2], n = pd[3], k = std::min(m, n);
    TP Q = alloc(step, size_t(m) * k);
    TP R = alloc(step, size_t(k) * n);
    qr_thin(cx, m, n, P.p[x], n, 1, Q, k, 1, R);
    P.p[x] = Q;
    P.dims[x] = {pd[0], pd[1], pd[2], k};
    const Dims nd = ein_dims("kb,bnoc->knoc", {k, n}, P.dims[x + 1]);
    TP nx = alloc(step, numel(nd));
    ein(cx, "kb,bnoc->knoc", R, {k, n}, P.p[x + 1], P.dims[x + 1], nx);
    P.p[x + 1] = nx;
    P.dims[x + 1] = nd;
  }
}

void Engine::svd_truncate(Mps& P, const std::vector<int>& caps, Arena& step) {
  const int Lx = int(P.p.size());
  for (int x = Lx - 1; x >= 1; --x) {
    const Dims pd = P.dims[x];
    const int m = pd[0], n = pd[1] * pd[2] * pd[3];
    const int kk = std::min(caps[x - 1], std::min(m, n));
    TP US = alloc(step, size_t(m) * kk);
    TP Vt = alloc(step, size_t(kk) * n);
    svd_trunc(cx, m, n, P.p[x], kk, US, Vt);
    P.p[x] = Vt;
    P.dims[x] = {kk, pd[1], pd[2], pd[3]};
    const Dims nd = ein_dims("anob,bk->anok", P.dims[x - 1], {m, kk});
    TP nx = alloc(step, numel(nd));
    ein(cx, "anob,bk->anok", P.p[x - 1], P.dims[x - 1], US, {m, kk}, nx);
    P.p[x - 1] = nx;
    P.dims[x - 1] = nd;
  }
}

Mps Engine::var_compress(const Mps& T, const OLat& lat, int y, const std::vector<int>& caps,
                         int tag, int& centre, Arena& step) {
  const int Lx = lat.Lx;
  Mps N;
  N.p.resize(Lx);
  N.dims.resize(Lx);
  for (int x = 0; x < Lx; ++x) {
    const int c = x == 0 ? 1 : caps[x - 1];
    const int e = x == Lx - 1 ? 1 : caps[x];
    const int D = lat.at(y, x).dn;
    N.dims[x] = {c, D, D, e};
    N.p[x] = alloc(step, numel(N.dims[x]));
    var_init(cx, T.p[x], T.dims[x].data(), N.p[x], N.dims[x].data(), opt.seed, tag, y, x, tmp1_);
  }
  // Right-canonicalise the start: N[x] = R^T Q^T (QR of N[x]^T), R^T moves left.
  // A start that is a plain copy of a right-canonical boundary (the previous
  // fit ended on a right-to-left half-sweep and no bond grew) is already in
  // that form: there each QR would return N[x]^T up to column signs and
  // rounding, so the pass is skipped.  The skipped pass changes only the sign
  // gauge of the bonds, which no contracted quantity sees.
  bool copy_of_canonical = T.right_canonical;
  for (int x = 0; x < Lx; ++x) copy_of_canonical = copy_of_canonical && N.dims[x] == T.dims[x];
  for (int x = Lx - 1; x >= 1 && !copy_of_canonical; --x) {
    const Dims nd = N.dims[x];
    const int c = nd[0], noe = nd[1] * nd[2] * nd[3];
    PEPS_REQUIRE(c <= noe, "internal: inconsistent bond caps");
    TP Rt = alloc(step, size_t(c) * c);
    qr_thin(cx, noe, c, N.p[x], 1, noe, N.p[x], 1, noe, Rt);
    const Dims pd = N.dims[x - 1];
    ein(cx, "anob,kb->anok", N.p[x - 1], pd, Rt, {c, c}, bb_);
    copy(cx, N.p[x - 1], bb_, (long long)numel(pd));
  }
  std::vector<Dims> ld(Lx), rd(Lx);
  {
    const Mat& r = lat.right[y];
    rd[Lx - 1] = {1, r.n, r.n, 1};
    copy(cx, Renv_[Lx - 1], r.p, (long long)r.n * r.n);
    const Mat& l = lat.left[y];
    ld[0] = {1, l.n, l.n, 1};
    copy(cx, Lenv_[0], l.p, (long long)l.n * l.n);
  }
  for (int x = Lx - 1; x >= 1; --x) {
    const Dims y3 = chain_right(Renv_[x], rd[x], T.p[x], T.dims[x], lat.at(y, x), X3_);
    rd[x - 1] = ein_dims("aelnmo,cnoe->almc", y3, N.dims[x]);
    con("aelnmo,cnoe->almc", X3_, x64_, y3, N.p[x], true, N.dims[x], Renv_[x - 1], true);
  }
  for (int h = 0; h < opt.sweeps; ++h) {
    if (h % 2 == 0) {
      for (int x = 0; x < Lx; ++x) {
        const Dims x3 = chain_left(Lenv_[x], ld[x], T.p[x], T.dims[x], lat.at(y, x), X3_);
        const Dims bd = ein_dims("cbnroq,brqe->cnoe", x3, rd[x]);
        con("cbnroq,brqe->cnoe", X3_, x64_, x3, Renv_[x], true, rd[x], bb_, true);
        PEPS_REQUIRE(bd == N.dims[x], "internal: local tensor shape");
        if (x < Lx - 1) {
          const int m = bd[0] * bd[1] * bd[2], n = bd[3];
          PEPS_REQUIRE(n <= m, "internal: inconsistent bond caps");
          qr_thin(cx, m, n, bb_, n, 1, N.p[x], n, 1, TP());
          ld[x + 1] = ein_dims("cbnroq,cnoe->erqb", x3, N.dims[x]);
          con("cbnroq,cnoe->erqb", X3_, x64_, x3, N.p[x], true, N.dims[x], Lenv_[x + 1], true);
        } else {
          copy(cx, N.p[x], bb_, (long long)numel(bd));
        }
      }
      centre = Lx - 1;
    } else {
      for (int x = Lx - 1; x >= 0; --x) {
        const Dims y3 = chain_right(Renv_[x], rd[x], T.p[x], T.dims[x], lat.at(y, x), X3_);
        const Dims bd = ein_dims("clma,aelnmo->cnoe", ld[x], y3);
        con("clma,aelnmo->cnoe", Lenv_[x], true, ld[x], X3_, x64_, y3, bb_, true);
        PEPS_REQUIRE(bd == N.dims[x], "internal: local tensor shape");
        if (x > 0) {
          const int c = bd[0], noe = bd[1] * bd[2] * bd[3];
          qr_thin(cx, noe, c, bb_, 1, noe, N.p[x], 1, noe, TP());
          rd[x - 1] = ein_dims("aelnmo,cnoe->almc", y3, N.dims[x]);
          con("aelnmo,cnoe->almc", X3_, x64_, y3, N.p[x], true, N.dims[x], Renv_[x - 1], true);
        } else {
          copy(cx, N.p[x], bb_, (long long)numel(bd));
        }
      }
      centre = 0;
    }
  }
  N.right_canonical = centre == 0;
  return N;
}

Mps Engine::absorb_compress(const Mps& T, const OLat& lat, int y, int tag, const TP& lnacc, Arena& keep) {
  const int Lx = lat.Lx;
  std::vector<int> phys(Lx);
  std::vector<long long> prod(std::max(0, Lx - 1));
  for (int x = 0; x < Lx; ++x) phys[x] = lat.at(y, x).dn * lat.at(y, x).dn;
  for (int k = 0; k + 1 < Lx; ++k) prod[k] = (long long)T.dims[k][3] * lat.at(y, k).dr * lat.at(y, k).dr;
  const std::vector<int> caps = bond_caps(phys, prod, opt.chi);
  Arena step(cx.st);
  Mps P;
  int centre = 0;
  bool exact = true;
  for (int k = 0; k + 1 < Lx; ++k) exact = exact && prod[k] <= caps[k];
  if (opt.mode == PEPS_SVD) {
    P = product_mps(T, lat, y, step);
    left_canonicalize(P, step);
    svd_truncate(P, caps, step);
    centre = 0;
  } else if (exact) {
    P = product_mps(T, lat, y, step);
    left_canonicalize(P, step);
    centre = Lx - 1;
  } else {
    P = var_compress(T, lat, y, caps, tag, centre, step);
  }
  normalize(cx, P.p[centre], (long long)numel(P.dims[centre]), lnacc, tmp0_);
  Mps out;
  out.right_canonical = P.right_canonical;
  for (int x = 0; x < Lx; ++x) {
    const size_t n = numel(P.dims[x]);
    TP q = alloc(keep, n);
    copy(cx, q, P.p[x], (long long)n);
    out.p.push_back(q);
    out.dims.push_back(P.dims[x]);
  }
  return out;
}

std::vector<Mps> Engine::sweep(const OLat& lat, int tag, int upto, const TP& lnacc, Arena& keep,
                               const std::function<void(int, const Mps&)>& on_boundary) {
  std::vector<Mps> out;
  out.push_back(closure_mps(lat.top, keep));
  if (on_boundary) on_boundary(0, out.back());
  for (int y = 0; y < upto; ++y) {
    out.push_back(absorb_compress(out.back(), lat, y, tag, lnacc, keep));
    if (on_boundary) on_boundary(y + 1, out.back());
  }
  return out;
}

void Engine::row_envs(const OLat& lat, const Mps& T, const Mps& B, int y, int xmin, int xmax,
                      std::vector<Dims>& ld, std::vector<Dims>& rd) {
  const int Lx = lat.Lx;
  ld.assign(Lx, Dims());
  rd.assign(Lx, Dims());
  const Mat& lc = lat.left[y];
  const Mat& rc = lat.right[y];
  ld[0] = {1, lc.n, lc.n, 1};
  copy(cx, Lenv_[0], lc.p, (long long)lc.n * lc.n);
  rd[Lx - 1] = {1, rc.n, rc.n, 1};
  for (int x = 0; x + 1 < Lx && x + 1 < xmax; ++x) {
    const Dims x3 = chain_left(Lenv_[x], ld[x], T.p[x], T.dims[x], lat.at(y, x), X3_);
    ld[x + 1] = ein_dims("cbnroq,cnoe->erqb", x3, B.dims[x]);
    con("cbnroq,cnoe->erqb", X3_, x64_, x3, B.p[x], true, B.dims[x], Lenv_[x + 1], true);
    normalize(cx, Lenv_[x + 1], (long long)numel(ld[x + 1]), TP(), tmp0_);
  }
  // Right environments: on the second stream when there is one (they depend
  // only on T, B and the row, like the left ones).
  if (dual_) {
    cudaEvent_t e;
    PEPS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    PEPS_CUDA(cudaEventRecord(e, cx.st));
    PEPS_CUDA(cudaStreamWaitEvent(aux_.cx->st, e, 0));
    PEPS_CUDA(cudaEventDestroy(e));
    side_ = &aux_;
  }
  copy(*side_->cx, Renv_[Lx - 1], rc.p, (long long)rc.n * rc.n);
  for (int x = Lx - 1; x >= 1 && x - 1 >= xmin; --x) {
    const Dims y3 = chain_right(Renv_[x], rd[x], T.p[x], T.dims[x], lat.at(y, x), side_->X3);
    rd[x - 1] = ein_dims("aelnmo,cnoe->almc", y3, B.dims[x]);
    con("aelnmo,cnoe->almc", side_->X3, x64_, y3, B.p[x], true, B.dims[x], Renv_[x - 1], true);
    normalize(*side_->cx, Renv_[x - 1], (long long)numel(rd[x - 1]), TP(), side_->tmp);
  }
  if (dual_) {
    side_ = &main_;
    cudaEvent_t e;
    PEPS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    PEPS_CUDA(cudaEventRecord(e, aux_.cx->st));
    PEPS_CUDA(cudaStreamWaitEvent(cx.st, e, 0));
    PEPS_CUDA(cudaEventDestroy(e));
  }
}

Dims Engine::open_left(const Mps& T, const Mps& B, int x, const SiteT& A, const Dims& ldx) {
  const Dims ad = A.dims();
  Dims x3 = tc_ ? chain_left_tc(Lenv_[x], ldx, T.p[x], T.dims[x], A, X3_, true) : Dims();
  if (x3.empty()) {
    const Dims x1 = ein_dims("clma,auvb->clmuvb", ldx, T.dims[x]);
    con("clma,auvb->clmuvb", Lenv_[x], true, ldx, T.p[x], true, T.dims[x], X1_, x64_);
    const Dims x2 = ein_dims("clmuvb,sulnr->cmvbsnr", x1, ad);
    con("clmuvb,sulnr->cmvbsnr", X1_, x64_, x1, A.p, true, ad, X2_, x64_, true);
    x3 = ein_dims("cmvbsnr,tvmoq->cbsnrtoq", x2, ad);
    con("cmvbsnr,tvmoq->cbsnrtoq", X2_, x64_, x2, A.p, true, ad, X3_, x64_, true);
  }
  const Dims w = ein_dims("cbsnrtoq,cnoe->erqbst", x3, B.dims[x]);
  con("cbsnrtoq,cnoe->erqbst", X3_, x64_, x3, B.p[x], true, B.dims[x], bb_, true);
  return w;
}

// V[a,l,m,k,s,t] = sum M R A(s) A(t) B over the bonds and legs right of the site.
Dims Engine::open_right(const Mps& T, const Mps& B, int x, const SiteT& A, const Dims& rdx) {
  const Dims ad = A.dims();
  Dims y3 = tc_ ? chain_right_tc(Renv_[x], rdx, T.p[x], T.dims[x], A, X3_, true) : Dims();
  if (y3.empty()) {
    const Dims y1 = ein_dims("auvb,brqc->auvrqc", T.dims[x], rdx);
    con("auvb,brqc->auvrqc", T.p[x], true, T.dims[x], Renv_[x], true, rdx, X1_, x64_);
    const Dims y2 = ein_dims("auvrqc,sulnr->avqcsln", y1, ad);
    con("auvrqc,sulnr->avqcsln", X1_, x64_, y1, A.p, true, ad, X2_, x64_, true);
    y3 = ein_dims("avqcsln,tvmoq->acslntmo", y2, ad);
    con("avqcsln,tvmoq->acslntmo", X2_, x64_, y2, A.p, true, ad, X3_, x64_, true);
  }
  const Dims v = ein_dims("acslntmo,knoc->almkst", y3, B.dims[x]);
  con("acslntmo,knoc->almkst", X3_, x64_, y3, B.p[x], true, B.dims[x], vv_, true);
  return v;
}

void Engine::row_rhos(const OLat& lat, const Mps& T, const Mps& B, int y, const Targets& sites,
                      const Targets& bonds) {
  const int Lx = lat.Lx;
  int xmax = 0, xmin = lat.Lx;
  for (const auto& t : sites) {
    xmax = std::max(xmax, t.first + 1);
    xmin = std::min(xmin, t.first);
  }
  for (const auto& t : bonds) {
    xmax = std::max(xmax, t.first + 2);
    xmin = std::min(xmin, t.first);
  }
  std::vector<Dims> ld, rd;
  row_envs(lat, T, B, y, xmin, xmax, ld, rd);
  // Every target column once, left to right: W(x) (open from the left) gives
  // rho_site(x) with the right environment; the bond (x, x+1) is W(x) joined
  // with V(x+1) (open from the right) over the bonds and legs between them --
  // the same network as pushing W(x) through site x+1 with both pairs open,
  // contracted in an order whose intermediates stay at d^2 chi^2 D^4.
  std::map<int, TP> site_dst, bond_dst;
  for (const auto& t : sites) site_dst[t.first] = t.second;
  for (const auto& t : bonds) {
    PEPS_REQUIRE(t.first + 1 < Lx, "internal: bond outside the row");
    bond_dst[t.first] = t.second;
  }
  std::set<int> cols;
  for (const auto& kv : site_dst) cols.insert(kv.first);
  for (const auto& kv : bond_dst) cols.insert(kv.first);
  for (const int x : cols) {
    const Dims w = open_left(T, B, x, lat.at(y, x), ld[x]);
    auto si = site_dst.find(x);
    if (si != site_dst.end()) ein(cx, "erqbst,brqe->st", bb_, w, Renv_[x], rd[x], si->second);
    auto bi = bond_dst.find(x);
    if (bi != bond_dst.end()) {
      const Dims v = open_right(T, B, x + 1, lat.at(y, x + 1), rd[x + 1]);
      ein(cx, "erqbij,brqest->isjt", bb_, w, vv_, v, bi->second);
    }
  }
}

void Engine::row_bond_norms(const OLat& lat, const Mps& T, const Mps& B, int y, const std::vector<BondNorm>& bonds) {
  PEPS_REQUIRE(nb_ == 1, "internal: bond norms are computed for one lattice");
  const int Lx = lat.Lx;
  int xmax = 0, xmin = Lx;
  for (const auto& b : bonds) {
    PEPS_REQUIRE(b.x >= 0 && b.x + 1 < Lx, "internal: bond outside the row");
    xmax = std::max(xmax, b.x + 2);
    xmin = std::min(xmin, b.x);
  }
  std::vector<Dims> ld, rd;
  row_envs(lat, T, B, y, xmin, xmax, ld, rd);
  for (const auto& b : bonds) {
    const SiteT& L = lat.at(y, b.x);
    const SiteT& R = lat.at(y, b.x + 1);
    const int d = L.d;
    // the two sites as matrices, then their thin QR (Householder, FP64)
    const int dl5[5] = {d, L.du, L.dl, L.dn, L.dr}, pl[5] = {1, 2, 3, 0, 4};
    const int dr5[5] = {d, R.du, R.dl, R.dn, R.dr}, pr[5] = {1, 3, 4, 0, 2};
    permute5(cx, L.p.d(0), dl5, pl, b.ml);
    permute5(cx, R.p.d(0), dr5, pr, b.mr);
    const int ml = L.du * L.dl * L.dn, nl = d * L.dr, mr = R.du * R.dn * R.dr, nr = d * R.dl;
    const int kl = std::min(ml, nl), kr = std::min(mr, nr);
    qr_thin(cx, ml, nl, TP(b.ml), nl, 1, TP(b.xl), 1, ml, TP(b.al));
    qr_thin(cx, mr, nr, TP(b.mr), nr, 1, TP(b.xr), 1, mr, TP(b.ar));
    SiteT XL, XR;
    XL.p = TP(b.xl);
    XL.d = kl;
    XL.du = L.du;
    XL.dl = L.dl;
    XL.dn = L.dn;
    XL.dr = 1;
    XR.p = TP(b.xr);
    XR.d = kr;
    XR.du = R.du;
    XR.dl = 1;
    XR.dn = R.dn;
    XR.dr = R.dr;
    const Dims w = open_left(T, B, b.x, XL, ld[b.x]);
    const Dims v = open_right(T, B, b.x + 1, XR, rd[b.x + 1]);
    ein(cx, "erqbij,brqest->isjt", bb_, w, vv_, v, TP(b.N));
  }
}

void Engine::norm_from_top(const OLat& lat, const Mps& T, const TP& lns_acc, const TP& out) {
  PEPS_REQUIRE(nb_ == 1, "internal: the norm is computed for one lattice");
  const int Lx = lat.Lx, y = lat.Ly - 1;
  double* extra = cx.ws->dalloc(1);
  double* s = cx.ws->dalloc(1);
  fill(cx, extra, 1, 0.0);
  const Mat& lc = lat.left[y];
  Dims ld = {1, lc.n, lc.n, 1};
  copy(cx, Lenv_[0], lc.p, (long long)lc.n * lc.n);
  int cur = 0;
  for (int x = 0; x < Lx; ++x) {
    const Dims x3 = chain_left(Lenv_[cur], ld, T.p[x], T.dims[x], lat.at(y, x), X3_);
    const Mat& bc = lat.bottom[x];
    const Dims bd = {1, bc.n, bc.n, 1};
    const Dims nd = ein_dims("cbnroq,cnoe->erqb", x3, bd);
    con("cbnroq,cnoe->erqb", X3_, x64_, x3, bc.p, true, bd, Lenv_[1 - cur], true);
    cur = 1 - cur;
    ld = nd;
    if (x + 1 < Lx) normalize(cx, Lenv_[cur], (long long)numel(ld), extra, tmp0_);
  }
  const Mat& rc = lat.right[y];
  ein(cx, "erqb,rq->", Lenv_[cur], ld, rc.p, {rc.n, rc.n}, s);
  finish_norm(cx, lns_acc.d(0), 1, extra, s, out.d(0), out.d(0) + 1);
}

}  // namespace peps
