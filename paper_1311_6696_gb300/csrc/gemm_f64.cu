// FP64 gather-GEMM: C[m,n] = alpha * sum_k A[m,k] B[k,n] + beta * C[m,n]
// where m, n, k (and a batch index) are each a group of tensor indices with
// arbitrary strides.  A pairwise tensor contraction therefore runs without
// any permutation copy: each CTA decomposes the row, column and k indices of
// its tile into element offsets once, keeps them in shared memory and
// gathers the operands through them.
//
// On GB300 the FP64 pipe issues about 2 DFMA per clock per SM (~1.2 TFLOP/s
// for the chip), so this kernel is bound by the FP64 ALU long before memory:
// a 64x64x16 tile step performs 65,536 DFMA against 2,048 loaded doubles.
// Grid = (tiles, split-K, batch x problems); split-K partials are reduced by
// a second kernel in a fixed order, so results are deterministic.  Independent
// problems of one shape (TP pointer sets) share a launch.
#include <algorithm>
#include <cstring>
#include <map>

#include "ein.cuh"

namespace peps {

namespace {

constexpr int MAXG = 8;
constexpr int BK = 16;

struct Grp {
  int n;
  int dim[MAXG];
  long long sa[MAXG], sb[MAXG], sc[MAXG];
};

struct GemmArgs {
  TP A, B, C;        // per problem
  int nprob;
  double* part;
  Grp gm, gn, gk, gb;
  long long M, N, K, NB;
  long long kchunk;
  int splitk;
  double alpha, beta;
};

__device__ __forceinline__ void decomp(const Grp& g, long long idx, long long& oa, long long& ob,
                                       long long& oc) {
  oa = ob = oc = 0;
  for (int i = g.n - 1; i >= 0; --i) {
    long long q = idx / g.dim[i];
    long long r = idx - q * g.dim[i];
    idx = q;
    oa += r * g.sa[i];
    ob += r * g.sb[i];
    oc += r * g.sc[i];
  }
}

template <int BM, int BN>
__global__ void __launch_bounds__(256) k_gemm_f64(const GemmArgs g) {
  constexpr int TX = BN / 4, TY = BM / 4;
  static_assert(TX * TY == 256, "256 threads, 4x4 outputs each");
  __shared__ double As[BK][BM];
  __shared__ double Bs[BK][BN];
  __shared__ long long oAm[BM], oCm[BM], oBn[BN], oCn[BN], oAk[BK], oBk[BK];
  __shared__ long long bA, bB, bC;

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const long long tiles_n = (g.N + BN - 1) / BN;
  const long long tm = (long long)blockIdx.x / tiles_n, tn = (long long)blockIdx.x % tiles_n;
  const long long m0 = tm * BM, n0 = tn * BN;
  const int split = blockIdx.y;
  const long long bz = blockIdx.z;              // problem * NB + batch index
  const long long bi = bz % g.NB;
  const int pb = int(bz / g.NB);
  const double* __restrict__ Ap = static_cast<const double*>(g.A.p[pb]);
  const double* __restrict__ Bp = static_cast<const double*>(g.B.p[pb]);
  const long long kbeg = split * g.kchunk;
  const long long kend = min(g.K, kbeg + g.kchunk);

  if (tid == 0) {
    long long a, b, c;
    decomp(g.gb, bi, a, b, c);
    bA = a;
    bB = b;
    bC = c;
  }
  for (int i = tid; i < BM; i += 256) {
    long long m = m0 + i, a = -1, b, c = -1;
    if (m < g.M) decomp(g.gm, m, a, b, c);
    oAm[i] = a;
    oCm[i] = c;
  }
  for (int i = tid; i < BN; i += 256) {
    long long n = n0 + i, a, b = -1, c = -1;
    if (n < g.N) decomp(g.gn, n, a, b, c);
    oBn[i] = b;
    oCn[i] = c;
  }

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (long long k0 = kbeg; k0 < kend; k0 += BK) {
    if (tid < BK) {
      long long k = k0 + tid, a = -1, b = -1, c;
      if (k < kend) decomp(g.gk, k, a, b, c);
      oAk[tid] = a;
      oBk[tid] = b;
    }
    __syncthreads();
    for (int e = tid; e < BK * BM; e += 256) {
      int kk = e / BM, mm = e % BM;
      long long om = oAm[mm], ok = oAk[kk];
      As[kk][mm] = (om >= 0 && ok >= 0) ? Ap[bA + om + ok] : 0.0;
    }
    for (int e = tid; e < BK * BN; e += 256) {
      int kk = e / BN, nn = e % BN;
      long long on = oBn[nn], ok = oBk[kk];
      Bs[kk][nn] = (on >= 0 && ok >= 0) ? Bp[bB + ok + on] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + TY * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + TX * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = ty + TY * i;
    const long long m = m0 + r;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = tx + TX * j;
      const long long n = n0 + c;
      if (n >= g.N) continue;
      if (g.splitk > 1) {
        g.part[((split * g.NB * g.nprob + bz) * g.M + m) * g.N + n] = acc[i][j];
      } else {
        double* p = static_cast<double*>(g.C.p[pb]) + bC + oCm[r] + oCn[c];
        double v = g.alpha * acc[i][j];
        if (g.beta != 0.0) v += g.beta * *p;
        *p = v;
      }
    }
  }
}

__global__ void k_splitk_reduce(const GemmArgs g) {
  const long long nbt = g.NB * g.nprob;
  const long long total = nbt * g.M * g.N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    long long n = t % g.N, m = (t / g.N) % g.M, bz = t / (g.N * g.M);
    double s = 0.0;
    for (int sp = 0; sp < g.splitk; ++sp) s += g.part[((sp * nbt + bz) * g.M + m) * g.N + n];
    long long a, b, cb, cm, cn;
    decomp(g.gb, bz % g.NB, a, b, cb);
    decomp(g.gm, m, a, b, cm);
    decomp(g.gn, n, a, b, cn);
    double* p = static_cast<double*>(g.C.p[bz / g.NB]) + cb + cm + cn;
    double v = g.alpha * s;
    if (g.beta != 0.0) v += g.beta * *p;
    *p = v;
  }
}

// Few outputs, long K (density matrices, scalars): each block reduces one K
// chunk for every output at once; partials are summed in a fixed order.
constexpr int DOT_MAXP = 16;

// Grid = (K chunks, problems).
__global__ void __launch_bounds__(256) k_dot_partial(const GemmArgs g, long long kchunk, double* part) {
  __shared__ long long oa[DOT_MAXP], ob[DOT_MAXP];
  __shared__ double red[8][DOT_MAXP];
  const int P = int(g.M * g.N * g.NB);
  const int tid = threadIdx.x;
  const int pb = blockIdx.y;
  const double* __restrict__ Ap = static_cast<const double*>(g.A.p[pb]);
  const double* __restrict__ Bp = static_cast<const double*>(g.B.p[pb]);
  if (tid < P) {
    const long long bi = tid / (g.M * g.N), mn = tid % (g.M * g.N), m = mn / g.N, n = mn % g.N;
    long long a0, b0, c0, a1, b1, c1, a2, b2, c2;
    decomp(g.gb, bi, a0, b0, c0);
    decomp(g.gm, m, a1, b1, c1);
    decomp(g.gn, n, a2, b2, c2);
    oa[tid] = a0 + a1;
    ob[tid] = b0 + b2;
  }
  __syncthreads();
  double acc[DOT_MAXP];
#pragma unroll
  for (int p = 0; p < DOT_MAXP; ++p) acc[p] = 0.0;
  const long long k0 = blockIdx.x * kchunk, k1 = min(g.K, k0 + kchunk);
  for (long long k = k0 + tid; k < k1; k += blockDim.x) {
    long long ka, kb, kc;
    decomp(g.gk, k, ka, kb, kc);
#pragma unroll
    for (int p = 0; p < DOT_MAXP; ++p)
      if (p < P) acc[p] = fma(Ap[oa[p] + ka], Bp[ob[p] + kb], acc[p]);
  }
  const int lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int p = 0; p < DOT_MAXP; ++p) {
    if (p >= P) break;
    double v = acc[p];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[w][p] = v;
  }
  __syncthreads();
  if (tid < P) {
    double v = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) v += red[i][tid];
    part[((long long)pb * gridDim.x + blockIdx.x) * DOT_MAXP + tid] = v;
  }
}

// Grid = problems.
__global__ void k_dot_finish(const GemmArgs g, int nblk, const double* part) {
  const int P = int(g.M * g.N * g.NB);
  const int p = threadIdx.x;
  const int pb = blockIdx.x;
  if (p >= P) return;
  double v = 0.0;
  for (int b = 0; b < nblk; ++b) v += part[((long long)pb * nblk + b) * DOT_MAXP + p];
  const long long bi = p / (g.M * g.N), mn = p % (g.M * g.N), m = mn / g.N, n = mn % g.N;
  long long a, b, c0, c1, c2;
  decomp(g.gb, bi, a, b, c0);
  decomp(g.gm, m, a, b, c1);
  decomp(g.gn, n, a, b, c2);
  double* out = static_cast<double*>(g.C.p[pb]) + c0 + c1 + c2;
  double r = g.alpha * v;
  if (g.beta != 0.0) r += g.beta * *out;
  *out = r;
}

struct Parsed {
  std::string a, b, c;
};

Parsed parse(const char* spec) {
  std::string s(spec);
  auto comma = s.find(',');
  auto arrow = s.find("->");
  PEPS_REQUIRE(comma != std::string::npos && arrow != std::string::npos && comma < arrow,
               std::string("bad contraction spec ") + spec);
  return {s.substr(0, comma), s.substr(comma + 1, arrow - comma - 1), s.substr(arrow + 2)};
}

std::vector<long long> strides_of(const Dims& d) {
  std::vector<long long> s(d.size());
  long long acc = 1;
  for (int i = int(d.size()) - 1; i >= 0; --i) {
    s[i] = acc;
    acc *= d[i];
  }
  return s;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

}  // namespace

Dims ein_dims(const char* spec, const Dims& ad, const Dims& bd) {
  Parsed p = parse(spec);
  PEPS_REQUIRE(p.a.size() == ad.size() && p.b.size() == bd.size(),
               std::string("operand rank mismatch in ") + spec);
  Dims out;
  for (char ch : p.c) {
    auto ia = p.a.find(ch);
    auto ib = p.b.find(ch);
    PEPS_REQUIRE(ia != std::string::npos || ib != std::string::npos,
                 std::string("output index not in operands: ") + spec);
    out.push_back(ia != std::string::npos ? ad[ia] : bd[ib]);
  }
  return out;
}

TP strided(double* base, int count, size_t per) {
  TP t;
  t.n = count;
  const size_t stride = (per + 31) / 32 * 32;
  for (int b = 0; b < count; ++b) t.p[b] = base + b * stride;
  return t;
}

int problems(std::initializer_list<const TP*> args) {
  int B = 1;
  for (const TP* t : args) B = std::max(B, t->n);
  for (const TP* t : args) PEPS_REQUIRE(t->n <= 1 || t->n == B, "internal: problem counts differ");
  PEPS_REQUIRE(B <= MAXB, "internal: too many problems in one launch");
  return B;
}

void ein(Ctx& cx, const char* spec, const TP& A, const Dims& ad, const TP& B,
         const Dims& bd, const TP& C, double alpha, double beta) {
  Parsed p = parse(spec);
  Dims cd = ein_dims(spec, ad, bd);
  auto sa = strides_of(ad), sb = strides_of(bd), sc = strides_of(cd);
  const int np = problems({&A, &B, &C});
  PEPS_REQUIRE(!A.null() && !B.null() && C.n == np, "internal: contraction operands");
  GemmArgs g;
  std::memset(static_cast<void*>(&g), 0, sizeof(g));
  g.A = A.all(np);
  g.B = B.all(np);
  g.C = C.all(np);
  g.nprob = np;
  g.alpha = alpha;
  g.beta = beta;
  auto push = [&](Grp& gr, int dim, long long a, long long b, long long c) {
    PEPS_REQUIRE(gr.n < MAXG, std::string("too many indices in one group: ") + spec);
    gr.dim[gr.n] = dim;
    gr.sa[gr.n] = a;
    gr.sb[gr.n] = b;
    gr.sc[gr.n] = c;
    gr.n++;
  };
  // M, N and batch groups in C's order (so the fastest C index is last).
  for (size_t i = 0; i < p.c.size(); ++i) {
    char ch = p.c[i];
    auto ia = p.a.find(ch), ib = p.b.find(ch);
    bool inA = ia != std::string::npos, inB = ib != std::string::npos;
    if (inA && inB) {
      PEPS_REQUIRE(ad[ia] == bd[ib], std::string("dim mismatch in ") + spec);
      push(g.gb, cd[i], sa[ia], sb[ib], sc[i]);
    } else if (inA) {
      push(g.gm, cd[i], sa[ia], 0, sc[i]);
    } else {
      push(g.gn, cd[i], 0, sb[ib], sc[i]);
    }
  }
  // K group in A's order.  An index summed in one operand only has stride 0 in
  // the other (sum_e A[..e..] B = (sum_e A) B).
  for (size_t i = 0; i < p.a.size(); ++i) {
    char ch = p.a[i];
    if (p.c.find(ch) != std::string::npos) continue;
    auto ib = p.b.find(ch);
    if (ib != std::string::npos) {
      PEPS_REQUIRE(ad[i] == bd[ib], std::string("dim mismatch in ") + spec);
      push(g.gk, ad[i], sa[i], sb[ib], 0);
    } else {
      push(g.gk, ad[i], sa[i], 0, 0);
    }
  }
  for (size_t i = 0; i < p.b.size(); ++i) {
    char ch = p.b[i];
    if (p.c.find(ch) == std::string::npos && p.a.find(ch) == std::string::npos) push(g.gk, bd[i], 0, sb[i], 0);
  }
  auto prodg = [](const Grp& gr) {
    long long n = 1;
    for (int i = 0; i < gr.n; ++i) n *= gr.dim[i];
    return n;
  };
  g.M = prodg(g.gm);
  g.N = prodg(g.gn);
  g.K = prodg(g.gk);
  g.NB = prodg(g.gb);
  if (g.M == 0 || g.N == 0 || g.NB == 0) return;
  if (g.K == 0) {
    PEPS_REQUIRE(false, "empty contraction dimension");
  }
  PEPS_REQUIRE(g.NB * np <= 65535, "batch too large");

  if (g.M * g.N * g.NB <= DOT_MAXP && g.K >= 1024) {
    const long long kchunk = 2048;
    const int nblk = int(std::max<long long>(1, std::min<long long>((g.K + kchunk - 1) / kchunk, 4 * num_sms() / np)));
    const long long kc = (g.K + nblk - 1) / nblk;
    double* part = cx.scratch(size_t(nblk) * np * DOT_MAXP);
    Launch L(cx.f64_class >= 0 ? KClass(cx.f64_class) : K_GEMM_F64, cx.st,
             cx.f64_flops ? 2.0 * double(g.M * g.N * g.NB) * double(g.K) * np : 0.0, 0);
    k_dot_partial<<<dim3(nblk, np), 256, 0, cx.st>>>(g, kc, part);
    k_dot_finish<<<np, 32, 0, cx.st>>>(g, nblk, part);
    L.more();
    PEPS_CHECK_LAUNCH();
    return;
  }
  // Tile shape: minimise padded area, prefer square.
  static const int BMs[5] = {16, 32, 64, 128, 256};
  int best = 2;
  double bestw = 1e300;
  for (int t = 0; t < 5; ++t) {
    int bm = BMs[t], bn = 4096 / bm;
    double w = double(cdiv(g.M, bm)) * bm * double(cdiv(g.N, bn)) * bn;
    w *= (t == 2 ? 1.0 : 1.05);
    if (w < bestw) {
      bestw = w;
      best = t;
    }
  }
  const int BM = BMs[best], BN = 4096 / BM;
  const long long tiles = (long long)cdiv(g.M, BM) * cdiv(g.N, BN);
  const long long ctas = tiles * g.NB * np;
  const int target = 2 * num_sms();
  int splitk = 1;
  if (ctas < target) {
    long long want = (target + ctas - 1) / ctas;
    long long maxs = std::max<long long>(1, g.K / 64);
    splitk = int(std::min<long long>({want, maxs, 64}));
  }
  g.kchunk = ((g.K + splitk - 1) / splitk + BK - 1) / BK * BK;
  splitk = int((g.K + g.kchunk - 1) / g.kchunk);
  g.splitk = splitk;
  if (splitk > 1) g.part = cx.scratch(size_t(splitk) * g.NB * np * g.M * g.N);
  PEPS_REQUIRE(tiles < (1LL << 31), "too many tiles");

  const double flops = 2.0 * double(g.M) * double(g.N) * double(g.K) * double(g.NB) * np;
  {
    Launch L(cx.f64_class >= 0 ? KClass(cx.f64_class) : K_GEMM_F64, cx.st, cx.f64_flops ? flops : 0.0, 0);
    dim3 grid(unsigned(tiles), unsigned(splitk), unsigned(g.NB * np));
    switch (BM) {
      case 16: k_gemm_f64<16, 256><<<grid, 256, 0, cx.st>>>(g); break;
      case 32: k_gemm_f64<32, 128><<<grid, 256, 0, cx.st>>>(g); break;
      case 64: k_gemm_f64<64, 64><<<grid, 256, 0, cx.st>>>(g); break;
      case 128: k_gemm_f64<128, 32><<<grid, 256, 0, cx.st>>>(g); break;
      default: k_gemm_f64<256, 16><<<grid, 256, 0, cx.st>>>(g); break;
    }
    PEPS_CHECK_LAUNCH();
  }
  if (splitk > 1) {
    Launch L(K_AUX, cx.st);
    long long total = g.NB * np * g.M * g.N;
    unsigned blocks = unsigned(std::min<long long>((total + 255) / 256, 4 * 1024));
    k_splitk_reduce<<<blocks, 256, 0, cx.st>>>(g);
    PEPS_CHECK_LAUNCH();
  }
}

}  // namespace peps
