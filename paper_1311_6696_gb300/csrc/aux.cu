// Auxiliary kernels: lattice repacking, OBC validation, norms and rescaling,
// counter-based var initialisation, local observables and CU_0.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "aux.cuh"
#include "linalg.cuh"

namespace peps {
namespace {

constexpr int RED_BLOCKS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

__global__ void k_orient(const void* src, int f32, int Lx, int d, int D, const OrientSite* sites,
                         double* dst) {
  const OrientSite s = sites[blockIdx.x];
  const int dims[4] = {s.du, s.dl, s.dn, s.dr};
  const int n = d * s.du * s.dl * s.dn * s.dr;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    int t = e;
    int idx[4];
    for (int k = 3; k >= 0; --k) {
      idx[k] = t % dims[k];
      t /= dims[k];
    }
    const int ph = t;
    int o[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4; ++k) o[s.perm[k]] = idx[k];
    const long long so = (((((long long)s.y * Lx + s.x) * d + ph) * D + o[0]) * D + o[1]) * D * D +
                         (long long)o[2] * D + o[3];
    dst[s.dst + e] = f32 ? double(static_cast<const float*>(src)[so])
                         : static_cast<const double*>(src)[so];
  }
}

// count[0]: nonzero entries on outward (OBC) legs; count[1]: non-finite entries.
__global__ void k_obc_count(const void* src, int f32, int Ly, int Lx, int d, int D,
                            unsigned long long* count) {
  const long long per = (long long)d * D * D * D * D;
  const long long total = (long long)Ly * Lx * per;
  unsigned long long c = 0, nf = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const double ve = f32 ? double(static_cast<const float*>(src)[e]) : static_cast<const double*>(src)[e];
    if (!isfinite(ve)) ++nf;
    const long long site = e / per;
    const int y = int(site / Lx), x = int(site % Lx);
    long long r = e % per;
    const int ri = int(r % D);
    r /= D;
    const int ni = int(r % D);
    r /= D;
    const int li = int(r % D);
    r /= D;
    const int ui = int(r % D);
    const bool out = (y == 0 && ui) || (x == 0 && li) || (y == Ly - 1 && ni) || (x == Lx - 1 && ri);
    if (out) {
      const double v = f32 ? double(static_cast<const float*>(src)[e]) : static_cast<const double*>(src)[e];
      if (v != 0.0) ++c;
    }
  }
  if (c) atomicAdd(count, c);
  if (nf) atomicAdd(count + 1, nf);
}

__global__ void k_plant_nan(void* p, int f32) {
  if (f32)
    static_cast<float*>(p)[0] = __int_as_float(0x7fc00000);
  else
    static_cast<double*>(p)[0] = __longlong_as_double(0x7ff8000000000000LL);
}

// Spins on a flag nothing sets, for at most budget_ns of the global timer,
// then records a timeout in the status word: the same bounded-wait shape as
// the library's other device-side waits, with a wait that is certain to run out.
__global__ void k_wait_unset(const volatile int* never, long long budget_ns, int* status) {
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (*never == 0) {
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if ((long long)(t - t0) > budget_ns) {
      atomicOr(status, FLAG_TIMEOUT);
      return;
    }
  }
}

// Batched element-wise kernels: grid = (blocks, problems), problem = blockIdx.y.
__global__ void k_sumsq_partial(const TP x, long long n, double* part) {
  __shared__ double red[32];
  const double* xp = x.d(blockIdx.y);
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = xp[i];
    s += v * v;
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// Grid = problems.
__global__ void k_sumsq_finish(const double* part, int np, const TP out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[(long long)blockIdx.x * np + i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out.d(blockIdx.x)[0] = sqrt(s);
}

__global__ void k_rescale(const TP x, long long n, const TP nrm, const TP lnacc, int* flag) {
  const int pb = blockIdx.y;
  const double v = nrm.d(pb)[0];
  const bool ok = v > 0.0 && isfinite(v);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (!ok && flag) atomicOr(flag, FLAG_BAD_VALUE);
    if (lnacc.n && ok) lnacc.d(pb)[0] += log(v);
  }
  if (!ok) return;
  const double inv = 1.0 / v;
  double* xp = x.d(pb);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    xp[i] *= inv;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

struct VarInitArgs {
  TP src;
  int s0, s1, s2, s3;
  TP dst;
  int d0, d1, d2, d3;
  unsigned long long key;
  TP srcnorm;
};

__global__ void k_var_init(const VarInitArgs a) {
  const int pb = blockIdx.y;
  const double* src = a.src.d(pb);
  double* dst = a.dst.d(pb);
  const long long n = (long long)a.d0 * a.d1 * a.d2 * a.d3;
  const double scale = 1e-3 * a.srcnorm.d(pb)[0] / sqrt(double(n));
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    long long t = e;
    const int i3 = int(t % a.d3);
    t /= a.d3;
    const int i2 = int(t % a.d2);
    t /= a.d2;
    const int i1 = int(t % a.d1);
    const int i0 = int(t / a.d1);
    const bool inside = i0 < a.s0 && i1 < a.s1 && i2 < a.s2 && i3 < a.s3;
    if (inside) {
      dst[e] = src[(((long long)i0 * a.s1 + i1) * a.s2 + i2) * a.s3 + i3];
    } else {
      const unsigned long long z = mix64(a.key + (unsigned long long)e + 0x9E3779B97F4A7C15ULL);
      const double u = double(z >> 11) * (1.0 / 4503599627370496.0) - 1.0;   // 2^-52
      dst[e] = scale * u;
    }
  }
}

__global__ void k_expect(const double* rho, int count, int k, const double* op, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double* r = rho + (long long)i * k * k;
  double num = 0.0, tr = 0.0;
  for (int a = 0; a < k; ++a) {
    tr += r[a * k + a];
    for (int b = 0; b < k; ++b) num += r[a * k + b] * op[b * k + a];
  }
  out[i] = num / tr;
}

__global__ void k_finish_norm(const double* lns, int nl, const double* extra, const double* s,
                              double* out_ln, double* out_sign) {
  if (threadIdx.x || blockIdx.x) return;
  double acc = extra ? extra[0] : 0.0;
  for (int i = 0; i < nl; ++i) acc += lns[i];
  const double v = s[0];
  out_ln[0] = acc + log(fabs(v));
  out_sign[0] = v > 0 ? 1.0 : (v < 0 ? -1.0 : 0.0);
}

__global__ void k_fill(const TP x, long long n, double v) {
  double* xp = x.d(blockIdx.y);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    xp[i] = v;
}

__global__ void k_copy(const TP dst, const TP src, long long n) {
  double* dp = dst.d(blockIdx.y);
  const double* sp = src.d(blockIdx.y);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dp[i] = sp[i];
}

unsigned grid_for(long long n) {
  return unsigned(std::max<long long>(1, std::min<long long>((n + 255) / 256, 2048)));
}

// ----------------------------------------------------------------------------
// CU_0 (Section 5.1): one CTA per oriented lattice.
// ----------------------------------------------------------------------------
struct SiteDims {
  int du, dl, dn, dr;
};

__device__ __forceinline__ long long aidx(const SiteDims& s, int ph, int u, int l, int n, int r) {
  return ((((long long)ph * s.du + u) * s.dl + l) * s.dn + n) * s.dr + r;
}

// b[n,o] = sum Lm[l,m] S[u,v] A[s,u,l,n,r] A[s,v,m,o,q] Rm[r,q]   (O(d D^5))
__device__ void cu0_local(const double* Lm, const double* S, const double* A, const SiteDims& sd,
                          int d, const double* Rm, double* Y, double* Z, double* b) {
  const int du = sd.du, dl = sd.dl, dn = sd.dn, dr = sd.dr;
  const int tid = threadIdx.x, nt = blockDim.x;
  // Y[s,m,u,n,r] = sum_l Lm[l,m] A[s,u,l,n,r]
  const int nY = d * dl * du * dn * dr;
  for (int e = tid; e < nY; e += nt) {
    int t = e;
    const int r = t % dr; t /= dr;
    const int n = t % dn; t /= dn;
    const int u = t % du; t /= du;
    const int m = t % dl; t /= dl;
    const int s = t;
    double acc = 0.0;
    for (int l = 0; l < dl; ++l) acc += Lm[l * dl + m] * A[aidx(sd, s, u, l, n, r)];
    Y[e] = acc;
  }
  __syncthreads();
  // Z[s,m,v,n,r] = sum_u Y[s,m,u,n,r] S[u,v]
  for (int e = tid; e < nY; e += nt) {
    int t = e;
    const int r = t % dr; t /= dr;
    const int n = t % dn; t /= dn;
    const int v = t % du; t /= du;
    const int sm = t;   // s*dl + m
    double acc = 0.0;
    for (int u = 0; u < du; ++u) acc += Y[(((long long)sm * du + u) * dn + n) * dr + r] * S[u * du + v];
    Z[e] = acc;
  }
  __syncthreads();
  // Y[s,m,v,n,q] = sum_r Z[s,m,v,n,r] Rm[r,q]
  for (int e = tid; e < nY; e += nt) {
    const int q = e % dr;
    const long long base = (long long)(e / dr) * dr;
    double acc = 0.0;
    for (int r = 0; r < dr; ++r) acc += Z[base + r] * Rm[r * dr + q];
    Y[e] = acc;
  }
  __syncthreads();
  // b[n,o] = sum_{s,m,v,q} Y[s,m,v,n,q] A[s,v,m,o,q]
  for (int e = tid; e < dn * dn; e += nt) {
    const int n = e / dn, o = e % dn;
    double acc = 0.0;
    for (int s = 0; s < d; ++s)
      for (int m = 0; m < dl; ++m)
        for (int v = 0; v < du; ++v)
          for (int q = 0; q < dr; ++q)
            acc += Y[((((long long)s * dl + m) * du + v) * dn + n) * dr + q] * A[aidx(sd, s, v, m, o, q)];
    b[e] = acc;
  }
  __syncthreads();
}

// L'[r,q] = sum Lm[l,m] S[u,v] A[s,u,l,n,r] A[s,v,m,o,q] N[n,o]
__device__ void cu0_lenv(const double* Lm, const double* S, const double* A, const SiteDims& sd,
                         int d, const double* N, double* Y, double* Z, double* out) {
  const int du = sd.du, dl = sd.dl, dn = sd.dn, dr = sd.dr;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nY = d * dl * du * dn * dr;
  for (int e = tid; e < nY; e += nt) {
    int t = e;
    const int r = t % dr; t /= dr;
    const int n = t % dn; t /= dn;
    const int u = t % du; t /= du;
    const int m = t % dl; t /= dl;
    const int s = t;
    double acc = 0.0;
    for (int l = 0; l < dl; ++l) acc += Lm[l * dl + m] * A[aidx(sd, s, u, l, n, r)];
    Y[e] = acc;
  }
  __syncthreads();
  for (int e = tid; e < nY; e += nt) {
    int t = e;
    const int r = t % dr; t /= dr;
    const int n = t % dn; t /= dn;
    const int v = t % du; t /= du;
    const int sm = t;
    double acc = 0.0;
    for (int u = 0; u < du; ++u) acc += Y[(((long long)sm * du + u) * dn + n) * dr + r] * S[u * du + v];
    Z[e] = acc;
  }
  __syncthreads();
  // Y[s,m,v,o,r] = sum_n Z[s,m,v,n,r] N[n,o]
  for (int e = tid; e < nY; e += nt) {
    int t = e;
    const int r = t % dr; t /= dr;
    const int o = t % dn; t /= dn;
    const int smv = t;
    double acc = 0.0;
    for (int n = 0; n < dn; ++n) acc += Z[((long long)smv * dn + n) * dr + r] * N[n * dn + o];
    Y[e] = acc;
  }
  __syncthreads();
  // out[r,q] = sum_{s,m,v,o} Y[s,m,v,o,r] A[s,v,m,o,q]
  for (int e = tid; e < dr * dr; e += nt) {
    const int r = e / dr, q = e % dr;
    double acc = 0.0;
    for (int s = 0; s < d; ++s)
      for (int m = 0; m < dl; ++m)
        for (int v = 0; v < du; ++v)
          for (int o = 0; o < dn; ++o)
            acc += Y[((((long long)s * dl + m) * du + v) * dn + o) * dr + r] * A[aidx(sd, s, v, m, o, q)];
    out[e] = acc;
  }
  __syncthreads();
}

// R'[l,m] = sum Rm[r,q] S[u,v] A[s,u,l,n,r] A[s,v,m,o,q] N[n,o]
__device__ void cu0_renv(const double* Rm, const double* S, const double* A, const SiteDims& sd,
                         int d, const double* N, double* Y, double* Z, double* out) {
  const int du = sd.du, dl = sd.dl, dn = sd.dn, dr = sd.dr;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nY = d * du * dl * dn * dr;
  // Y[s,u,l,n,q] = sum_r Rm[r,q] A[s,u,l,n,r]
  for (int e = tid; e < nY; e += nt) {
    const int q = e % dr;
    const long long base = (long long)(e / dr) * dr;
    double acc = 0.0;
    for (int r = 0; r < dr; ++r) acc += A[base + r] * Rm[r * dr + q];
    Y[e] = acc;
  }
  __syncthreads();
  // Z[s,v,l,n,q] = sum_u Y[s,u,l,n,q] S[u,v]
  for (int e = tid; e < nY; e += nt) {
    int t = e;
    const int q = t % dr; t /= dr;
    const int n = t % dn; t /= dn;
    const int l = t % dl; t /= dl;
    const int v = t % du; t /= du;
    const int s = t;
    double acc = 0.0;
    for (int u = 0; u < du; ++u) acc += Y[aidx(sd, s, u, l, n, q)] * S[u * du + v];
    Z[e] = acc;
  }
  __syncthreads();
  // Y[s,v,l,o,q] = sum_n Z[s,v,l,n,q] N[n,o]
  for (int e = tid; e < nY; e += nt) {
    int t = e;
    const int q = t % dr; t /= dr;
    const int o = t % dn; t /= dn;
    const int svl = t;
    double acc = 0.0;
    for (int n = 0; n < dn; ++n) acc += Z[((long long)svl * dn + n) * dr + q] * N[n * dn + o];
    Y[e] = acc;
  }
  __syncthreads();
  // out[l,m] = sum_{s,v,o,q} Y[s,v,l,o,q] A[s,v,m,o,q]
  for (int e = tid; e < dl * dl; e += nt) {
    const int l = e / dl, m = e % dl;
    double acc = 0.0;
    for (int s = 0; s < d; ++s)
      for (int v = 0; v < du; ++v)
        for (int o = 0; o < dn; ++o)
          for (int q = 0; q < dr; ++q)
            acc += Y[aidx(sd, s, v, l, o, q)] * A[aidx(sd, s, v, m, o, q)];
    out[e] = acc;
  }
  __syncthreads();
}

__device__ double cta_fro_normalize(double* x, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i] * x[i];
  s = sqrt(block_sum(s, red));
  const double inv = s > 0.0 ? 1.0 / s : 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] *= inv;
  __syncthreads();
  return s;
}

// Infinite lattice (Section 5.4): the dominant separable boundary of a row of
// copies of one tensor, from one side per CTA.  Each step moves the left and
// the right fixed-point environments of the row once and then the boundary
// matrix (the local CU_0 update between it and itself), all to unit norm;
// identities to start; stops when none moves by tol, else at max_iter.
struct Cu0Inf {
  const double* A[4];   // the tensor in the four sweep orientations, [s][u][l][n][r], all legs D
  double* sigma;        // [4][D][D]
  double* work;         // 4 x cu0_inf_work(d, D) doubles
  int d, D, max_iter;
  double tol;
  int* flag;
};

__global__ void __launch_bounds__(256) k_cu0_inf(const Cu0Inf a) {
  __shared__ double red[32];
  const int o = blockIdx.x, D = a.D, DD = D * D, d = a.d;
  const int tid = threadIdx.x, nt = blockDim.x;
  const SiteDims sd{D, D, D, D};
  const long long big = (long long)d * DD * DD;
  double* Y = a.work + o * (2 * big + 6 * DD + 32);
  double* Z = Y + big;
  double* sig = Z + big;
  double* L = sig + DD;
  double* R = L + DD;
  double* Ln = R + DD;
  double* Rn = Ln + DD;
  double* b = Rn + DD;
  const double* A = a.A[o];
  const double v0 = 1.0 / sqrt(double(D));
  for (int e = tid; e < DD; e += nt) {
    const double v = (e / D == e % D) ? v0 : 0.0;
    sig[e] = v;
    L[e] = v;
    R[e] = v;
  }
  __syncthreads();
  bool conv = false;
  for (int it = 0; it < a.max_iter && !conv; ++it) {
    cu0_lenv(L, sig, A, sd, d, sig, Y, Z, Ln);
    cta_fro_normalize(Ln, DD, red);
    cu0_renv(R, sig, A, sd, d, sig, Y, Z, Rn);
    cta_fro_normalize(Rn, DD, red);
    cu0_local(Ln, sig, A, sd, d, Rn, Y, Z, b);
    cta_fro_normalize(b, DD, red);
    double c1 = 0.0, c2 = 0.0, c3 = 0.0;
    for (int e = tid; e < DD; e += nt) {
      c1 += (Ln[e] - L[e]) * (Ln[e] - L[e]);
      c2 += (Rn[e] - R[e]) * (Rn[e] - R[e]);
      c3 += (b[e] - sig[e]) * (b[e] - sig[e]);
    }
    c1 = sqrt(block_sum(c1, red));
    c2 = sqrt(block_sum(c2, red));
    c3 = sqrt(block_sum(c3, red));
    for (int e = tid; e < DD; e += nt) {
      L[e] = Ln[e];
      R[e] = Rn[e];
      sig[e] = b[e];
    }
    __syncthreads();
    conv = fmax(c1, fmax(c2, c3)) < a.tol;
  }
  if (!conv && tid == 0) atomicOr(a.flag, FLAG_CU0_NOCONV);
  for (int e = tid; e < DD; e += nt) a.sigma[(long long)o * DD + e] = sig[e];
}

// A site of a CU_0 row: its tensor and effective leg dimensions.
struct Cu0Site {
  const double* A;
  SiteDims sd;
};

// One cut of the separable boundary (Section 5.1): ALS half-sweeps over the
// row's sites that fit the matrices nxt(x) (on the down legs of site x)
// between the row and the matrices above it, prv(x).  On entry nxt holds the
// start and Lm[0], Rm[(Lx-1)*DM2] the row's left / right closures; the right
// environments are built here.  Each local update is b_x itself, scaled to
// unit Frobenius norm.  Returns whether a half-sweep moved no matrix by tol.
// site(x) may stage the tensor in scratch (it is called again for every use).
template <class SiteF, class PrvF, class NxtF>
__device__ bool cu0_cut(int Lx, int d, int DM2, SiteF site, PrvF prv, NxtF nxt, double* Lm, double* Rm, double* Y,
                        double* Z, double* b, int max_half, double tol, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int x = Lx - 1; x >= 1; --x) {
    const Cu0Site st = site(x);
    cu0_renv(Rm + (long long)x * DM2, prv(x), st.A, st.sd, d, nxt(x), Y, Z, Rm + (long long)(x - 1) * DM2);
    cta_fro_normalize(Rm + (long long)(x - 1) * DM2, st.sd.dl * st.sd.dl, red);
  }
  bool conv = false;
  for (int h = 0; h < max_half && !conv; ++h) {
    double change = 0.0;
    for (int step = 0; step < Lx; ++step) {
      const int x = (h % 2 == 0) ? step : Lx - 1 - step;
      const Cu0Site st = site(x);
      const SiteDims sd = st.sd;
      cu0_local(Lm + (long long)x * DM2, prv(x), st.A, sd, d, Rm + (long long)x * DM2, Y, Z, b);
      cta_fro_normalize(b, sd.dn * sd.dn, red);
      double* cur = nxt(x);
      double part = 0.0;
      for (int e = tid; e < sd.dn * sd.dn; e += nt) {
        const double df = b[e] - cur[e];
        part += df * df;
      }
      change = fmax(change, sqrt(block_sum(part, red)));
      for (int e = tid; e < sd.dn * sd.dn; e += nt) cur[e] = b[e];
      __syncthreads();
      if (h % 2 == 0 && x < Lx - 1) {
        cu0_lenv(Lm + (long long)x * DM2, prv(x), st.A, sd, d, cur, Y, Z, Lm + (long long)(x + 1) * DM2);
        cta_fro_normalize(Lm + (long long)(x + 1) * DM2, sd.dr * sd.dr, red);
      } else if (h % 2 == 1 && x > 0) {
        cu0_renv(Rm + (long long)x * DM2, prv(x), st.A, sd, d, cur, Y, Z, Rm + (long long)(x - 1) * DM2);
        cta_fro_normalize(Rm + (long long)(x - 1) * DM2, sd.dl * sd.dl, red);
      }
    }
    conv = change < tol;
  }
  return conv;
}

__global__ void __launch_bounds__(256) k_cu0(const Cu0Lattice* lats, int* flag) {
  __shared__ double red[32];
  const Cu0Lattice L = lats[blockIdx.x];
  const int Ly = L.Ly, Lx = L.Lx, d = L.d, DM2 = L.Dmax * L.Dmax;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long big = (long long)d * L.Dmax * L.Dmax * L.Dmax * L.Dmax;
  double* Y = L.work;
  double* Z = Y + big;
  double* Lm = Z + big;
  double* Rm = Lm + (long long)Lx * DM2;
  double* b = Rm + (long long)Lx * DM2;
  auto dims = [&](int y, int x) {
    const int* p = L.dims + 4 * (y * Lx + x);
    return SiteDims{p[0], p[1], p[2], p[3]};
  };
  auto site = [&](int y, int x) { return L.A + L.off[y * Lx + x]; };
  auto outm = [&](int r, int x) { return L.out + ((long long)r * Lx + x) * DM2; };
  // row 0: top closures
  for (int x = 0; x < Lx; ++x) {
    const int du = dims(0, x).du;
    for (int e = tid; e < du * du; e += nt) outm(0, x)[e] = L.top[(long long)x * DM2 + e];
  }
  __syncthreads();
  for (int r = 0; r + 1 < Ly; ++r) {
    // identity start, unit Frobenius norm
    for (int x = 0; x < Lx; ++x) {
      const int dn = dims(r, x).dn;
      const double v = 1.0 / sqrt(double(dn));
      for (int e = tid; e < dn * dn; e += nt) outm(r + 1, x)[e] = (e / dn == e % dn) ? v : 0.0;
    }
    __syncthreads();
    {
      const int dr = dims(r, Lx - 1).dr;
      for (int e = tid; e < dr * dr; e += nt) Rm[(long long)(Lx - 1) * DM2 + e] = L.right[(long long)r * DM2 + e];
      const int dl = dims(r, 0).dl;
      for (int e = tid; e < dl * dl; e += nt) Lm[e] = L.left[(long long)r * DM2 + e];
    }
    __syncthreads();
    const bool conv = cu0_cut(
        Lx, d, DM2, [&](int x) { return Cu0Site{site(r, x), dims(r, x)}; }, [&](int x) { return outm(r, x); },
        [&](int x) { return outm(r + 1, x); }, Lm, Rm, Y, Z, b, L.max_half, L.tol, red);
    if (!conv && tid == 0) atomicOr(flag, FLAG_CU0_NOCONV);
    __syncthreads();
  }
}

}  // namespace

void orient_lattice(Ctx& cx, const void* src, int src_f32, int /*Ly*/, int Lx, int d, int D,
                    const OrientSite* host_sites, int nsites, double* dst) {
  auto* dev = static_cast<const OrientSite*>(stage(cx, host_sites, sizeof(OrientSite) * nsites));
  Launch L(K_AUX, cx.st);
  k_orient<<<nsites, 256, 0, cx.st>>>(src, src_f32, Lx, d, D, dev, dst);
  PEPS_CHECK_LAUNCH();
}

void* stage(Ctx& cx, const void* host, size_t bytes) {
  if (!cx.persist) {
    void* dev = cx.ws->alloc(bytes);
    PEPS_CUDA(cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, cx.st));
    PEPS_CUDA(cudaStreamSynchronize(cx.st));   // the host buffer may go out of scope
    return dev;
  }
  // Recording a graph: copy now, on a private stream that takes no part in the capture.
  static std::mutex mu;
  static cudaStream_t side[64] = {};
  int dev_id = 0;
  PEPS_CUDA(cudaGetDevice(&dev_id));
  PEPS_REQUIRE(dev_id < 64, "device index above 63");
  void* dev = cx.persist->alloc(bytes);
  std::lock_guard<std::mutex> g(mu);
  if (!side[dev_id]) PEPS_CUDA(cudaStreamCreateWithFlags(&side[dev_id], cudaStreamNonBlocking));
  PEPS_CUDA(cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, side[dev_id]));
  PEPS_CUDA(cudaStreamSynchronize(side[dev_id]));
  return dev;
}

void cu0_infinite(Ctx& cx, const double* const A[4], int d, int D, double* sigma, int max_iter) {
  const long long DD = (long long)D * D, big = (long long)d * DD * DD;
  double* work = cx.ws->dalloc(size_t(4) * (2 * big + 6 * DD + 32));
  Cu0Inf a;
  for (int o = 0; o < 4; ++o) a.A[o] = A[o];
  a.sigma = sigma;
  a.work = work;
  a.d = d;
  a.D = D;
  a.max_iter = max_iter;
  a.tol = 1e-13;
  a.flag = cx.flag;
  Launch L(K_CU0, cx.st, 0, 0);
  k_cu0_inf<<<4, 256, 0, cx.st>>>(a);
  PEPS_CHECK_LAUNCH();
}

std::pair<long long, long long> input_violations_device(Ctx& cx, const void* src, int src_f32, int Ly, int Lx,
                                                        int d, int D) {
  auto* cnt = static_cast<unsigned long long*>(cx.ws->alloc(2 * sizeof(unsigned long long)));
  PEPS_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), cx.st));
  {
    Launch L(K_AUX, cx.st);
    k_obc_count<<<1024, 256, 0, cx.st>>>(src, src_f32, Ly, Lx, d, D, cnt);
    PEPS_CHECK_LAUNCH();
  }
  unsigned long long h[2] = {0, 0};
  PEPS_CUDA(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, cx.st));
  PEPS_CUDA(cudaStreamSynchronize(cx.st));
  return {(long long)h[0], (long long)h[1]};
}

void plant_nan_value(Ctx& cx, void* p, int f32) {
  Launch L(K_AUX, cx.st);
  k_plant_nan<<<1, 1, 0, cx.st>>>(p, f32);
  PEPS_CHECK_LAUNCH();
}

void wait_unset_flag(Ctx& cx, long long budget_ns) {
  int* never = static_cast<int*>(cx.ws->alloc(sizeof(int)));
  PEPS_CUDA(cudaMemsetAsync(never, 0, sizeof(int), cx.st));
  Launch L(K_AUX, cx.st);
  k_wait_unset<<<1, 1, 0, cx.st>>>(never, budget_ns, cx.flag);
  PEPS_CHECK_LAUNCH();
}

void fro_norm(Ctx& cx, const TP& x, long long n, const TP& out) {
  const int np = problems({&x, &out});
  const unsigned nb = unsigned(std::max<long long>(1, std::min<long long>(RED_BLOCKS, (n + 255) / 256)));
  double* part = cx.scratch(size_t(nb) * np);
  Launch L(K_AUX, cx.st);
  k_sumsq_partial<<<dim3(nb, np), 256, 0, cx.st>>>(x.all(np), n, part);
  k_sumsq_finish<<<np, 256, 0, cx.st>>>(part, int(nb), out.all(np));
  L.more();
  PEPS_CHECK_LAUNCH();
}

void rescale(Ctx& cx, const TP& x, long long n, const TP& nrm, const TP& lnacc) {
  const int np = problems({&x, &nrm, &lnacc});
  Launch L(K_AUX, cx.st);
  k_rescale<<<dim3(grid_for(n), np), 256, 0, cx.st>>>(x.all(np), n, nrm.all(np), lnacc.all(np), cx.flag);
  PEPS_CHECK_LAUNCH();
}

void normalize(Ctx& cx, const TP& x, long long n, const TP& lnacc, const TP& tmp) {
  const TP t = tmp.null() ? TP(cx.tmp) : tmp;
  fro_norm(cx, x, n, t);
  rescale(cx, x, n, t, lnacc);
}

void var_init(Ctx& cx, const TP& src, const int sdims[4], const TP& dst, const int ddims[4],
              unsigned long long seed, int tag, int y, int x, const TP& tmp) {
  const int np = problems({&src, &dst, &tmp});
  const long long ns = (long long)sdims[0] * sdims[1] * sdims[2] * sdims[3];
  const TP sn = tmp.null() ? TP(cx.tmp + 1) : tmp;
  fro_norm(cx, src, ns, sn);
  VarInitArgs a;
  a.src = src.all(np);
  a.s0 = sdims[0];
  a.s1 = sdims[1];
  a.s2 = sdims[2];
  a.s3 = sdims[3];
  a.dst = dst.all(np);
  a.d0 = ddims[0];
  a.d1 = ddims[1];
  a.d2 = ddims[2];
  a.d3 = ddims[3];
  a.key = seed * 0x9E3779B97F4A7C15ULL + ((unsigned long long)tag << 56) +
          ((unsigned long long)y << 44) + ((unsigned long long)x << 32);
  a.srcnorm = sn.all(np);
  const long long n = (long long)ddims[0] * ddims[1] * ddims[2] * ddims[3];
  Launch L(K_AUX, cx.st);
  k_var_init<<<dim3(grid_for(n), np), 256, 0, cx.st>>>(a);
  PEPS_CHECK_LAUNCH();
}

void expect_batch(Ctx& cx, const double* rho, int count, int k, const double* op, double* out) {
  Launch L(K_OBS, cx.st, 2.0 * count * k * k, 8.0 * count * k * k);
  k_expect<<<(count + 127) / 128, 128, 0, cx.st>>>(rho, count, k, op, out);
  PEPS_CHECK_LAUNCH();
}

void finish_norm(Ctx& cx, const double* lns, int nl, const double* extra, const double* s,
                 double* out_ln, double* out_sign) {
  Launch L(K_AUX, cx.st);
  k_finish_norm<<<1, 32, 0, cx.st>>>(lns, nl, extra, s, out_ln, out_sign);
  PEPS_CHECK_LAUNCH();
}

void fill(Ctx& cx, const TP& x, long long n, double v) {
  const int np = problems({&x});
  Launch L(K_AUX, cx.st);
  k_fill<<<dim3(grid_for(n), np), 256, 0, cx.st>>>(x.all(np), n, v);
  PEPS_CHECK_LAUNCH();
}

void copy(Ctx& cx, const TP& dst, const TP& src, long long n) {
  const int np = problems({&dst, &src});
  PEPS_REQUIRE(dst.n == np, "internal: copy destination");
  Launch L(K_AUX, cx.st);
  k_copy<<<dim3(grid_for(n), np), 256, 0, cx.st>>>(dst.all(np), src.all(np), n);
  PEPS_CHECK_LAUNCH();
}

size_t cu0_work_size(int Lx, int d, int Dmax) {
  const size_t D2 = size_t(Dmax) * Dmax;
  return 2 * size_t(d) * D2 * D2 + 2 * size_t(Lx) * D2 + D2;
}

void cu0_launch(Ctx& cx, const Cu0Lattice* lats, int nlat) {
  auto* dev = static_cast<const Cu0Lattice*>(stage(cx, lats, sizeof(Cu0Lattice) * nlat));
  Launch L(K_CU0, cx.st);
  k_cu0<<<nlat, 256, 0, cx.st>>>(dev, cx.flag);
  PEPS_CHECK_LAUNCH();
}

}  // namespace peps

// ============================================================================
// Allocation-free entry point: CU_0 boundaries with file-scope scratch.
//
// Some callers cannot call cudaMalloc: a serving process whose allocator has
// already reserved the device memory it may use, code in a latency-critical
// loop where cudaMalloc / cudaFree would synchronise the device, or a host
// framework that forbids device allocation after start-up.  peps_cu0_noalloc
// serves them: it reads the caller's dense lattice, writes the caller's
// output buffer, and keeps its scratch in the static array below.
// ============================================================================
namespace peps {
namespace {

// Scratch: 8 words of status, then the repacked site tensor, two
// intermediates (3 d D^4), the previous / current separable row and the left /
// right environments (4 Lx D^2) and the local vector (D^2).
constexpr int NOALLOC_MAX_D = 8;
constexpr int NOALLOC_MAX_d = 4;
constexpr int NOALLOC_MAX_LX = 64;
constexpr int NOALLOC_MAX_LY = 4096;
constexpr size_t NOALLOC_WORDS =
    8 + 3 * size_t(NOALLOC_MAX_d) * NOALLOC_MAX_D * NOALLOC_MAX_D * NOALLOC_MAX_D * NOALLOC_MAX_D +
    4 * size_t(NOALLOC_MAX_LX) * NOALLOC_MAX_D * NOALLOC_MAX_D + size_t(NOALLOC_MAX_D) * NOALLOC_MAX_D;

static __device__ __align__(256) double g_cu0_scratch[NOALLOC_WORDS];

struct DenseCu0 {
  const double* A;   // dense [Ly][Lx][d][D][D][D][D]
  double* out;       // [Ly][Lx][D][D], zero-padded
  double* scr;       // device address of g_cu0_scratch
  int Ly, Lx, d, D, max_half;
  double tol;
};

__device__ SiteDims dense_dims(const DenseCu0& a, int y, int x) {
  return SiteDims{y == 0 ? 1 : a.D, x == 0 ? 1 : a.D, y == a.Ly - 1 ? 1 : a.D, x == a.Lx - 1 ? 1 : a.D};
}

// Copy site (y,x) from the dense layout into `dst` with its effective dims.
__device__ SiteDims load_dense_site(const DenseCu0& a, int y, int x, double* dst) {
  const SiteDims sd = dense_dims(a, y, x);
  const int D = a.D, n = a.d * sd.du * sd.dl * sd.dn * sd.dr;
  const long long base = ((long long)y * a.Lx + x) * a.d * D * D * D * D;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    int t = e;
    const int r = t % sd.dr; t /= sd.dr;
    const int nn = t % sd.dn; t /= sd.dn;
    const int l = t % sd.dl; t /= sd.dl;
    const int u = t % sd.du;
    const int s = t / sd.du;
    dst[e] = a.A[base + ((((long long)s * D + u) * D + l) * D + nn) * D + r];
  }
  __syncthreads();
  return sd;
}

__global__ void __launch_bounds__(256) k_cu0_dense(const DenseCu0 a) {
  __shared__ double red[32];
  const int Ly = a.Ly, Lx = a.Lx, d = a.d, D = a.D, DM2 = D * D;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long big = (long long)d * DM2 * DM2;
  int* flag = reinterpret_cast<int*>(a.scr);
  double* As = a.scr + 8;
  double* Y = As + big;
  double* Z = Y + big;
  double* sigP = Z + big;
  double* sigN = sigP + (long long)Lx * DM2;
  double* Lm = sigN + (long long)Lx * DM2;
  double* Rm = Lm + (long long)Lx * DM2;
  double* b = Rm + (long long)Lx * DM2;
  auto P = [&](int x) { return sigP + (long long)x * DM2; };
  auto N = [&](int x) { return sigN + (long long)x * DM2; };
  auto emit = [&](int r, const double* src, int x, int n) {   // padded D x D output
    double* o = a.out + ((long long)r * Lx + x) * DM2;
    for (int e = tid; e < DM2; e += nt) {
      const int i = e / D, j = e % D;
      o[e] = (i < n && j < n) ? src[i * n + j] : 0.0;
    }
  };
  for (int x = 0; x < Lx; ++x) {
    if (tid == 0) P(x)[0] = 1.0;   // top closure of the OBC lattice: 1 x 1 identity
    __syncthreads();
    emit(0, P(x), x, 1);
  }
  __syncthreads();
  for (int r = 0; r + 1 < Ly; ++r) {
    for (int x = 0; x < Lx; ++x) {
      const int dn = dense_dims(a, r, x).dn;
      const double v = 1.0 / sqrt(double(dn));
      for (int e = tid; e < dn * dn; e += nt) N(x)[e] = (e / dn == e % dn) ? v : 0.0;
    }
    if (tid == 0) {
      Rm[(long long)(Lx - 1) * DM2] = 1.0;
      Lm[0] = 1.0;
    }
    __syncthreads();
    // the same cut routine as the library's CU_0, each site staged from the dense layout
    const bool conv = cu0_cut(
        Lx, d, DM2, [&](int x) { return Cu0Site{As, load_dense_site(a, r, x, As)}; }, P, N, Lm, Rm, Y, Z, b,
        a.max_half, a.tol, red);
    if (!conv && tid == 0) atomicOr(flag, FLAG_CU0_NOCONV);
    for (int x = 0; x < Lx; ++x) {
      const int dn = dense_dims(a, r, x).dn;
      emit(r + 1, N(x), x, dn);
      for (int e = tid; e < dn * dn; e += nt) P(x)[e] = N(x)[e];
    }
    __syncthreads();
  }
}

// Device address of the scratch array, looked up once per device.
double* noalloc_scratch(int dev) {
  static std::mutex mu;
  static std::vector<double*> addr;
  std::lock_guard<std::mutex> g(mu);
  if (int(addr.size()) <= dev) addr.resize(dev + 1, nullptr);
  if (!addr[dev]) {
    void* p = nullptr;
    PEPS_CUDA(cudaGetSymbolAddress(&p, g_cu0_scratch));
    addr[dev] = static_cast<double*>(p);
  }
  return addr[dev];
}

}  // namespace
}  // namespace peps

extern "C" int peps_cu0_noalloc(const double* A, int Ly, int Lx, int d, int D, double* sigma,
                                void* cuda_stream) {
  using namespace peps;
  try {
    PEPS_REQUIRE(A != nullptr && sigma != nullptr, "NULL argument");
    PEPS_REQUIRE(Ly >= 1 && Lx >= 1 && d >= 1 && D >= 1, "sizes must be >= 1");
    PEPS_REQUIRE(Ly <= NOALLOC_MAX_LY && Lx <= NOALLOC_MAX_LX && d <= NOALLOC_MAX_d && D <= NOALLOC_MAX_D,
                 "peps_cu0_noalloc: sizes beyond the static scratch (Ly <= 4096, Lx <= 64, d <= 4, D <= 8)");
    const size_t need = 8 + 3 * size_t(d) * D * D * D * D + 4 * size_t(Lx) * D * D + size_t(D) * D;
    PEPS_REQUIRE(need <= NOALLOC_WORDS, "peps_cu0_noalloc: scratch too small for these sizes");
    int dev = 0;
    PEPS_CUDA(cudaGetDevice(&dev));
    double* scr = noalloc_scratch(dev);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    PEPS_CUDA(cudaMemsetAsync(scr, 0, 8 * sizeof(double), st));   // status words start at zero
    DenseCu0 a{A, sigma, scr, Ly, Lx, d, D, 200, 1e-13};
    {
      Launch L(K_CU0, st);
      k_cu0_dense<<<1, 256, 0, st>>>(a);
      PEPS_CHECK_LAUNCH();
    }
    int flag = 0;
    PEPS_CUDA(cudaMemcpyAsync(&flag, scr, sizeof(int), cudaMemcpyDeviceToHost, st));
    PEPS_CUDA(cudaStreamSynchronize(st));
    if (flag & FLAG_CU0_NOCONV) throw Error(PEPS_ECONVERGE, "CU_0 separable boundary did not converge within 200 half-sweeps");
    return PEPS_OK;
  } catch (const Error& e) {
    return peps_set_error(e.code, e.what());
  } catch (const std::exception& e) {
    return peps_set_error(PEPS_ECUDA, e.what());
  }
}
