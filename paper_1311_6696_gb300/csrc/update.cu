// Tensor update of the full / cluster update (Section 2).
//
// After a Trotter gate acts on a bond, the two tensors of the bond are refit
// by alternating least squares, one tensor at a time, each solving
// N_l A_l = b_l.  The variational parameters are the reduced tensors (the
// part of each site tensor carrying its physical leg and the shared bond),
// which makes every linear system small: (k * Dn) unknowns per physical
// value, k <= d * D.  Everything here is FP64 and small; the contractions go
// through the FP64 gather-GEMM, the solves through one Cholesky kernel.
//
// Rules (the oracle states the same ones in its own code):
//   * N is symmetrised over (ket, bra) and replaced by its positive part,
//     N+ = (N + |N|) / 2 with |N| = V S V^T from its SVD;
//   * Theta[k1,s,t,k2] = sum G[s,t,s',t'] a_l[k1,s',r] a_r[k2,t',r];
//   * ALS start: truncated SVD of Theta as (k1 s) x (t k2), Dn triplets,
//     a_l = U S, a_r = V;
//   * each round solves for a_l, then for a_r; a system is shifted by
//     1e-12 * trace / size on its diagonal and solved by Cholesky;
//   * the result is split again by an SVD, a_l = U sqrt(S), a_r = sqrt(S) V^T,
//     with the largest entry of every U column made positive.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "aux.cuh"
#include "linalg.cuh"
#include "update.cuh"

namespace peps {

namespace {

__global__ void k_permute5(const double* __restrict__ src, int d0, int d1, int d2, int d3, int d4, int p0, int p1,
                           int p2, int p3, int p4, double* __restrict__ dst) {
  const int dims[5] = {d0, d1, d2, d3, d4};
  const int perm[5] = {p0, p1, p2, p3, p4};
  long long sstr[5];
  sstr[4] = 1;
  for (int k = 3; k >= 0; --k) sstr[k] = sstr[k + 1] * dims[k + 1];
  const long long n = sstr[0] * dims[0];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    long long t = e, so = 0;
    for (int k = 4; k >= 0; --k) {
      const int ext = dims[perm[k]];
      so += (t % ext) * sstr[perm[k]];
      t /= ext;
    }
    dst[e] = src[so];
  }
}

// A <- (A + A^T) / 2 for every problem (n x n, row-major).
__global__ void k_symmetrize(TP A, int n) {
  double* a = A.d(blockIdx.y);
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
    const int i = int(e / n), j = int(e % n);
    if (j <= i) {
      const double v = 0.5 * (a[(long long)i * n + j] + a[(long long)j * n + i]);
      a[(long long)i * n + j] = v;
      a[(long long)j * n + i] = v;
    }
  }
}

// SVt[i][:] = ||US[:, i]|| * Vt[i][:] (US m x k, Vt k x n, row-major).
__global__ void k_scale_by_sigma(TP US, TP Vt, TP SVt, int m, int k, int n) {
  const int b = blockIdx.y;
  const double* us = US.d(b);
  const double* vt = Vt.d(b);
  double* out = SVt.d(b);
  for (int i = blockIdx.x; i < k; i += gridDim.x) {
    __shared__ double red[256];
    double s = 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) s += us[(long long)r * k + i] * us[(long long)r * k + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    const double sig = sqrt(red[0]);
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) out[(long long)i * n + c] = sig * vt[(long long)i * n + c];
  }
}

// y <- a * x + b * y for every problem.
__global__ void k_axpby(TP X, TP Y, long long n, double a, double bcoef) {
  const double* x = X.d(blockIdx.y);
  double* y = Y.d(blockIdx.y);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] = a * x[e] + bcoef * y[e];
}

// One Cholesky solve per problem: (A + eps I) X = B, eps = 1e-12 * trace / n,
// A n x n (row-major), B n x nrhs (row-major).  Row i of the solution is
// unknown (i / n2, i % n2); X[i][c] goes to out[(i / n2) * s_hi + c * s_c +
// (i % n2) * s_lo].  A pivot that is not positive and finite sets
// FLAG_BAD_VALUE and leaves the output unwritten.
struct CholArgs {
  TP A, B, out;
  int n, nrhs, n2;
  long long s_hi, s_c, s_lo;
  int* flag;
};

__global__ void __launch_bounds__(256) k_chol_solve(const CholArgs g) {
  extern __shared__ double sm[];
  const int n = g.n, ld = n + 1;
  double* L = sm;                          // n x ld
  double* y = sm + (size_t)n * ld;         // n x nrhs
  __shared__ int bad;
  __shared__ double eps;
  const int b = blockIdx.x;
  const double* A = g.A.d(b);
  const double* B = g.B.d(b);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) L[(e / n) * ld + e % n] = A[e];
  for (int e = threadIdx.x; e < n * g.nrhs; e += blockDim.x) y[e] = B[e];
  if (threadIdx.x == 0) {
    bad = 0;
    double tr = 0.0;
    for (int i = 0; i < n; ++i) tr += A[(long long)i * n + i];
    eps = 1e-12 * tr / n;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) L[i * ld + i] += eps;
  __syncthreads();
  // right-looking Cholesky, lower triangle
  for (int j = 0; j < n; ++j) {
    const double p = L[j * ld + j];
    if (!(p > 0.0) || !isfinite(p)) {
      if (threadIdx.x == 0) bad = 1;
      __syncthreads();
      break;
    }
    const double ljj = sqrt(p);
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) L[i * ld + j] /= ljj;
    __syncthreads();
    if (threadIdx.x == 0) L[j * ld + j] = ljj;
    const int m = n - j - 1;
    for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
      const int i = j + 1 + int(e / m), k = j + 1 + int(e % m);
      if (k <= i) L[i * ld + k] -= L[i * ld + j] * L[k * ld + j];
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) atomicOr(g.flag, FLAG_BAD_VALUE);
    return;
  }
  // forward: L z = b; backward: L^T x = z (column-oriented, one column per step)
  for (int j = 0; j < n; ++j) {
    for (int c = threadIdx.x; c < g.nrhs; c += blockDim.x) y[j * g.nrhs + c] /= L[j * ld + j];
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)(n - j - 1) * g.nrhs; e += blockDim.x) {
      const int i = j + 1 + int(e / g.nrhs), c = int(e % g.nrhs);
      y[i * g.nrhs + c] -= L[i * ld + j] * y[j * g.nrhs + c];
    }
    __syncthreads();
  }
  for (int j = n - 1; j >= 0; --j) {
    for (int c = threadIdx.x; c < g.nrhs; c += blockDim.x) y[j * g.nrhs + c] /= L[j * ld + j];
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)j * g.nrhs; e += blockDim.x) {
      const int i = int(e / g.nrhs), c = int(e % g.nrhs);
      y[i * g.nrhs + c] -= L[j * ld + i] * y[j * g.nrhs + c];
    }
    __syncthreads();
  }
  double* out = g.out.d(b);
  for (int e = threadIdx.x; e < n * g.nrhs; e += blockDim.x) {
    const int i = e / g.nrhs, c = e % g.nrhs;
    out[(long long)(i / g.n2) * g.s_hi + (long long)c * g.s_c + (long long)(i % g.n2) * g.s_lo] = y[e];
  }
}

// Balanced split of a truncated SVD: US (m x k), Vt (k x n) ->
// al = U sqrt(S) (m x k), ar = sqrt(S) Vt (k x n), U's largest entry (first
// on ties) of every column positive.  One CTA per problem.
__global__ void k_balance(TP US, TP Vt, TP AL, TP AR, int m, int k, int n) {
  const int b = blockIdx.x;
  const double* us = US.d(b);
  const double* vt = Vt.d(b);
  double* al = AL.d(b);
  double* ar = AR.d(b);
  __shared__ double rs[256];
  __shared__ double rv[256];
  __shared__ int ri[256];
  for (int i = 0; i < k; ++i) {
    double s = 0.0, best = -1.0;
    int bi = 0x7fffffff;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
      const double v = us[(long long)r * k + i];
      s += v * v;
      if (fabs(v) > best) {
        best = fabs(v);
        bi = r;
      }
    }
    rs[threadIdx.x] = s;
    rv[threadIdx.x] = best;
    ri[threadIdx.x] = bi;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        rs[threadIdx.x] += rs[threadIdx.x + w];
        const double ov = rv[threadIdx.x + w];
        const int oi = ri[threadIdx.x + w];
        if (ov > rv[threadIdx.x] || (ov == rv[threadIdx.x] && oi < ri[threadIdx.x])) {
          rv[threadIdx.x] = ov;
          ri[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    const double sig = sqrt(rs[0]);
    const double sgn = (ri[0] < m && us[(long long)ri[0] * k + i] < 0.0) ? -1.0 : 1.0;
    const double fl = sig > 0.0 ? sgn / sqrt(sig) : 0.0;   // U sqrt(S) = US / sqrt(S)
    const double fr = sgn * sqrt(sig);
    for (int r = threadIdx.x; r < m; r += blockDim.x) al[(long long)r * k + i] = fl * us[(long long)r * k + i];
    for (int c = threadIdx.x; c < n; c += blockDim.x) ar[(long long)i * n + c] = fr * vt[(long long)i * n + c];
    __syncthreads();
  }
}

__global__ void k_store_sites(const SiteStore* sites, void* dst, int f32, int Lx, int d, int D) {
  const SiteStore s = sites[blockIdx.x];
  const long long per = (long long)d * D * D * D * D;
  const long long base = ((long long)s.y * Lx + s.x) * per;
  for (long long e = threadIdx.x; e < per; e += blockDim.x) {
    long long t = e;
    int o[4];
    for (int k = 3; k >= 0; --k) {
      o[k] = int(t % D);
      t /= D;
    }
    const int ph = int(t);
    int idx[4];
    bool in = true;
    for (int k = 0; k < 4; ++k) {
      idx[k] = o[s.perm[k]];
      in = in && idx[k] < s.dims[k + 1];
    }
    double v = 0.0;
    if (in)
      v = s.src[((((long long)ph * s.dims[1] + idx[0]) * s.dims[2] + idx[1]) * s.dims[3] + idx[2]) * s.dims[4] +
                idx[3]];
    if (f32)
      static_cast<float*>(dst)[base + e] = float(v);
    else
      static_cast<double*>(dst)[base + e] = v;
  }
}

unsigned blocks_for(long long n, int threads) {
  return unsigned(std::max<long long>(1, std::min<long long>(1184, (n + threads - 1) / threads)));
}

TP per_problem(double* base, int np, size_t per) { return strided(base, np, per); }

}  // namespace

void permute5(Ctx& cx, const double* src, const int dims[5], const int perm[5], double* dst) {
  long long n = 1;
  for (int k = 0; k < 5; ++k) n *= dims[k];
  Launch L(K_AUX, cx.st, 0, 16.0 * double(n));
  k_permute5<<<blocks_for(n, 256), 256, 0, cx.st>>>(src, dims[0], dims[1], dims[2], dims[3], dims[4], perm[0],
                                                    perm[1], perm[2], perm[3], perm[4], dst);
  PEPS_CHECK_LAUNCH();
}

void bond_als(Ctx& cx, int d, int kl, int kr, int Do, int Dn, const double* gate, const std::vector<BondAls>& bonds,
              int iters) {
  PEPS_REQUIRE(kl * Dn <= kCholMax && kr * Dn <= kCholMax, "internal: bond update system too large");
  const int n2 = kl * kr;
  const size_t sN = size_t(n2) * n2, sTh = size_t(kl) * d * d * kr;
  const size_t sP = size_t(std::max(kl, kr)) * kl * kr * d * Dn;
  const size_t sNt = size_t(std::max(kl, kr)) * Dn * std::max(kl, kr) * Dn;
  const size_t sb = size_t(std::max(kl, kr)) * Dn * d;
  const size_t sT1 = size_t(kl) * d * d * d * Do;
  const size_t sU = size_t(kl) * d * Dn, sV = size_t(Dn) * d * kr;
  const Dims nd = {kl, kr, kl, kr}, thd = {kl, d, d, kr}, gd = {d, d, d, d};
  const Dims ald = {kl, d, Do}, ard = {kr, d, Do};
  const Dims ad = {kl, d, Dn}, bd = {Dn, d, kr};
  const TP G(gate);
  for (size_t c0 = 0; c0 < bonds.size(); c0 += MAXB) {
    const int np = int(std::min<size_t>(MAXB, bonds.size() - c0));
    TP N, al0, ar0, aln, arn, q;
    N.n = al0.n = ar0.n = aln.n = arn.n = q.n = np;
    for (int b = 0; b < np; ++b) {
      const BondAls& x = bonds[c0 + b];
      N.p[b] = const_cast<double*>(x.N);
      al0.p[b] = const_cast<double*>(x.al);
      ar0.p[b] = const_cast<double*>(x.ar);
      aln.p[b] = x.al_new;
      arn.p[b] = x.ar_new;
      q.p[b] = x.q;
    }
    auto blk = [&](size_t per) { return per_problem(cx.ws->dalloc(((per + 31) / 32 * 32) * np), np, per); };
    const TP Np = blk(sN), US = blk(sN), Vt = blk(sN), SV = blk(sN), Th = blk(sTh), T1 = blk(sT1), P = blk(sP),
             P2 = blk(size_t(kl) * kr * d * d), Nt = blk(sNt), rhs = blk(sb), al = blk(sU), ar = blk(sV),
             psi = blk(sTh), pu = blk(sU), pv = blk(sV);
    // positive part of the symmetrised N
    copy(cx, Np, N, (long long)sN);
    {
      Launch L(K_AUX, cx.st);
      k_symmetrize<<<dim3(blocks_for((long long)sN, 256), np), 256, 0, cx.st>>>(Np, n2);
      PEPS_CHECK_LAUNCH();
    }
    svd_trunc(cx, n2, n2, Np, n2, US, Vt);
    {
      Launch L(K_AUX, cx.st);
      k_scale_by_sigma<<<dim3(unsigned(std::min(n2, 1024)), np), 256, 0, cx.st>>>(US, Vt, SV, n2, n2, n2);
      PEPS_CHECK_LAUNCH();
    }
    ein(cx, "ia,ib->ab", Vt, {n2, n2}, SV, {n2, n2}, US);   // |N| into US (no longer needed)
    {
      Launch L(K_AUX, cx.st);
      k_axpby<<<dim3(blocks_for((long long)sN, 256), np), 256, 0, cx.st>>>(US, Np, (long long)sN, 0.5, 0.5);
      PEPS_CHECK_LAUNCH();
    }
    // Theta, then the ALS start
    ein(cx, "stuv,aur->astvr", G, gd, al0, ald, T1);
    ein(cx, "astvr,bvr->astb", T1, {kl, d, d, d, Do}, ar0, ard, Th);
    svd_trunc(cx, kl * d, d * kr, Th, Dn, al, ar);
    // sum_ij N[i,j,k,l] Theta[i,s,t,j]: fixed over the rounds
    ein(cx, "ijkl,istj->klst", Np, nd, Th, thd, P2);
    auto solve = [&](int k, int nrhs_hi, const TP& out, long long s_hi, long long s_c, long long s_lo) {
      CholArgs g;
      g.A = Nt.all(np);
      g.B = rhs.all(np);
      g.out = out.all(np);
      g.n = k * Dn;
      g.nrhs = d;
      g.n2 = Dn;
      g.s_hi = s_hi;
      g.s_c = s_c;
      g.s_lo = s_lo;
      g.flag = cx.flag;
      (void)nrhs_hi;
      const size_t smem = sizeof(double) * (size_t(g.n) * (g.n + 1) + size_t(g.n) * d);
      static bool attr = false;
      if (!attr) {
        PEPS_CUDA(cudaFuncSetAttribute(k_chol_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
        attr = true;
      }
      PEPS_REQUIRE(smem <= 220 * 1024, "internal: Cholesky system exceeds shared memory");
      const double n3 = double(g.n) * g.n * g.n;
      Launch L(K_QR, cx.st, n3 / 3.0 + 2.0 * double(g.n) * g.n * d, 0);
      k_chol_solve<<<unsigned(np), 256, smem, cx.st>>>(g);
      PEPS_CHECK_LAUNCH();
    };
    for (int it = 0; it < iters; ++it) {
      // left: Nt[(k q),(i r)] = sum N[i,j,k,l] ar[r,t,j] ar[q,t,l]; b[(k q), s]
      ein(cx, "ijkl,qtl->ijktq", Np, nd, ar, bd, P);
      ein(cx, "ijktq,rtj->kqir", P, {kl, kr, kl, d, Dn}, ar, bd, Nt);
      ein(cx, "klst,qtl->kqs", P2, {kl, kr, d, d}, ar, bd, rhs);
      solve(kl, 0, al, (long long)d * Dn, Dn, 1);      // al[i][s][r]
      // right: Nt[(l q),(j r)] = sum N[i,j,k,l] al[i,s,r] al[k,s,q]; b[(l q), t]
      ein(cx, "ijkl,ksq->ijlsq", Np, nd, al, ad, P);
      ein(cx, "ijlsq,isr->lqjr", P, {kl, kr, kr, d, Dn}, al, ad, Nt);
      ein(cx, "klst,ksq->lqt", P2, {kl, kr, d, d}, al, ad, rhs);
      solve(kr, 0, ar, 1, kr, (long long)d * kr);      // ar[r][t][j]
    }
    // the pair, its cost, and its balanced split
    ein(cx, "asr,rtb->astb", al, ad, ar, bd, psi);
    svd_trunc(cx, kl * d, d * kr, psi, Dn, pu, pv);
    {
      Launch L(K_AUX, cx.st);
      k_balance<<<unsigned(np), 256, 0, cx.st>>>(pu, pv, aln, arn, kl * d, Dn, d * kr);
      PEPS_CHECK_LAUNCH();
    }
    ein(cx, "klst,kstl->", P2, {kl, kr, d, d}, Th, thd, q.off(1));
    {
      Launch L(K_AUX, cx.st);
      k_axpby<<<dim3(blocks_for((long long)sTh, 256), np), 256, 0, cx.st>>>(Th, psi, (long long)sTh, -1.0, 1.0);
      PEPS_CHECK_LAUNCH();
    }
    ein(cx, "ijkl,istj->klst", Np, nd, psi, thd, P2);
    ein(cx, "klst,kstl->", P2, {kl, kr, d, d}, psi, thd, q);
  }
}

void store_sites(Ctx& cx, void* dst, int dst_f32, int Lx, int d, int D, const std::vector<SiteStore>& sites) {
  if (sites.empty()) return;
  auto* dev = static_cast<const SiteStore*>(stage(cx, sites.data(), sizeof(SiteStore) * sites.size()));
  Launch L(K_AUX, cx.st);
  k_store_sites<<<unsigned(sites.size()), 256, 0, cx.st>>>(dev, dst, dst_f32, Lx, d, D);
  PEPS_CHECK_LAUNCH();
}

}  // namespace peps
