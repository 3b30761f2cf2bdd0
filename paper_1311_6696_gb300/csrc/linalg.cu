// FP64 Householder QR and one-sided Jacobi SVD, batched over independent
// problems of one shape.
//
// Small matrices take one CTA each (working copy in global memory, L2
// resident; one warp per column reduction).  Larger ones are split by rows
// over a thread-block cluster of 2-16 CTAs that exchange partial sums through
// distributed shared memory: the QR with one cluster barrier per Householder
// column, the SVD with one per round of the round-robin Jacobi schedule.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <mutex>
#include <tuple>
#include <vector>

#include "linalg.cuh"

namespace cg = cooperative_groups;

namespace peps {
namespace {

constexpr int QR_THREADS = 512;
constexpr int SVD_THREADS = 512;

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

struct QrArgs {
  int m, n;
  TP A;         // per problem
  long long rs, cs;
  TP Q;
  long long qrs, qcs;
  TP R;         // absent: R not wanted
  double* W;    // m*n work per problem, column-major (problem p at W + p * wst)
  double* Qw;   // m*k work per problem, column-major (+ p * qst)
  double* tau;  // k per problem (+ p * tst)
  long long wst, qst, tst;
};

// Grid = problems, one CTA each.
__global__ void __launch_bounds__(QR_THREADS) k_qr_house(const QrArgs q) {
  __shared__ double red[32];
  __shared__ double s_tau, s_scale;
  const int m = q.m, n = q.n, k = min(m, n);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int pb = blockIdx.x;
  const double* A = q.A.d(pb);
  double* const Qo = q.Q.d(pb);
  double* const Ro = q.R.n ? q.R.d(pb) : nullptr;
  double* const tau_g = q.tau + pb * q.tst;
  double* W = q.W + pb * q.wst;
  for (long long e = tid; e < (long long)m * n; e += nt) {
    int i = int(e % m), j = int(e / m);
    W[e] = A[i * q.rs + j * q.cs];
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    double part = 0.0;
    for (int i = j + 1 + tid; i < m; i += nt) {
      double v = W[(long long)j * m + i];
      part += v * v;
    }
    const double sig = block_sum(part, red);
    if (tid == 0) {
      const double alpha = W[(long long)j * m + j];
      if (sig == 0.0) {
        s_tau = 0.0;
        s_scale = 0.0;
      } else {
        const double nrm = sqrt(alpha * alpha + sig);
        const double beta = alpha >= 0.0 ? -nrm : nrm;
        s_tau = (beta - alpha) / beta;
        s_scale = 1.0 / (alpha - beta);
        W[(long long)j * m + j] = beta;
      }
      tau_g[j] = s_tau;
    }
    __syncthreads();
    const double tau = s_tau, scale = s_scale;
    if (tau != 0.0) {
      for (int i = j + 1 + tid; i < m; i += nt) W[(long long)j * m + i] *= scale;
      __syncthreads();
      for (int c = j + 1 + warp; c < n; c += nw) {
        double w = 0.0;
        for (int i = j + 1 + lane; i < m; i += 32) w += W[(long long)j * m + i] * W[(long long)c * m + i];
        w = warp_sum(w) + W[(long long)c * m + j];
        w *= tau;
        if (lane == 0) W[(long long)c * m + j] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) W[(long long)c * m + i] -= w * W[(long long)j * m + i];
      }
    }
    __syncthreads();
  }
  // Q = H_0 ... H_{k-1} [I_k; 0], accumulated backwards.
  double* Qw = q.Qw + pb * q.qst;
  for (long long e = tid; e < (long long)m * k; e += nt) {
    int i = int(e % m), j = int(e / m);
    Qw[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const double tau = tau_g[j];
    if (tau != 0.0) {
      for (int c = j + warp; c < k; c += nw) {
        double w = 0.0;
        for (int i = j + 1 + lane; i < m; i += 32) w += W[(long long)j * m + i] * Qw[(long long)c * m + i];
        w = warp_sum(w) + Qw[(long long)c * m + j];
        w *= tau;
        if (lane == 0) Qw[(long long)c * m + j] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) Qw[(long long)c * m + i] -= w * W[(long long)j * m + i];
      }
    }
    __syncthreads();
  }
  for (long long e = tid; e < (long long)m * k; e += nt) {
    int i = int(e % m), j = int(e / m);
    Qo[i * q.qrs + j * q.qcs] = Qw[e];
  }
  if (Ro) {
    for (long long e = tid; e < (long long)k * n; e += nt) {
      int i = int(e / n), j = int(e % n);
      Ro[e] = (j >= i) ? W[(long long)j * m + i] : 0.0;
    }
  }
}

// ---------------------------------------------------------------------------
// Householder QR on a thread-block cluster: the rows of one matrix are split
// over the cluster's CTAs (one SM each); every column reduction (the norm
// below the diagonal, the reflector's inner products with the trailing
// columns) is a per-CTA partial sum exchanged through distributed shared
// memory between hardware cluster barriers.  Same reflectors, same order and
// same sign convention as the one-CTA kernel; the FP64 work is spread over C
// SMs instead of one.
// ---------------------------------------------------------------------------
constexpr int QRC_THREADS = 512;
// Each CTA keeps its block of rows of the working matrix and of Q in shared
// memory when they fit (column-major within the block, odd column stride),
// else in global scratch.  Work per column is split as (column, row quarter)
// per thread: every thread runs a plain FMA loop over its rows, so the FP64
// pipe executes the factorisation's own multiply-adds and almost nothing else
// (a shuffle tree per column would cost more FP64 issue slots than the dot
// products at 64 rows per CTA).
constexpr int QS = 8;   // threads per column (rows interleaved mod QS)

// Strided dot product and update over rows start, start + QS, ... < end with
// four rows' loads in flight per step (when the rows live in global memory a
// thread's loop is otherwise one dependent load after another); fixed
// summation order.
__device__ __forceinline__ double dot_qs(const double* __restrict__ x, const double* __restrict__ y, int start,
                                         int end) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int i = start;
  for (; i + 3 * QS < end; i += 4 * QS) {
    const double x0 = x[i], x1 = x[i + QS], x2 = x[i + 2 * QS], x3 = x[i + 3 * QS];
    const double y0 = y[i], y1 = y[i + QS], y2 = y[i + 2 * QS], y3 = y[i + 3 * QS];
    a0 = fma(x0, y0, a0);
    a1 = fma(x1, y1, a1);
    a2 = fma(x2, y2, a2);
    a3 = fma(x3, y3, a3);
  }
  for (; i < end; i += QS) a0 = fma(x[i], y[i], a0);
  return (a0 + a1) + (a2 + a3);
}

// y[i] -= w x[i] over the same rows (x and y are different columns).
__device__ __forceinline__ void axpy_qs(double w, const double* __restrict__ x, double* __restrict__ y, int start,
                                        int end) {
  int i = start;
  for (; i + 3 * QS < end; i += 4 * QS) {
    const double x0 = x[i], x1 = x[i + QS], x2 = x[i + 2 * QS], x3 = x[i + 3 * QS];
    const double y0 = y[i], y1 = y[i + QS], y2 = y[i + 2 * QS], y3 = y[i + 3 * QS];
    y[i] = fma(-w, x0, y0);
    y[i + QS] = fma(-w, x1, y1);
    y[i + 2 * QS] = fma(-w, x2, y2);
    y[i + 3 * QS] = fma(-w, x3, y3);
  }
  for (; i < end; i += QS) y[i] = fma(-w, x[i], y[i]);
}

// Sum of one double over the cluster's CTAs, all remote loads issued first.
__device__ __forceinline__ double remote_sum(cg::cluster_group& cl, double* slot, int C) {
  double v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = r < C ? *cl.map_shared_rank(slot, r) : 0.0;
  double s = 0.0;
#pragma unroll
  for (int r = 0; r < 16; ++r) s += v[r];
  return s;
}

__global__ void __launch_bounds__(QRC_THREADS) k_qr_cluster(const QrArgs q, int in_smem, int ld) {
  extern __shared__ double qsm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = int(cluster.num_blocks());
  const int rank = int(cluster.block_rank());
  const int pb = blockIdx.x / C;               // one cluster per problem
  const double* A = q.A.d(pb);
  double* const Qo = q.Q.d(pb);
  double* const Ro = q.R.n ? q.R.d(pb) : nullptr;
  const int m = q.m, n = q.n, k = min(m, n);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int chunk = (m + C - 1) / C;
  const int r0 = min(m, rank * chunk), r1 = min(m, r0 + chunk), rows = r1 - r0;
  // Cluster-visible, double-buffered by column parity:
  double* wpart = qsm;              // [2][n] my partial raw inner products of column j with columns c > j
  double* rowj = wpart + 2 * n;     // [2][n] row j of the trailing matrix (valid in the row's owner)
  double* npart = rowj + 2 * n;     // [2]    my partial squared norm of column j below the diagonal
  double* tau_s = npart + 2;        // [k]
  double* part4 = tau_s + k;        // [n][QS] quarter sums
  double* wfin = part4 + (long long)n * QS;   // [n]
  double* coef = wfin + n;          // [2] scale, beta of the current reflector
  double* W;                        // [n][ld] my rows, column-major (row i at i - r0); Q is formed in place
  if (in_smem) {
    W = coef + 2 + QS;
  } else {
    W = q.W + pb * q.wst + (long long)rank * ld * n;
  }
  for (long long e = tid; e < (long long)rows * n; e += nt) {
    const int li = int(e % rows), j = int(e / rows);
    W[(long long)j * ld + li] = A[(r0 + li) * q.rs + j * q.cs];
  }
  __syncthreads();
  // My partial sums for column j into buffer b: sum over my rows i > j of
  // a_ji * a_ci for every c >= j (c = j: the squared norm), and, in the owner
  // of row j, that row.  The reflector's inner products with the trailing
  // columns are taken with the unscaled column, w_c = tau (a_cj + scale *
  // sum_i a_ji a_ci), so one cluster barrier per column carries both the norm
  // (for tau) and the inner products.
  auto partials = [&](int j, int b) {
    const int i0 = max(r0, j + 1);
    const double* xj = W + (long long)j * ld - r0;
    for (int t = tid; t < (n - j) * QS; t += nt) {
      const int c = j + t / QS, qq = t % QS;
      const double* wc = W + (long long)c * ld - r0;
      part4[(long long)c * QS + qq] = dot_qs(xj, wc, i0 + ((qq - i0 % QS + QS) % QS), r1);
    }
    __syncthreads();
    const bool has_row = j >= r0 && j < r1;
    for (int c = j + tid; c < n; c += nt) {
      double w = 0.0;
      for (int qq = 0; qq < QS; ++qq) w += part4[(long long)c * QS + qq];
      if (c == j)
        npart[b] = w;
      else
        wpart[b * n + c] = w;
      if (has_row) rowj[b * n + c] = W[(long long)c * ld + (j - r0)];
    }
  };
  partials(0, 0);
  for (int j = 0; j < k; ++j) {
    const int b = j & 1;
    const int owner = j / chunk;
    const bool own = (owner == rank);
    cluster.sync();                                   // column j: norms, inner products, row j visible
    if (tid < 32) {
      const double alpha = *cluster.map_shared_rank(rowj + b * n + j, owner);
      double sig = 0.0;
      for (int r = tid; r < C; r += 32) sig += *cluster.map_shared_rank(npart + b, r);
      sig = warp_sum(sig);
      double tau = 0.0, scale = 0.0, beta = alpha;
      if (sig != 0.0) {
        const double nrm = sqrt(alpha * alpha + sig);
        beta = alpha >= 0.0 ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
      if (tid == 0) {
        tau_s[j] = tau;
        coef[0] = scale;
        coef[1] = beta;
      }
    }
    __syncthreads();
    const double tau = tau_s[j], scale = coef[0], beta = coef[1];
    const int i0 = max(r0, j + 1);                    // my rows below the diagonal
    double* vj = W + (long long)j * ld - r0;          // vj[i] for global row i
    const int nc = n - j - 1;                         // trailing columns
    if (tau != 0.0) {                                 // uniform across the cluster
      for (int c = j + 1 + tid; c < n; c += nt)
        wfin[c] = tau * fma(scale, remote_sum(cluster, wpart + b * n + c, C),
                            *cluster.map_shared_rank(rowj + b * n + c, owner));
      for (int i = i0 + tid; i < r1; i += nt) vj[i] *= scale;   // local rows only: no hazard with the loads above
      __syncthreads();
      for (int t = tid; t < nc * QS; t += nt) {
        const int c = j + 1 + t / QS, qq = t % QS;
        double* wc = W + (long long)c * ld - r0;
        const double w = wfin[c];
        if (own && qq == 0) wc[j] -= w;
        axpy_qs(w, vj, wc, i0 + ((qq - i0 % QS + QS) % QS), r1);
      }
      if (own && tid == 0) vj[j] = beta;
    }
    __syncthreads();
    if (j + 1 < k) partials(j + 1, 1 - b);
  }
  // R first: Q is formed over W below.
  if (Ro) {
    for (long long e = tid; e < (long long)rows * n; e += nt) {
      const int li = int(e % rows), j = int(e / rows), i = r0 + li;
      if (i < k) Ro[(long long)i * n + j] = (j >= i) ? W[(long long)j * ld + li] : 0.0;
    }
  }
  __syncthreads();
  // Q = H_0 ... H_{k-1} [I_k; 0], formed backwards in place on the same row
  // split: column j keeps its reflector below the diagonal until step j,
  // columns c > j already hold Q's columns and are zero in rows <= j.  Rows
  // above the diagonal (R) are cleared first.
  for (long long e = tid; e < (long long)rows * k; e += nt) {
    const int li = int(e % rows), c = int(e / rows);
    if (r0 + li < c) W[(long long)c * ld + li] = 0.0;
  }
  cluster.sync();
  int nsync = 0;   // double-buffer index: advances only with a cluster barrier
  for (int j = k - 1; j >= 0; --j) {
    const double tau = tau_s[j];
    const bool own = (j >= r0 && j < r1);
    const int i0 = max(r0, j + 1);
    double* vj = W + (long long)j * ld - r0;          // vj[i] for global row i
    const int nc = k - j - 1;                         // columns j+1 .. k-1
    if (tau != 0.0 && nc > 0) {                       // uniform across the cluster
      const int b = nsync & 1;
      ++nsync;
      for (int t = tid; t < nc * QS; t += nt) {
        const int c = j + 1 + t / QS, qq = t % QS;
        const double* qc = W + (long long)c * ld - r0;
        part4[(long long)c * QS + qq] = dot_qs(vj, qc, i0 + ((qq - i0 % QS + QS) % QS), r1);
      }
      __syncthreads();
      for (int c = j + 1 + tid; c < k; c += nt) {
        double w = 0.0;
        for (int qq = 0; qq < QS; ++qq) w += part4[(long long)c * QS + qq];
        wpart[b * n + c] = w;
      }
      cluster.sync();
      for (int c = j + 1 + tid; c < k; c += nt) wfin[c] = tau * remote_sum(cluster, wpart + b * n + c, C);
      __syncthreads();
      for (int t = tid; t < nc * QS; t += nt) {
        const int c = j + 1 + t / QS, qq = t % QS;
        double* qc = W + (long long)c * ld - r0;
        const double w = wfin[c];
        if (own && qq == 0) qc[j] = -w;
        axpy_qs(w, vj, qc, i0 + ((qq - i0 % QS + QS) % QS), r1);
      }
    }
    __syncthreads();                                  // every read of the reflector is done
    for (int i = i0 + tid; i < r1; i += nt) vj[i] *= -tau;
    if (own && tid == 0) vj[j] = 1.0 - tau;
    __syncthreads();
  }
  for (long long e = tid; e < (long long)rows * k; e += nt) {
    const int li = int(e % rows), c = int(e / rows);
    Qo[(r0 + li) * q.qrs + c * q.qcs] = W[(long long)c * ld + li];
  }
  cluster.sync();   // no CTA leaves while others may still read its shared memory
}

struct SvdArgs {
  int p, q;          // working matrix G is p x q (p >= q), column-major
  int m, n;          // original A is m x n row-major
  int trans;         // 1: G = A^T (m < n)
  TP A;              // per problem
  double* work;      // per problem (+ problem * wst): G (p x q), V (q x q), nrm (q), order (q ints)
  long long wst;
  int kk;
  TP US;             // m x kk row-major
  TP Vt;             // kk x n row-major
  int* flag;
  int max_sweeps;    // sweep cap (PEPS_ECONVERGE when reached)
};

// Grid = problems, one CTA each.
__global__ void __launch_bounds__(SVD_THREADS) k_svd_jacobi(const SvdArgs s) {
  __shared__ int s_rot;
  const int p = s.p, q = s.q;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int pb = blockIdx.x;
  const double* A = s.A.d(pb);
  double* const US = s.US.d(pb);
  double* const Vto = s.Vt.d(pb);
  double* G = s.work + pb * s.wst;
  double* V = G + (long long)p * q;
  double* const nrm = V + (long long)q * q;
  int* const order = reinterpret_cast<int*>(nrm + q);
  for (long long e = tid; e < (long long)p * q; e += nt) {
    int i = int(e % p), j = int(e / p);   // G(i,j)
    G[e] = s.trans ? A[(long long)j * s.n + i] : A[(long long)i * s.n + j];
  }
  for (long long e = tid; e < (long long)q * q; e += nt) V[e] = ((e % q) == (e / q)) ? 1.0 : 0.0;
  __syncthreads();
  const int qq = q + (q & 1);   // even number of slots for the round-robin pairing
  // a pair is orthogonal once |gamma| <= tol sqrt(alpha beta); rounding alone
  // leaves |gamma| / sqrt(alpha beta) of order p * eps after a rotation, so the
  // threshold scales with the row count (as in LAPACK's one-sided Jacobi)
  const double tol = fmax(1e-15, 4.0 * double(p) * 2.220446049250313e-16);
  int sweep = 0;
  for (; sweep < s.max_sweeps; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < qq - 1; ++round) {
      for (int pr = warp; pr < qq / 2; pr += nw) {
        // round-robin (circle) schedule: slot 0 fixed, others rotate
        int a = (pr == 0) ? 0 : 1 + (pr - 1 + round) % (qq - 1);
        int b = 1 + (qq - 2 - pr + round) % (qq - 1);
        if (a >= q || b >= q) continue;
        if (a > b) { int t = a; a = b; b = t; }
        double al = 0.0, be = 0.0, ga = 0.0;
        const double* ga_ = G + (long long)a * p;
        const double* gb_ = G + (long long)b * p;
        for (int i = lane; i < p; i += 32) {
          double x = ga_[i], y = gb_[i];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != 0.0 && fabs(ga) > tol * sqrt(al * be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
          double* gA = G + (long long)a * p;
          double* gB = G + (long long)b * p;
          for (int i = lane; i < p; i += 32) {
            double x = gA[i], y = gB[i];
            gA[i] = c * x - sn * y;
            gB[i] = sn * x + c * y;
          }
          double* vA = V + (long long)a * q;
          double* vB = V + (long long)b * q;
          for (int i = lane; i < q; i += 32) {
            double x = vA[i], y = vB[i];
            vA[i] = c * x - sn * y;
            vB[i] = sn * x + c * y;
          }
          if (lane == 0) s_rot = 1;
        }
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (!rot) break;
  }
  if (sweep >= s.max_sweeps && tid == 0) atomicOr(s.flag, FLAG_SVD_NOCONV);
  // column norms and a stable descending order
  for (int j = warp; j < q; j += nw) {
    double v = 0.0;
    for (int i = lane; i < p; i += 32) {
      double x = G[(long long)j * p + i];
      v += x * x;
    }
    v = warp_sum(v);
    if (lane == 0) nrm[j] = sqrt(v);
  }
  __syncthreads();
  for (int j = tid; j < q; j += nt) {
    const double vj = nrm[j];
    int r = 0;
    for (int i = 0; i < q; ++i) {
      const double vi = nrm[i];
      r += (vi > vj) || (vi == vj && i < j);
    }
    order[r] = j;
  }
  __syncthreads();
  // A V = G  (A = G V^T when trans = 0;  A^T = G V^T  =>  A = V G^T when trans = 1)
  const int kk = s.kk;
  if (!s.trans) {
    // US[i][r] = G(i, order[r]);  Vt[r][j] = V(j, order[r])
    for (long long e = tid; e < (long long)s.m * kk; e += nt) {
      int i = int(e / kk), r = int(e % kk);
      US[e] = (r < q) ? G[(long long)order[r] * p + i] : 0.0;
    }
    for (long long e = tid; e < (long long)kk * s.n; e += nt) {
      int r = int(e / s.n), j = int(e % s.n);
      Vto[e] = (r < q) ? V[(long long)order[r] * q + j] : 0.0;
    }
  } else {
    // US[i][r] = V(i, order[r]) * nrm;  Vt[r][j] = G(j, order[r]) / nrm
    for (long long e = tid; e < (long long)s.m * kk; e += nt) {
      int i = int(e / kk), r = int(e % kk);
      US[e] = (r < q) ? V[(long long)order[r] * q + i] * nrm[order[r]] : 0.0;
    }
    for (long long e = tid; e < (long long)kk * s.n; e += nt) {
      int r = int(e / s.n), j = int(e % s.n);
      double nr = (r < q) ? nrm[order[r]] : 0.0;
      Vto[e] = (r < q && nr > 0.0) ? G[(long long)order[r] * p + j] / nr : 0.0;
    }
  }
}

// ---------------------------------------------------------------------------
// One-sided Jacobi on a thread-block cluster: the rows of the working matrix G
// (p x q) and of V (q x q) are split over the cluster's CTAs.  A round of the
// round-robin schedule is one cluster barrier: every CTA publishes its partial
// (alpha, beta, gamma) of every pair, then sums all CTAs' partials in the same
// order -- so every CTA forms the same rotations -- and rotates its own rows.
// Same rotations, threshold, ordering and output as the one-CTA kernel.
// ---------------------------------------------------------------------------
constexpr int SVC_THREADS = 256;

__global__ void __launch_bounds__(SVC_THREADS) k_svd_cluster(const SvdArgs s, double* work, long long wst) {
  extern __shared__ double ssm[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = int(cluster.num_blocks()), rank = int(cluster.block_rank());
  const int pb = blockIdx.x / C;
  const int p = s.p, q = s.q, tid = threadIdx.x, nt = blockDim.x;
  const int qq = q + (q & 1), npair = qq / 2;
  const int cp = (p + C - 1) / C, cv = (q + C - 1) / C;
  const int g0 = min(p, rank * cp), g1 = min(p, g0 + cp), gr = g1 - g0;   // my rows of G
  const int v0 = min(q, rank * cv), v1 = min(q, v0 + cv), vr = v1 - v0;   // my rows of V
  double* part = ssm;                         // [2][3][npair] my partial sums (cluster-visible)
  double* cs = part + 6 * npair;              // [2][2][npair] rotation (c, s) of this round
  double* nrm = cs + 4 * npair;               // [q]
  int* order = reinterpret_cast<int*>(nrm + q);   // [q]
  __shared__ int s_rot;
  double* G = work + pb * wst + (long long)rank * cp * q;                   // [q][cp] column-major block
  double* V = work + pb * wst + (long long)C * cp * q + (long long)rank * cv * q;   // [q][cv]
  const double* A = s.A.d(pb);
  for (long long e = tid; e < (long long)gr * q; e += nt) {
    const int li = int(e % gr), j = int(e / gr), i = g0 + li;
    G[(long long)j * cp + li] = s.trans ? A[(long long)j * s.n + i] : A[(long long)i * s.n + j];
  }
  for (long long e = tid; e < (long long)vr * q; e += nt) {
    const int li = int(e % vr), j = int(e / vr);
    V[(long long)j * cv + li] = (v0 + li == j) ? 1.0 : 0.0;
  }
  // a pair is orthogonal once |gamma| <= tol sqrt(alpha beta); rounding alone
  // leaves |gamma| / sqrt(alpha beta) of order p * eps after a rotation, so the
  // threshold scales with the row count (as in LAPACK's one-sided Jacobi)
  const double tol = fmax(1e-15, 4.0 * double(p) * 2.220446049250313e-16);
  int sweep = 0, t = 0;
  for (; sweep < s.max_sweeps; ++sweep) {
    int rotated = 0;
    for (int round = 0; round < qq - 1; ++round, ++t) {
      const int b = t & 1;
      __syncthreads();
      for (int pr = tid; pr < npair; pr += nt) {
        int a = (pr == 0) ? 0 : 1 + (pr - 1 + round) % (qq - 1);
        int c = 1 + (qq - 2 - pr + round) % (qq - 1);
        if (a > c) {
          const int tmp = a;
          a = c;
          c = tmp;
        }
        double al = 0.0, be = 0.0, ga = 0.0;
        if (a < q && c < q) {
          const double* xa = G + (long long)a * cp;
          const double* xc = G + (long long)c * cp;
          for (int i = 0; i < gr; ++i) {
            const double x = xa[i], y = xc[i];
            al = fma(x, x, al);
            be = fma(y, y, be);
            ga = fma(x, y, ga);
          }
        }
        part[(b * 3 + 0) * npair + pr] = al;
        part[(b * 3 + 1) * npair + pr] = be;
        part[(b * 3 + 2) * npair + pr] = ga;
      }
      cluster.sync();
      for (int pr = tid; pr < npair; pr += nt) {
        int a = (pr == 0) ? 0 : 1 + (pr - 1 + round) % (qq - 1);
        int c = 1 + (qq - 2 - pr + round) % (qq - 1);
        double cc = 1.0, sn = 0.0;
        if (a < q && c < q) {
          if (a > c) {
            const int tmp = a;
            a = c;
            c = tmp;
          }
          // all 3C remote loads in flight before any add (one round trip), summed in rank order
          double va[16], vb[16], vg[16];
#pragma unroll
          for (int r = 0; r < 16; ++r) {
            va[r] = r < C ? *cluster.map_shared_rank(part + (b * 3 + 0) * npair + pr, r) : 0.0;
            vb[r] = r < C ? *cluster.map_shared_rank(part + (b * 3 + 1) * npair + pr, r) : 0.0;
            vg[r] = r < C ? *cluster.map_shared_rank(part + (b * 3 + 2) * npair + pr, r) : 0.0;
          }
          double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
          for (int r = 0; r < 16; ++r) {
            al += va[r];
            be += vb[r];
            ga += vg[r];
          }
          if (ga != 0.0 && fabs(ga) > tol * sqrt(al * be)) {
            const double zeta = (be - al) / (2.0 * ga);
            const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            cc = 1.0 / sqrt(1.0 + tt * tt);
            sn = cc * tt;
            rotated = 1;
          }
        }
        cs[(b * 2 + 0) * npair + pr] = cc;
        cs[(b * 2 + 1) * npair + pr] = sn;
      }
      __syncthreads();
      // rotate my rows of G and V: consecutive threads take consecutive rows of one pair
      for (long long e = tid; e < (long long)npair * (gr + vr); e += nt) {
        const int row = int(e % (gr + vr)), pr = int(e / (gr + vr));
        const double cc = cs[(b * 2 + 0) * npair + pr], sn = cs[(b * 2 + 1) * npair + pr];
        if (sn == 0.0) continue;
        int a = (pr == 0) ? 0 : 1 + (pr - 1 + round) % (qq - 1);
        int c = 1 + (qq - 2 - pr + round) % (qq - 1);
        if (a > c) {
          const int tmp = a;
          a = c;
          c = tmp;
        }
        double* X;
        int ld, li;
        if (row < gr) {
          X = G;
          ld = cp;
          li = row;
        } else {
          X = V;
          ld = cv;
          li = row - gr;
        }
        const double x = X[(long long)a * ld + li], y = X[(long long)c * ld + li];
        X[(long long)a * ld + li] = cc * x - sn * y;
        X[(long long)c * ld + li] = sn * x + cc * y;
      }
    }
    if (tid == 0) s_rot = 0;
    __syncthreads();
    if (rotated) s_rot = 1;   // benign race: every writer stores 1
    __syncthreads();
    if (!s_rot) break;        // identical in every CTA (same sums, same decisions)
  }
  if (sweep >= s.max_sweeps && tid == 0 && rank == 0) atomicOr(s.flag, FLAG_SVD_NOCONV);
  // column norms of G over all rows, then a stable descending order
  cluster.sync();
  const int b = t & 1;
  for (int j = tid; j < q; j += nt) {
    const double* x = G + (long long)j * cp;
    double v = 0.0;
    for (int i = 0; i < gr; ++i) v = fma(x[i], x[i], v);
    nrm[j] = v;
  }
  __syncthreads();
  // publish squared norms through the part buffer (size 3*npair >= q)
  for (int j = tid; j < q; j += nt) part[b * 3 * npair + j] = nrm[j];
  cluster.sync();
  for (int j = tid; j < q; j += nt) {
    double v = 0.0;
    v = remote_sum(cluster, part + b * 3 * npair + j, C);
    nrm[j] = sqrt(v);
  }
  __syncthreads();
  for (int j = tid; j < q; j += nt) {
    const double vj = nrm[j];
    int r = 0;
    for (int i = 0; i < q; ++i) {
      const double vi = nrm[i];
      r += (vi > vj) || (vi == vj && i < j);
    }
    order[r] = j;
  }
  __syncthreads();
  const int kk = s.kk;
  double* const US = s.US.d(pb);
  double* const Vt = s.Vt.d(pb);
  if (!s.trans) {
    // US[i][r] = G(i, order[r]) for my G rows; Vt[r][j] = V(j, order[r]) for my V rows
    for (long long e = tid; e < (long long)gr * kk; e += nt) {
      const int li = int(e / kk), r = int(e % kk);
      US[(long long)(g0 + li) * kk + r] = (r < q) ? G[(long long)order[r] * cp + li] : 0.0;
    }
    for (long long e = tid; e < (long long)vr * kk; e += nt) {
      const int li = int(e / kk), r = int(e % kk);
      if (r < kk) Vt[(long long)r * s.n + (v0 + li)] = (r < q) ? V[(long long)order[r] * cv + li] : 0.0;
    }
  } else {
    // US[i][r] = V(i, order[r]) * nrm for my V rows; Vt[r][j] = G(j, order[r]) / nrm for my G rows
    for (long long e = tid; e < (long long)vr * kk; e += nt) {
      const int li = int(e / kk), r = int(e % kk);
      US[(long long)(v0 + li) * kk + r] = (r < q) ? V[(long long)order[r] * cv + li] * nrm[order[r]] : 0.0;
    }
    for (long long e = tid; e < (long long)gr * kk; e += nt) {
      const int li = int(e / kk), r = int(e % kk);
      const double nr = (r < q) ? nrm[order[r]] : 0.0;
      Vt[(long long)r * s.n + (g0 + li)] = (r < q && nr > 0.0) ? G[(long long)order[r] * cp + li] / nr : 0.0;
    }
  }
  cluster.sync();   // no CTA leaves while others may still read its shared memory
}

}  // namespace

namespace {
// Largest cluster size (16 non-portable, else 8, 4, 2) with which `kern` can be
// launched with `smem` bytes of dynamic shared memory per CTA; 1 if clusters
// are unavailable.  Cached per kernel and size.
template <class K>
int cluster_size_for(K kern, int threads, size_t smem) {
  static std::mutex mu;
  static std::vector<std::tuple<const void*, size_t, int>> cache;
  static std::vector<std::pair<const void*, bool>> attrs;
  std::lock_guard<std::mutex> g(mu);
  const void* id = reinterpret_cast<const void*>(kern);
  const size_t key = (smem + 4095) / 4096 * 4096;
  for (auto& e : cache)
    if (std::get<0>(e) == id && std::get<1>(e) == key) return std::get<2>(e);
  bool attrs_ok = false, seen = false;
  for (auto& a : attrs)
    if (a.first == id) {
      attrs_ok = a.second;
      seen = true;
    }
  if (!seen) {
    attrs_ok = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
               cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) == cudaSuccess;
    cudaGetLastError();
    attrs.push_back({id, attrs_ok});
  }
  int best = 1;
  if (attrs_ok) {
    for (int c : {16, 8, 4, 2}) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(c, 1, 1);
      cfg.blockDim = dim3(threads, 1, 1);
      cfg.dynamicSmemBytes = key;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = c;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      const cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
      if (std::getenv("PEPS_VERBOSE"))
        std::fprintf(stderr, "[peps] qr cluster %d smem %zu: %s, %d active clusters\n", c, key,
                     cudaGetErrorString(e), nclusters);
      cudaGetLastError();
      if (e == cudaSuccess && nclusters > 0) {
        best = c;
        break;
      }
    }
  }
  cache.push_back(std::make_tuple(id, key, best));
  return best;
}

int qr_cluster_size(size_t smem) { return cluster_size_for(k_qr_cluster, QRC_THREADS, smem); }
}  // namespace

namespace {

constexpr size_t kQrSmemMax = 200 * 1024;

// Shared memory a cluster QR of an m x n matrix needs per CTA with its rows
// split over c CTAs (rows of the working matrix and of Q, odd column stride).
size_t qr_smem(int m, int n, int c) {
  const int k = std::min(m, n);
  const size_t base = sizeof(double) * (4 * size_t(n) + 2 + k + size_t(n) * QS + n + 2 + QS);
  const size_t ld = size_t(((m + c - 1) / c) | 1);
  return base + sizeof(double) * ld * size_t(n);
}

// dst[b][i*qrs + j*qcs] = src[b][i*n + j]
__global__ void k_copy_strided(const TP src, const TP dst, int m, int n, long long qrs, long long qcs) {
  const double* s = src.d(blockIdx.y);
  double* d = dst.d(blockIdx.y);
  const long long total = (long long)m * n;
  const bool rows_fast = qrs < qcs;   // write along whichever index is contiguous in dst
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = rows_fast ? e % m : e / n, j = rows_fast ? e / m : e % n;
    d[i * qrs + j * qcs] = s[i * n + j];
  }
}

// Leaves of a tall-skinny QR: the smallest power of two L >= 2 that divides m
// and whose leaves (m / L rows, at least 32 per CTA of a 16-CTA cluster)
// keep their rows in shared memory; 0 if none.
int tsqr_leaves(int m, int n) {
  for (int L = 2; L <= 16; L *= 2) {
    if (m % L) return 0;
    const int ml = m / L;
    if (ml < n || ml < 16 * 32) return 0;
    if (qr_smem(ml, n, 16) <= kQrSmemMax) return L;
  }
  return 0;
}

}  // namespace

void qr_direct(Ctx& cx, int m, int n, const TP& A, long long rs, long long cs, const TP& Q, long long qrs,
               long long qcs, const TP& R, double counted_flops);

// Algorithmic flops of one thin QR (the count used for rooflines): 2mn^2 - 2n^3/3.
double qr_flops(int m, int n) {
  const double k = std::min(m, n);
  return 2.0 * m * double(n) * k - 2.0 / 3.0 * k * k * k;
}

// Tall-skinny QR (Demmel, Grigori, Hoemmen & Langou): the rows are split into
// L leaves factored together as one batched cluster QR (rows in shared
// memory), the L stacked R factors are factored once more, and each leaf's Q
// is its own Q times its block of the second Q (one batched FP64 GEMM).  Q is
// the Householder Q of A up to the sign of each column; R likewise.
void qr_tsqr(Ctx& cx, int m, int n, int L, const TP& A, long long rs, long long cs, const TP& Q, long long qrs,
             long long qcs, const TP& R, int np) {
  const int ml = m / L;
  const size_t qn = size_t(ml) * n, rn = size_t(n) * n;
  double* qleaf = cx.ws->dalloc(size_t(np) * L * qn);
  double* rstack = cx.ws->dalloc(size_t(np) * L * rn);
  double* qtree = cx.ws->dalloc(size_t(np) * L * rn);
  TP Al, Ql, Rl, Bt, Ct, At, Qt;
  Al.n = Ql.n = Rl.n = Bt.n = Ct.n = np * L;
  At.n = Qt.n = np;
  const bool direct_out = (qrs == n && qcs == 1);
  double* qout = direct_out ? nullptr : cx.ws->dalloc(size_t(np) * m * n);
  for (int b = 0; b < np; ++b) {
    At.p[b] = rstack + size_t(b) * L * rn;
    Qt.p[b] = qtree + size_t(b) * L * rn;
    for (int i = 0; i < L; ++i) {
      const int j = b * L + i;
      Al.p[j] = A.d(b) + (long long)i * ml * rs;
      Ql.p[j] = qleaf + size_t(j) * qn;
      Rl.p[j] = rstack + size_t(j) * rn;
      Bt.p[j] = qtree + size_t(j) * rn;
      Ct.p[j] = direct_out ? Q.d(b) + size_t(i) * qn : qout + size_t(b) * m * n + size_t(i) * qn;
    }
  }
  // The three steps are charged to the QR class, with the algorithmic flops of
  // the whole factorisation counted once.
  qr_direct(cx, ml, n, Al, rs, cs, Ql, n, 1, Rl, qr_flops(m, n) * np);
  qr_direct(cx, L * n, n, At, n, 1, Qt, n, 1, R, 0.0);
  cx.f64_class = K_QR;
  cx.f64_flops = false;
  ein(cx, "ik,kj->ij", Ql, {ml, n}, Bt, {n, n}, Ct);
  cx.f64_class = -1;
  cx.f64_flops = true;
  if (!direct_out) {
    TP src;
    src.n = np;
    for (int b = 0; b < np; ++b) src.p[b] = qout + size_t(b) * m * n;
    Launch Lc(K_QR, cx.st);
    k_copy_strided<<<dim3(unsigned(std::min<long long>(4096, ((long long)m * n + 255) / 256)), np), 256, 0, cx.st>>>(
        src, Q.all(np), m, n, qrs, qcs);
    PEPS_CHECK_LAUNCH();
  }
}

void qr_thin(Ctx& cx, int m, int n, const TP& A, long long rs, long long cs, const TP& Q, long long qrs,
             long long qcs, const TP& R) {
  PEPS_REQUIRE(m > 0 && n > 0, "qr of an empty matrix");
  const int np = problems({&A, &Q, &R});
  PEPS_REQUIRE(!A.null() && Q.n == np && (R.null() || R.n == np), "internal: qr operands");
  // Rows that do not fit in the shared memory of a 16-CTA cluster: tall-skinny
  // QR over leaves that do (more SMs per factorisation, rows on chip).
  if (m >= n && cx.qr_cmax <= 0 && qr_smem(m, n, 16) > kQrSmemMax) {
    const int L = tsqr_leaves(m, n);
    if (L > 1 && np * L <= MAXB) {
      qr_tsqr(cx, m, n, L, A, rs, cs, Q, qrs, qcs, R, np);
      return;
    }
  }
  qr_direct(cx, m, n, A, rs, cs, Q, qrs, qcs, R, qr_flops(m, n) * np);
}

void qr_direct(Ctx& cx, int m, int n, const TP& A, long long rs, long long cs, const TP& Q, long long qrs,
               long long qcs, const TP& R, double counted_flops) {
  const int np = problems({&A, &Q, &R});
  const int k = std::min(m, n);
  // work of the Householder factorisation with Q formed (for the cluster-size model)
  const double flops = 4.0 * m * double(n) * k - 4.0 / 3.0 * double(k) * k * k;
  const size_t base = sizeof(double) * (4 * size_t(n) + 2 + k + size_t(n) * QS + n + 2 + QS);
  auto ld_of = [&](int c) { return (((m + c - 1) / c) | 1); };   // odd column stride
  auto full_of = [&](int c) { return qr_smem(m, n, c); };
  // Cluster size: rows per CTA >= 32; among the sizes whose rows fit in shared
  // memory, the one with the least estimated time for all problems: waves of
  // clusters over the SMs x (FP64 work per CTA + three cluster barriers per column).
  int cmax = std::max(1, std::min(cx.qr_cmax > 0 ? cx.qr_cmax : 16, m / 32));
  while (cmax > 1 && (cmax & (cmax - 1))) --cmax;
  int C = cmax;
  if (cmax > 1) {
    double best = 1e300;
    for (int c = 2; c <= cmax; c *= 2) {
      if (full_of(c) > kQrSmemMax && c < cmax) continue;
      const double waves = std::ceil(double(np) * c / 144.0);
      const double t = waves * (flops / (c * 8.0e9) + 3.0 * k * 1.5e-6);
      if (t < best) {
        best = t;
        C = c;
      }
    }
    C = std::min(C, qr_cluster_size(full_of(C) <= kQrSmemMax ? full_of(C) : base));
    while (C > 1 && (C & (C - 1))) --C;
  }
  if (std::getenv("PEPS_VERBOSE")) std::fprintf(stderr, "[peps] qr %dx%d x%d: cluster %d\n", m, n, np, C);
  const int ld = ld_of(std::max(C, 1));
  const bool in_smem = C > 1 && full_of(C) <= kQrSmemMax;
  QrArgs a;
  std::memset(static_cast<void*>(&a), 0, sizeof(a));
  a.m = m;
  a.n = n;
  a.A = A.all(np);
  a.rs = rs;
  a.cs = cs;
  a.Q = Q.all(np);
  a.qrs = qrs;
  a.qcs = qcs;
  a.R = R.all(np);
  if (C <= 1) {
    a.wst = (long long)m * n;
    a.qst = (long long)m * k;
  } else {   // the global-memory fallback uses [C][n][ld] blocks per problem (Q formed in place)
    a.wst = (long long)C * ld * n;
    a.qst = 0;
  }
  a.tst = k;
  double* w = cx.scratch(size_t(np) * (a.wst + a.qst + a.tst) + 64);
  a.W = w;
  a.Qw = w + size_t(np) * a.wst;
  a.tau = a.Qw + size_t(np) * a.qst;
  Launch L(K_QR, cx.st, counted_flops, 0);
  if (C <= 1) {
    k_qr_house<<<np, QR_THREADS, 0, cx.st>>>(a);
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C * np, 1, 1);
    cfg.blockDim = dim3(QRC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = in_smem ? full_of(C) : base;
    cfg.stream = cx.st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    PEPS_CUDA(cudaLaunchKernelEx(&cfg, k_qr_cluster, a, in_smem ? 1 : 0, ld));
  }
  PEPS_CHECK_LAUNCH();
}

void svd_trunc(Ctx& cx, int m, int n, const TP& A, int kk, const TP& US, const TP& Vt) {
  PEPS_REQUIRE(m > 0 && n > 0 && kk > 0, "svd of an empty matrix");
  const int np = problems({&A, &US, &Vt});
  PEPS_REQUIRE(!A.null() && US.n == np && Vt.n == np, "internal: svd operands");
  SvdArgs s;
  std::memset(static_cast<void*>(&s), 0, sizeof(s));
  s.trans = (m < n) ? 1 : 0;
  s.p = s.trans ? n : m;
  s.q = s.trans ? m : n;
  s.m = m;
  s.n = n;
  s.A = A.all(np);
  s.kk = kk;
  s.US = US.all(np);
  s.Vt = Vt.all(np);
  s.flag = cx.flag;
  s.max_sweeps = std::max(1, cx.svd_cap);
  s.wst = ((long long)s.p * s.q + (long long)s.q * s.q + 2LL * s.q + 31) / 32 * 32;
  s.work = cx.scratch(size_t(np) * s.wst);
  const double flops = 8.0 * 4.0 * double(s.p) * s.q * s.q;
  // Matrices of 4096+ entries: rows split over a thread-block cluster (16 rows per CTA or more).
  int C = 1;
  if (double(s.p) * s.q >= 4096.0) {
    C = std::max(1, std::min(16, s.p / 16));
    while (C > 1 && (C & (C - 1))) --C;
  }
  const int npair = (s.q + (s.q & 1)) / 2;
  const size_t smem = sizeof(double) * (10 * size_t(npair) + s.q + (s.q + 1) / 2 + 8);
  if (C > 1) C = std::min(C, cluster_size_for(k_svd_cluster, SVC_THREADS, smem));
  while (C > 1 && (C & (C - 1))) --C;
  Launch L(K_SVD, cx.st, flops * np, 0);
  if (C <= 1) {
    k_svd_jacobi<<<np, SVD_THREADS, 0, cx.st>>>(s);
  } else {
    const int cp = (s.p + C - 1) / C, cv = (s.q + C - 1) / C;
    const long long cwst = (long long)C * cp * s.q + (long long)C * cv * s.q;
    double* cwork = cx.scratch(size_t(np) * cwst + 64);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C * np, 1, 1);
    cfg.blockDim = dim3(SVC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = cx.st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    PEPS_CUDA(cudaLaunchKernelEx(&cfg, k_svd_cluster, s, cwork, cwst));
  }
  PEPS_CHECK_LAUNCH();
}

}  // namespace peps
