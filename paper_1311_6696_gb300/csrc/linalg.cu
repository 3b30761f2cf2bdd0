// FP64 Householder QR and one-sided Jacobi SVD, one CTA per matrix.
//
// The working copy lives in global memory (column-major) and stays in L2 at
// the sizes used here (<= a few MB).  Reductions over a column are done by one
// warp per column; a CTA handles all columns of one matrix.
#include <algorithm>
#include <cmath>

#include "linalg.cuh"

namespace peps {
namespace {

constexpr int QR_THREADS = 512;
constexpr int SVD_THREADS = 512;
constexpr int SVD_MAX_SWEEPS = 60;

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
  const double* A;
  long long rs, cs;
  double* Q;
  long long qrs, qcs;
  double* R;
  double* W;    // m*n work, column-major
  double* Qw;   // m*k work, column-major
  double* tau;  // k
};

__global__ void __launch_bounds__(QR_THREADS) k_qr_house(const QrArgs q) {
  __shared__ double red[32];
  __shared__ double s_tau, s_scale;
  const int m = q.m, n = q.n, k = min(m, n);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  double* W = q.W;
  for (long long e = tid; e < (long long)m * n; e += nt) {
    int i = int(e % m), j = int(e / m);
    W[e] = q.A[i * q.rs + j * q.cs];
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
      q.tau[j] = s_tau;
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
  double* Qw = q.Qw;
  for (long long e = tid; e < (long long)m * k; e += nt) {
    int i = int(e % m), j = int(e / m);
    Qw[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const double tau = q.tau[j];
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
    q.Q[i * q.qrs + j * q.qcs] = Qw[e];
  }
  if (q.R) {
    for (long long e = tid; e < (long long)k * n; e += nt) {
      int i = int(e / n), j = int(e % n);
      q.R[e] = (j >= i) ? W[(long long)j * m + i] : 0.0;
    }
  }
}

struct SvdArgs {
  int p, q;          // working matrix G is p x q (p >= q), column-major
  int m, n;          // original A is m x n row-major
  int trans;         // 1: G = A^T (m < n)
  const double* A;
  double* G;
  double* V;         // q x q column-major
  double* nrm;       // q
  int* order;        // q
  int kk;
  double* US;        // m x kk row-major
  double* Vt;        // kk x n row-major
  int* flag;
};

__global__ void __launch_bounds__(SVD_THREADS) k_svd_jacobi(const SvdArgs s) {
  __shared__ int s_rot;
  const int p = s.p, q = s.q;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  double* G = s.G;
  double* V = s.V;
  for (long long e = tid; e < (long long)p * q; e += nt) {
    int i = int(e % p), j = int(e / p);   // G(i,j)
    G[e] = s.trans ? s.A[(long long)j * s.n + i] : s.A[(long long)i * s.n + j];
  }
  for (long long e = tid; e < (long long)q * q; e += nt) V[e] = ((e % q) == (e / q)) ? 1.0 : 0.0;
  __syncthreads();
  const int qq = q + (q & 1);   // even number of slots for the round-robin pairing
  const double tol = 1e-15;
  int sweep = 0;
  for (; sweep < SVD_MAX_SWEEPS; ++sweep) {
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
  if (sweep >= SVD_MAX_SWEEPS && tid == 0) atomicOr(s.flag, FLAG_SVD_NOCONV);
  // column norms and a stable descending order
  for (int j = warp; j < q; j += nw) {
    double v = 0.0;
    for (int i = lane; i < p; i += 32) {
      double x = G[(long long)j * p + i];
      v += x * x;
    }
    v = warp_sum(v);
    if (lane == 0) s.nrm[j] = sqrt(v);
  }
  __syncthreads();
  for (int j = tid; j < q; j += nt) {
    const double vj = s.nrm[j];
    int r = 0;
    for (int i = 0; i < q; ++i) {
      const double vi = s.nrm[i];
      r += (vi > vj) || (vi == vj && i < j);
    }
    s.order[r] = j;
  }
  __syncthreads();
  // A V = G  (A = G V^T when trans = 0;  A^T = G V^T  =>  A = V G^T when trans = 1)
  const int kk = s.kk;
  if (!s.trans) {
    // US[i][r] = G(i, order[r]);  Vt[r][j] = V(j, order[r])
    for (long long e = tid; e < (long long)s.m * kk; e += nt) {
      int i = int(e / kk), r = int(e % kk);
      s.US[e] = (r < q) ? G[(long long)s.order[r] * p + i] : 0.0;
    }
    for (long long e = tid; e < (long long)kk * s.n; e += nt) {
      int r = int(e / s.n), j = int(e % s.n);
      s.Vt[e] = (r < q) ? V[(long long)s.order[r] * q + j] : 0.0;
    }
  } else {
    // US[i][r] = V(i, order[r]) * nrm;  Vt[r][j] = G(j, order[r]) / nrm
    for (long long e = tid; e < (long long)s.m * kk; e += nt) {
      int i = int(e / kk), r = int(e % kk);
      s.US[e] = (r < q) ? V[(long long)s.order[r] * q + i] * s.nrm[s.order[r]] : 0.0;
    }
    for (long long e = tid; e < (long long)kk * s.n; e += nt) {
      int r = int(e / s.n), j = int(e % s.n);
      double nr = (r < q) ? s.nrm[s.order[r]] : 0.0;
      s.Vt[e] = (r < q && nr > 0.0) ? G[(long long)s.order[r] * p + j] / nr : 0.0;
    }
  }
}

}  // namespace

void qr_thin(Ctx& cx, int m, int n, const double* A, long long rs, long long cs, double* Q,
             long long qrs, long long qcs, double* R) {
  PEPS_REQUIRE(m > 0 && n > 0, "qr of an empty matrix");
  const int k = std::min(m, n);
  double* w = cx.scratch(size_t(m) * n + size_t(m) * k + k);
  QrArgs a{m, n, A, rs, cs, Q, qrs, qcs, R, w, w + size_t(m) * n, w + size_t(m) * n + size_t(m) * k};
  const double flops = 4.0 * m * double(n) * k - 4.0 / 3.0 * double(k) * k * k;
  Launch L(K_QR, cx.st, flops, 0);
  k_qr_house<<<1, QR_THREADS, 0, cx.st>>>(a);
  PEPS_CHECK_LAUNCH();
}

void svd_trunc(Ctx& cx, int m, int n, const double* A, int kk, double* US, double* Vt) {
  PEPS_REQUIRE(m > 0 && n > 0 && kk > 0, "svd of an empty matrix");
  SvdArgs s;
  s.trans = (m < n) ? 1 : 0;
  s.p = s.trans ? n : m;
  s.q = s.trans ? m : n;
  s.m = m;
  s.n = n;
  s.A = A;
  s.kk = kk;
  s.US = US;
  s.Vt = Vt;
  s.flag = cx.flag;
  const size_t need = size_t(s.p) * s.q + size_t(s.q) * s.q + s.q + s.q;
  double* w = cx.scratch(need);
  s.G = w;
  s.V = w + size_t(s.p) * s.q;
  s.nrm = s.V + size_t(s.q) * s.q;
  s.order = reinterpret_cast<int*>(s.nrm + s.q);
  const double flops = 8.0 * 4.0 * double(s.p) * s.q * s.q;
  Launch L(K_SVD, cx.st, flops, 0);
  k_svd_jacobi<<<1, SVD_THREADS, 0, cx.st>>>(s);
  PEPS_CHECK_LAUNCH();
}

}  // namespace peps
