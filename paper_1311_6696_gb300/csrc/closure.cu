// Learned cluster closure (build-defined; the paper has no learned part).
//
// A three-layer MLP maps local data at one outward leg of a cluster window --
// the site tensor just above the cut, the CU_0 matrix sigma0 there and its
// Cholesky factor L0 -- to X = L0 + net(x); the closure matrix is
// X X^T / ||X X^T||_F, which is positive and equals sigma0 when the network
// outputs zero.  Labels are the site matrices of the best product (D'=1)
// approximation of the full boundary at the same cut.  The three GEMMs of
// each pass run on the tensor cores (BF16 operands, FP32 accumulation);
// bias, ReLU, the sigma map with its loss and gradient, and AdamW are
// elementwise kernels here.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "closure.cuh"
#include "linalg.cuh"

namespace peps {
namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

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

// ---------------------------------------------------------------- features
__global__ void k_features(const RimSite* sites, int d, int D, int F, float* X) {
  const RimSite s = sites[blockIdx.x];
  float* x = X + (long long)blockIdx.x * F;
  const int DD = D * D, n1 = d * DD * DD;
  for (int e = threadIdx.x; e < n1; e += blockDim.x) {
    int t = e;
    const int r = t % D; t /= D;
    const int n = t % D; t /= D;
    const int l = t % D; t /= D;
    const int u = t % D;
    const int ph = t / D;
    float v = 0.f;
    if (u < s.du && l < s.dl && n < s.dn && r < s.dr)
      v = float(s.A[(((ph * s.du + u) * s.dl + l) * s.dn + n) * s.dr + r]);
    x[e] = v;
  }
  for (int e = threadIdx.x; e < DD; e += blockDim.x) x[n1 + e] = float(s.sigma[e]);
  if (threadIdx.x == 0) {
    // lower Cholesky factor of sigma (+ a tiny diagonal shift), in double
    double L[16 * 16];
    for (int i = 0; i < D; ++i)
      for (int j = 0; j <= i; ++j) {
        double a = s.sigma[i * D + j] + (i == j ? 1e-12 : 0.0);
        for (int k = 0; k < j; ++k) a -= L[i * D + k] * L[j * D + k];
        L[i * D + j] = (i == j) ? sqrt(fmax(a, 1e-30)) : a / L[j * D + j];
      }
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) x[n1 + DD + i * D + j] = j <= i ? float(L[i * D + j]) : 0.f;
  }
}

// ---------------------------------------------------------------- labels
__global__ void __launch_bounds__(256) k_rank1(const Rank1Job* jobs, int D, double* work, long long wstride,
                                               int* flag) {
  __shared__ double red[32];
  const Rank1Job J = jobs[blockIdx.x];
  const int L = J.L, DD = D * D, tid = threadIdx.x, nt = blockDim.x;
  int chi = 1;
  for (int x = 0; x <= L; ++x) chi = max(chi, J.bonds[x]);
  double* sig = work + blockIdx.x * wstride;       // [L][DD]
  double* rv = sig + (long long)L * DD;            // [L][chi]
  double* lv = rv + (long long)L * chi;            // [chi]
  double* tmp = lv + chi;                          // [max(chi, DD)]
  const double inv = 1.0 / sqrt(double(D));
  for (int x = 0; x < L; ++x)
    for (int e = tid; e < DD; e += nt) sig[x * DD + e] = (e / D == e % D) ? inv : 0.0;
  __syncthreads();
  bool conv = false;
  for (int h = 0; h < 200 && !conv; ++h) {
    // right vectors from the current matrices
    for (int e = tid; e < J.bonds[L]; e += nt) rv[(long long)(L - 1) * chi + e] = 1.0;
    __syncthreads();
    for (int x = L - 1; x >= 1; --x) {
      const int a = J.bonds[x], b = J.bonds[x + 1];
      const double* M = J.sites[x];
      for (int i = tid; i < a; i += nt) {
        double acc = 0.0;
        for (int uv = 0; uv < DD; ++uv)
          for (int j = 0; j < b; ++j) acc += M[((long long)i * DD + uv) * b + j] * sig[x * DD + uv] * rv[(long long)x * chi + j];
        tmp[i] = acc;
      }
      __syncthreads();
      double p = 0.0;
      for (int i = tid; i < a; i += nt) p += tmp[i] * tmp[i];
      const double nr = sqrt(block_sum(p, red));
      for (int i = tid; i < a; i += nt) rv[(long long)(x - 1) * chi + i] = tmp[i] / nr;
      __syncthreads();
    }
    for (int e = tid; e < J.bonds[0]; e += nt) lv[e] = 1.0;
    __syncthreads();
    double change = 0.0;
    for (int x = 0; x < L; ++x) {
      const int a = J.bonds[x], b = J.bonds[x + 1];
      const double* M = J.sites[x];
      for (int uv = tid; uv < DD; uv += nt) {
        double acc = 0.0;
        for (int i = 0; i < a; ++i)
          for (int j = 0; j < b; ++j) acc += lv[i] * M[((long long)i * DD + uv) * b + j] * rv[(long long)x * chi + j];
        tmp[uv] = acc;
      }
      __syncthreads();
      double p = 0.0, tr = 0.0;
      for (int uv = tid; uv < DD; uv += nt) {
        p += tmp[uv] * tmp[uv];
        if (uv / D == uv % D) tr += tmp[uv];
      }
      const double nr = sqrt(block_sum(p, red));
      const double trace = block_sum(tr, red);
      const double sgn = trace < 0 ? -1.0 : 1.0;
      double c = 0.0;
      for (int uv = tid; uv < DD; uv += nt) {
        const double v = sgn * tmp[uv] / nr;
        const double df = v - sig[x * DD + uv];
        c += df * df;
        sig[x * DD + uv] = v;
      }
      change = fmax(change, sqrt(block_sum(c, red)));
      if (x < L - 1) {
        for (int j = tid; j < b; j += nt) {
          double acc = 0.0;
          for (int i = 0; i < a; ++i)
            for (int uv = 0; uv < DD; ++uv) acc += lv[i] * M[((long long)i * DD + uv) * b + j] * sig[x * DD + uv];
          tmp[j] = acc;
        }
        __syncthreads();
        double q = 0.0;
        for (int j = tid; j < b; j += nt) q += tmp[j] * tmp[j];
        const double nq = sqrt(block_sum(q, red));
        for (int j = tid; j < b; j += nt) lv[j] = tmp[j] / nq;
        __syncthreads();
      }
    }
    conv = change < 1e-12;
  }
  if (!conv && tid == 0) atomicOr(flag, FLAG_CU0_NOCONV);
  for (int e = tid; e < L * DD; e += nt) J.out[e] = float(sig[e]);
}

// ---------------------------------------------------------------- MLP pieces
__global__ void k_init(float* w, int F, int W, int out, unsigned long long seed) {
  const long long n1 = (long long)W * F, n2 = n1 + W, n3 = n2 + (long long)W * W, n4 = n3 + W;
  const long long n5 = n4 + (long long)out * W, n6 = n5 + out;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n6; i += (long long)gridDim.x * blockDim.x) {
    const double u = double(mix64(seed * 0x9E3779B97F4A7C15ULL + (unsigned long long)i + 0x9E3779B97F4A7C15ULL) >> 11) *
                     (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    float v = 0.f;
    if (i < n1) v = float(u * sqrt(6.0 / F));
    else if (i >= n2 && i < n3) v = float(u * sqrt(6.0 / W));
    w[i] = v;   // biases and the output layer start at zero
  }
}

__global__ void k_bias_act(float* Z, const float* b, long long n, int W, int relu) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n * W; i += (long long)gridDim.x * blockDim.x) {
    float v = Z[i] + b[i % W];
    Z[i] = relu ? fmaxf(v, 0.f) : v;
  }
}

__global__ void k_relu_bwd(float* dH, const float* H, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (H[i] <= 0.f) dH[i] = 0.f;
}

// db[c] = sum_b dZ[b][c]: one block per column chunk, rows strided, fixed order
__global__ void k_colsum(const float* dZ, long long n, int W, float* db) {
  __shared__ double red[32];
  for (int c = blockIdx.x; c < W; c += gridDim.x) {
    double s = 0.0;
    for (long long b = threadIdx.x; b < n; b += blockDim.x) s += dZ[b * W + c];
    s = block_sum(s, red);
    if (threadIdx.x == 0) db[c] = float(s);
  }
}

// sigma = X X^T / ||X X^T||, X = L0 + Yo;  loss and dL/dYo (mean over n)
__global__ void k_sigma(const float* Xin, int F, const float* Yo, const float* lab, long long n, int D, float* sig,
                        float* dYo, double* loss_part) {
  __shared__ double red[32];
  const int DD = D * D;
  double lsum = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double X[64], S[64];
    const float* L0 = Xin + e * F + (F - DD);
    for (int i = 0; i < DD; ++i) X[i] = double(L0[i]) + double(Yo[e * DD + i]);
    double nr = 0.0;
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        double a = 0.0;
        for (int k = 0; k < D; ++k) a += X[i * D + k] * X[j * D + k];
        S[i * D + j] = a;
        nr += a * a;
      }
    nr = sqrt(nr);
    const double inv = nr > 0 ? 1.0 / nr : 0.0;
    if (sig)
      for (int i = 0; i < DD; ++i) sig[e * DD + i] = float(S[i] * inv);
    if (lab) {
      double G[64], gs = 0.0;
      for (int i = 0; i < DD; ++i) {
        const double df = S[i] * inv - double(lab[e * DD + i]);
        lsum += df * df;
        G[i] = 2.0 * df / double(n);
        gs += G[i] * S[i] * inv;
      }
      double dS[64];
      for (int i = 0; i < DD; ++i) dS[i] = (G[i] - S[i] * inv * gs) * inv;
      for (int i = 0; i < D; ++i)
        for (int k = 0; k < D; ++k) {
          double a = 0.0;
          for (int j = 0; j < D; ++j) a += (dS[i * D + j] + dS[j * D + i]) * X[j * D + k];
          dYo[e * DD + i * D + k] = float(a);
        }
    }
  }
  if (loss_part) {
    lsum = block_sum(lsum, red);
    if (threadIdx.x == 0) loss_part[blockIdx.x] = lsum;
  }
}

__global__ void k_sum_loss(const double* part, int np, long long n, double* out, int accumulate) {
  if (threadIdx.x || blockIdx.x) return;
  double s = 0.0;
  for (int i = 0; i < np; ++i) s += part[i];
  s /= double(n);
  out[0] = accumulate ? out[0] + s : s;
}

__global__ void k_adamw(float* w, const float* g, float* m1, float* m2, long long n, float lr, float wd, float b1,
                        float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    w[i] -= lr * ((a / c1) / (sqrtf(b / c2) + eps) + wd * w[i]);
  }
}

__global__ void k_gather_rows(const float* src, const long long* idx, long long n, int cols, float* dst) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * cols; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / cols;
    dst[t] = src[idx[r] * cols + (t - r * cols)];
  }
}

__global__ void k_apply(const float* pred, double* const* targets, long long n, int D) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int DD = D * D;
  double tr = 0.0;
  bool ok = true;
  for (int i = 0; i < DD; ++i) {
    const float v = pred[e * DD + i];
    ok = ok && isfinite(v);
    if (i / D == i % D) tr += v;
  }
  if (!ok || !(tr > 0.0)) return;      // fall back to the CU_0 matrix
  for (int i = 0; i < DD; ++i) targets[e][i] = double(pred[e * DD + i]);
}

unsigned grid_for(long long n) {
  return unsigned(std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096)));
}

struct Layers {
  const float *W1, *b1, *W2, *b2, *W3, *b3;
};

Layers layers(const MlpDims& m, const float* w) {
  const long long F = m.F(), W = m.W, o = m.out();
  Layers L;
  L.W1 = w;
  L.b1 = L.W1 + W * F;
  L.W2 = L.b1 + W;
  L.b2 = L.W2 + W * W;
  L.W3 = L.b2 + W;
  L.b3 = L.W3 + o * W;
  return L;
}

constexpr int kMlpPrec = PEPS_PREC_BF16;

// Forward pass; H1, H2 (n x W) and Yo (n x out) are caller buffers.
void forward(Ctx& cx, const MlpDims& m, const float* w, const float* X, long long n, float* H1, float* H2, float* Yo) {
  const Layers L = layers(m, w);
  const int F = m.F(), W = m.W, o = m.out();
  const int nn = int(n);
  ein_tc(cx, "bi,wi->bw", X, 0, {nn, F}, L.W1, 0, {W, F}, H1, 0, kMlpPrec);
  {
    Launch l(K_AUX, cx.st);
    k_bias_act<<<grid_for(n * W), 256, 0, cx.st>>>(H1, L.b1, n, W, 1);
  }
  ein_tc(cx, "bw,vw->bv", H1, 0, {nn, W}, L.W2, 0, {W, W}, H2, 0, kMlpPrec);
  {
    Launch l(K_AUX, cx.st);
    k_bias_act<<<grid_for(n * W), 256, 0, cx.st>>>(H2, L.b2, n, W, 1);
  }
  ein_tc(cx, "bv,ov->bo", H2, 0, {nn, W}, L.W3, 0, {o, W}, Yo, 0, kMlpPrec);
  Launch l(K_AUX, cx.st);
  k_bias_act<<<grid_for(n * o), 256, 0, cx.st>>>(Yo, L.b3, n, o, 0);
  PEPS_CHECK_LAUNCH();
}

}  // namespace

void closure_features(Ctx& cx, const MlpDims& m, const RimSite* host_sites, long long n, float* X) {
  if (n == 0) return;
  PEPS_REQUIRE(m.D <= 8, "learned closure supports D <= 8");
  auto* dev = static_cast<const RimSite*>(stage(cx, host_sites, sizeof(RimSite) * n));
  Launch l(K_AUX, cx.st);
  k_features<<<unsigned(n), 256, 0, cx.st>>>(dev, m.d, m.D, m.F(), X);
  PEPS_CHECK_LAUNCH();
}

void rank1_labels(Ctx& cx, int D, int maxchi, int maxL, const Rank1Job* host_jobs, int njobs) {
  if (njobs == 0) return;
  const long long DD = (long long)D * D;
  const long long wstride = maxL * DD + (long long)maxL * maxchi + maxchi + std::max<long long>(maxchi, DD) + 8;
  double* work = cx.ws->dalloc(size_t(wstride) * njobs);
  auto* dev = static_cast<const Rank1Job*>(stage(cx, host_jobs, sizeof(Rank1Job) * njobs));
  Launch l(K_CU0, cx.st);
  k_rank1<<<njobs, 256, 0, cx.st>>>(dev, D, work, wstride, cx.flag);
  PEPS_CHECK_LAUNCH();
}

void mlp_init(Ctx& cx, const MlpDims& m, float* w, unsigned long long seed) {
  Launch l(K_AUX, cx.st);
  k_init<<<grid_for(m.params()), 256, 0, cx.st>>>(w, m.F(), m.W, m.out(), seed);
  PEPS_CHECK_LAUNCH();
}

void mlp_predict(Ctx& cx, const MlpDims& m, const float* w, const float* X, long long n, float* sigma) {
  if (n == 0) return;
  float* H1 = cx.ws->falloc(size_t(n) * m.W);
  float* H2 = cx.ws->falloc(size_t(n) * m.W);
  float* Yo = cx.ws->falloc(size_t(n) * m.out());
  forward(cx, m, w, X, n, H1, H2, Yo);
  Launch l(K_AUX, cx.st);
  k_sigma<<<grid_for(n), 256, 0, cx.st>>>(X, m.F(), Yo, nullptr, n, m.D, sigma, nullptr, nullptr);
  PEPS_CHECK_LAUNCH();
}

namespace {
// Loss (accumulated into loss_dev if accumulate) and gradient for n examples,
// with caller-provided activation buffers.
void loss_grad_buf(Ctx& cx, const MlpDims& m, const float* w, const float* X, const float* Y, long long n,
                   double* loss_dev, int accumulate, float* grad, float* H1, float* H2, float* Yo, float* dYo,
                   float* dH1, float* dH2, double* part) {
  const Layers L = layers(m, w);
  const int F = m.F(), W = m.W, o = m.out(), nn = int(n);
  forward(cx, m, w, X, n, H1, H2, Yo);
  const unsigned gs = grid_for(n);
  {
    Launch l(K_AUX, cx.st);
    k_sigma<<<gs, 256, 0, cx.st>>>(X, F, Yo, Y, n, m.D, nullptr, dYo, part);
    k_sum_loss<<<1, 32, 0, cx.st>>>(part, int(gs), n, loss_dev, accumulate);
    PEPS_CHECK_LAUNCH();
    l.more();
  }
  float* gW1 = grad;
  float* gb1 = gW1 + (long long)W * F;
  float* gW2 = gb1 + W;
  float* gb2 = gW2 + (long long)W * W;
  float* gW3 = gb2 + W;
  float* gb3 = gW3 + (long long)o * W;
  ein_tc(cx, "bo,bv->ov", dYo, 0, {nn, o}, H2, 0, {nn, W}, gW3, 0, kMlpPrec);
  ein_tc(cx, "bo,ov->bv", dYo, 0, {nn, o}, L.W3, 0, {o, W}, dH2, 0, kMlpPrec);
  {
    Launch l(K_AUX, cx.st);
    k_colsum<<<std::min(o, 1024), 256, 0, cx.st>>>(dYo, n, o, gb3);
    k_relu_bwd<<<grid_for(n * W), 256, 0, cx.st>>>(dH2, H2, n * W);
    k_colsum<<<std::min(W, 1024), 256, 0, cx.st>>>(dH2, n, W, gb2);
    PEPS_CHECK_LAUNCH();
    l.more(2);
  }
  ein_tc(cx, "bv,bw->vw", dH2, 0, {nn, W}, H1, 0, {nn, W}, gW2, 0, kMlpPrec);
  ein_tc(cx, "bv,vw->bw", dH2, 0, {nn, W}, L.W2, 0, {W, W}, dH1, 0, kMlpPrec);
  {
    Launch l(K_AUX, cx.st);
    k_relu_bwd<<<grid_for(n * W), 256, 0, cx.st>>>(dH1, H1, n * W);
    k_colsum<<<std::min(W, 1024), 256, 0, cx.st>>>(dH1, n, W, gb1);
    PEPS_CHECK_LAUNCH();
    l.more();
  }
  ein_tc(cx, "bw,bi->wi", dH1, 0, {nn, W}, X, 0, {nn, F}, gW1, 0, kMlpPrec);
}
}  // namespace

void mlp_loss_grad(Ctx& cx, const MlpDims& m, const float* w, const float* X, const float* Y, long long n,
                   double* loss_dev, float* grad) {
  PEPS_REQUIRE(n > 0, "empty batch");
  const size_t W = m.W, o = m.out();
  float* H1 = cx.ws->falloc(n * W);
  float* H2 = cx.ws->falloc(n * W);
  float* Yo = cx.ws->falloc(n * o);
  float* dYo = cx.ws->falloc(n * o);
  float* dH1 = cx.ws->falloc(n * W);
  float* dH2 = cx.ws->falloc(n * W);
  double* part = cx.ws->dalloc(grid_for(n) + 1);
  loss_grad_buf(cx, m, w, X, Y, n, loss_dev, 0, grad, H1, H2, Yo, dYo, dH1, dH2, part);
}

void mlp_train(Ctx& cx, const MlpDims& m, float* w, const float* X, const float* Y, long long n, int steps,
               int batch, float lr, float wd, unsigned long long seed, double* final_loss_host, float* m1_ext,
               float* m2_ext, long long t0) {
  PEPS_REQUIRE(n > 0 && steps > 0 && batch > 0, "empty training set, steps or batch");
  PEPS_REQUIRE(t0 >= 0, "negative step count");
  const long long B = std::min<long long>(batch, n);
  const size_t P = size_t(m.params()), W = m.W, o = m.out(), F = m.F();
  float* grad = cx.ws->falloc(P);
  float* m1 = m1_ext;
  float* m2 = m2_ext;
  if (!m1 || !m2) {   // state of this call only
    m1 = cx.ws->falloc(P);
    m2 = cx.ws->falloc(P);
    PEPS_CUDA(cudaMemsetAsync(m1, 0, P * sizeof(float), cx.st));
    PEPS_CUDA(cudaMemsetAsync(m2, 0, P * sizeof(float), cx.st));
  }
  float* Xb = cx.ws->falloc(B * F);
  float* Yb = cx.ws->falloc(B * o);
  float* H1 = cx.ws->falloc(B * W);
  float* H2 = cx.ws->falloc(B * W);
  float* Yo = cx.ws->falloc(B * o);
  float* dYo = cx.ws->falloc(B * o);
  float* dH1 = cx.ws->falloc(B * W);
  float* dH2 = cx.ws->falloc(B * W);
  double* part = cx.ws->dalloc(grid_for(B) + 1);
  double* loss_acc = cx.ws->dalloc(1);
  PEPS_CUDA(cudaMemsetAsync(loss_acc, 0, sizeof(double), cx.st));
  long long* didx = static_cast<long long*>(cx.ws->alloc(sizeof(long long) * size_t(steps) * B));
  // minibatch indices: a seeded shuffle per epoch (host side, uploaded once);
  // a run resumed at step t0 continues the same stream
  std::vector<long long> idx(size_t(steps) * B), perm(n);
  std::iota(perm.begin(), perm.end(), 0LL);
  unsigned long long st = seed * 0x9E3779B97F4A7C15ULL + 1;
  auto next = [&st] {
    st += 0x9E3779B97F4A7C15ULL;
    unsigned long long z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  };
  long long pos = n;
  const long long skip = t0 * B;
  for (long long i = 0; i < skip + (long long)idx.size(); ++i) {
    if (pos >= n) {
      for (long long k = n - 1; k > 0; --k) std::swap(perm[k], perm[next() % (unsigned long long)(k + 1)]);
      pos = 0;
    }
    const long long v = perm[pos++];
    if (i >= skip) idx[size_t(i - skip)] = v;
  }
  PEPS_CUDA(cudaMemcpyAsync(didx, idx.data(), sizeof(long long) * idx.size(), cudaMemcpyHostToDevice, cx.st));
  const int tail = std::min(steps, 20);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int t = 0; t < steps; ++t) {
    {
      Launch l(K_AUX, cx.st);
      k_gather_rows<<<grid_for(B * F), 256, 0, cx.st>>>(X, didx + (long long)t * B, B, int(F), Xb);
      k_gather_rows<<<grid_for(B * o), 256, 0, cx.st>>>(Y, didx + (long long)t * B, B, int(o), Yb);
      PEPS_CHECK_LAUNCH();
      l.more();
    }
    const bool rec = t >= steps - tail;
    loss_grad_buf(cx, m, w, Xb, Yb, B, rec ? loss_acc : part + grid_for(B), rec ? 1 : 0, grad, H1, H2, Yo, dYo,
                  dH1, dH2, part);
    const float c1 = 1.f - std::pow(b1, float(t0 + t + 1)), c2 = 1.f - std::pow(b2, float(t0 + t + 1));
    Launch l(K_AUX, cx.st);
    k_adamw<<<grid_for(P), 256, 0, cx.st>>>(w, grad, m1, m2, (long long)P, lr, wd, b1, b2, eps, c1, c2);
    PEPS_CHECK_LAUNCH();
  }
  double h = 0.0;
  PEPS_CUDA(cudaMemcpyAsync(&h, loss_acc, sizeof(double), cudaMemcpyDeviceToHost, cx.st));
  PEPS_CUDA(cudaStreamSynchronize(cx.st));
  if (final_loss_host) *final_loss_host = h / tail;
}

void closure_apply(Ctx& cx, int D, const float* pred, double* const* host_targets, long long n) {
  if (n == 0) return;
  auto* dev = static_cast<double* const*>(stage(cx, host_targets, sizeof(double*) * n));
  Launch l(K_AUX, cx.st);
  k_apply<<<unsigned((n + 127) / 128), 128, 0, cx.st>>>(pred, dev, n, D);
  PEPS_CHECK_LAUNCH();
}

}  // namespace peps
