// Learned cluster closure: labels, features and the MLP (training and inference).
#pragma once
#include "ein.cuh"

namespace peps {

// Network shape: F inputs (site tensor d D^4, CU_0 matrix D^2, its Cholesky
// factor D^2), width W, D^2 outputs.
struct MlpDims {
  int d = 2, D = 2, W = 256;
  int F() const { return d * D * D * D * D + 2 * D * D; }
  int out() const { return D * D; }
  long long params() const {
    const long long f = F(), w = W, o = out();
    return w * f + w + w * w + w + o * w + o;
  }
};

// One rim position: the site above the cut and the CU_0 matrix at it.
struct RimSite {
  const double* A;        // site tensor, effective dims contiguous
  int du, dl, dn, dr;
  const double* sigma;    // D x D CU_0 matrix (row-major)
};

// X[e] = [dense site tensor | sigma | chol(sigma)] for every rim position.
void closure_features(Ctx& cx, const MlpDims& m, const RimSite* host_sites, long long n, float* X);

// One boundary MPS (the cut) whose best product approximation is fitted.
struct Rank1Job {
  const double* const* sites;   // device array of L site tensors M[a][u][v][b]
  const int* bonds;             // device array of L+1 bond dims
  int L;
  float* out;                   // L x D^2 labels
};
void rank1_labels(Ctx& cx, int D, int maxchi, int maxL, const Rank1Job* host_jobs, int njobs);

void mlp_init(Ctx& cx, const MlpDims& m, float* w, unsigned long long seed);
void mlp_predict(Ctx& cx, const MlpDims& m, const float* w, const float* X, long long n, float* sigma);
void mlp_loss_grad(Ctx& cx, const MlpDims& m, const float* w, const float* X, const float* Y, long long n,
                   double* loss_dev, float* grad);
// m1_ext / m2_ext: caller-owned AdamW moments (else zeroed state of this call
// only); t0: steps already taken with them (bias correction and the position
// in the seeded minibatch stream continue from there).
void mlp_train(Ctx& cx, const MlpDims& m, float* w, const float* X, const float* Y, long long n, int steps,
               int batch, float lr, float wd, unsigned long long seed, double* final_loss_host,
               float* m1_ext = nullptr, float* m2_ext = nullptr, long long t0 = 0);

// Replace sigma[e] by pred[e] where pred is finite with positive trace (else keep).
void closure_apply(Ctx& cx, int D, const float* pred, double* const* host_targets, long long n);

}  // namespace peps
