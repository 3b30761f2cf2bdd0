// FP64 factorizations used to gauge and truncate boundary MPS.
#pragma once
#include "ein.cuh"

namespace peps {

// Device status word values (Ctx::flag).
constexpr int FLAG_SVD_NOCONV = 1;
constexpr int FLAG_CU0_NOCONV = 2;
constexpr int FLAG_BAD_VALUE = 4;
constexpr int FLAG_TIMEOUT = 8;

// Thin QR of the m x n matrix with element (i,j) at A[i*rs + j*cs].
// Writes Q (m x k, k = min(m,n)) to Q[i*qrs + j*qcs] and, if R is not null,
// R (k x n) row-major.  Householder reflections (beta = -sign(alpha)*norm).
void qr_thin(Ctx& cx, int m, int n, const double* A, long long rs, long long cs, double* Q,
             long long qrs, long long qcs, double* R);

// Truncated SVD of the row-major m x n matrix A: writes US = U[:, :kk] * S[:kk]
// (m x kk, row-major) and Vt = V^T[:kk, :] (kk x n, row-major), singular values
// in decreasing order.  One-sided Jacobi (Hestenes) on the narrower side.
void svd_trunc(Ctx& cx, int m, int n, const double* A, int kk, double* US, double* Vt);

}  // namespace peps
