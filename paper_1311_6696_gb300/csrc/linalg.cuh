// FP64 factorizations used to gauge and truncate boundary MPS.
#pragma once
#include "ein.cuh"

namespace peps {

// Device status word values (Ctx::flag).
constexpr int FLAG_SVD_NOCONV = 1;
constexpr int FLAG_CU0_NOCONV = 2;
constexpr int FLAG_BAD_VALUE = 4;
constexpr int FLAG_TIMEOUT = 8;

// Thin QR of the m x n matrix with element (i,j) at A[i*rs + j*cs], for each
// problem of the pointer sets.  Writes Q (m x k, k = min(m,n)) to
// Q[i*qrs + j*qcs] and, if R is present, R (k x n) row-major.  Householder
// reflections (beta = -sign(alpha)*norm).  A may alias Q.
void qr_thin(Ctx& cx, int m, int n, const TP& A, long long rs, long long cs, const TP& Q,
             long long qrs, long long qcs, const TP& R);

// Truncated SVD of the row-major m x n matrix A: writes US = U[:, :kk] * S[:kk]
// (m x kk, row-major) and Vt = V^T[:kk, :] (kk x n, row-major), singular values
// in decreasing order.  One-sided Jacobi (Hestenes) on the narrower side.
void svd_trunc(Ctx& cx, int m, int n, const TP& A, int kk, const TP& US, const TP& Vt);

}  // namespace peps
