"""FP64 oracle for the learned cluster closure.

TEST INFRASTRUCTURE ONLY (see the oracle package header).

The closure replaces the CU_0 matrix on one outward leg of a cluster window
(Section 5.1, 5.2) by a positive matrix predicted from local data.  The paper
has no learned part; this is the build's reading of it:

* label at (direction, cut, column): the site matrix of the best D'=1 product
  approximation of the full boundary at that cut (rank-1 ALS on the boundary
  MPS: each update is the boundary contracted with every other matrix,
  scaled to unit Frobenius norm, positive trace);
* features: the site tensor just above the cut (dense, d*D^4, zero-padded),
  the CU_0 matrix there (D^2) and its lower Cholesky factor L0 (D^2);
* network: three layers, width W, ReLU; output Y (D x D); X = L0 + Y;
  sigma = X X^T / ||X X^T||_F (so sigma is positive and equals the CU_0
  matrix when Y = 0);
* loss: mean over the batch of ||sigma - label||_F^2.

Weight layout (flat): W1[W][F], b1[W], W2[W][W], b2[W], W3[D^2][W], b3[D^2].
"""
from __future__ import annotations

import numpy as np


def param_count(F: int, W: int, out: int) -> int:
    return W * F + W + W * W + W + out * W + out


def unpack(w, F, W, out):
    o = 0
    W1 = w[o:o + W * F].reshape(W, F); o += W * F
    b1 = w[o:o + W]; o += W
    W2 = w[o:o + W * W].reshape(W, W); o += W * W
    b2 = w[o:o + W]; o += W
    W3 = w[o:o + out * W].reshape(out, W); o += out * W
    b3 = w[o:o + out]
    return W1, b1, W2, b2, W3, b3


def forward(w, X, F, W, D):
    """sigma predictions (n, D, D) and the activations needed for backward."""
    out = D * D
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(w, dtype=np.float64), F, W, out)
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ W1.T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2.T + b2
    H2 = np.maximum(Z2, 0.0)
    Yo = H2 @ W3.T + b3
    L0 = X[:, F - out:].reshape(-1, D, D)
    Xm = L0 + Yo.reshape(-1, D, D)
    S = Xm @ Xm.transpose(0, 2, 1)
    nrm = np.sqrt(np.sum(S * S, axis=(1, 2)))
    sig = S / nrm[:, None, None]
    return sig, (X, Z1, H1, Z2, H2, Xm, S, nrm)


def loss_grad(w, X, Yl, F, W, D):
    """(loss, gradient w.r.t. the flat weights) in FP64."""
    out = D * D
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(w, dtype=np.float64), F, W, out)
    sig, (Xin, Z1, H1, Z2, H2, Xm, S, nrm) = forward(w, X, F, W, D)
    n = Xin.shape[0]
    lab = np.asarray(Yl, dtype=np.float64).reshape(n, D, D)
    diff = sig - lab
    loss = float(np.sum(diff * diff) / n)
    G = 2.0 * diff / n                                   # dL/dsigma
    dS = (G - sig * np.sum(G * sig, axis=(1, 2))[:, None, None]) / nrm[:, None, None]
    dX = (dS + dS.transpose(0, 2, 1)) @ Xm               # d(X X^T) -> dX
    dYo = dX.reshape(n, out)
    gW3 = dYo.T @ H2
    gb3 = dYo.sum(axis=0)
    dH2 = (dYo @ W3) * (Z2 > 0)
    gW2 = dH2.T @ H1
    gb2 = dH2.sum(axis=0)
    dH1 = (dH2 @ W2) * (Z1 > 0)
    gW1 = dH1.T @ Xin
    gb1 = dH1.sum(axis=0)
    return loss, np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def rank1_fit(T, tol: float = 1e-12, max_half: int = 200):
    """Best product (D'=1) approximation of a boundary MPS T (list of
    M[a,u,v,b]): list of unit-Frobenius matrices sigma_x[u,v]."""
    L = len(T)
    sig = [np.eye(M.shape[1]) / np.sqrt(M.shape[1]) for M in T]

    def site_vec(M, s):
        return np.einsum("auvb,uv->ab", M, s)

    for h in range(max_half):
        r = [None] * L
        r[L - 1] = np.ones(T[L - 1].shape[3])
        for x in range(L - 1, 0, -1):
            v = site_vec(T[x], sig[x]) @ r[x]
            r[x - 1] = v / np.linalg.norm(v)
        lv = np.ones(T[0].shape[0])
        change = 0.0
        for x in range(L):
            b = np.einsum("a,auvb,b->uv", lv, T[x], r[x])
            b = b / np.linalg.norm(b)
            if np.trace(b) < 0:
                b = -b
            change = max(change, float(np.linalg.norm(b - sig[x])))
            sig[x] = b
            if x < L - 1:
                v = lv @ site_vec(T[x], sig[x])
                lv = v / np.linalg.norm(v)
        if change < tol:
            break
    return sig
