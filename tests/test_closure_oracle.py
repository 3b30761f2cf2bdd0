"""Pins for the FP64 closure oracle: its gradient against central finite
differences, its output map at zero network output (the CU_0 matrix), and the
rank-1 boundary fit on an exact product boundary and as a stationary point."""
import numpy as np
import pytest

from oracle import closure_oracle as C


def _setup(n=6, d=2, D=3, W=16, seed=0):
    rng = np.random.default_rng(seed)
    F = d * D ** 4 + 2 * D * D
    X = rng.normal(size=(n, F))
    for i in range(n):                       # last D^2 features: a lower-triangular L0
        L0 = np.tril(rng.normal(size=(D, D))) + 2 * np.eye(D)
        X[i, F - D * D:] = L0.ravel()
    lab = rng.normal(size=(n, D, D))
    lab = lab @ lab.transpose(0, 2, 1)
    lab /= np.linalg.norm(lab, axis=(1, 2))[:, None, None]
    w = rng.normal(size=C.param_count(F, W, D * D)) * 0.1
    return w, X, lab.reshape(n, -1), F, W, D


def test_gradient_matches_central_differences():
    w, X, lab, F, W, D = _setup()
    loss, g = C.loss_grad(w, X, lab, F, W, D)
    rng = np.random.default_rng(1)
    idx = rng.choice(w.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (C.loss_grad(wp, X, lab, F, W, D)[0] - C.loss_grad(wm, X, lab, F, W, D)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_zero_output_layer_reproduces_the_cu0_matrix():
    w, X, lab, F, W, D = _setup()
    W1, b1, W2, b2, W3, b3 = C.unpack(w, F, W, D * D)
    W3[:] = 0.0
    b3[:] = 0.0
    sig, _ = C.forward(w, X, F, W, D)
    for i in range(X.shape[0]):
        L0 = X[i, F - D * D:].reshape(D, D)
        s0 = L0 @ L0.T
        assert np.allclose(sig[i], s0 / np.linalg.norm(s0), atol=1e-14)
        assert np.linalg.eigvalsh(sig[i]).min() > -1e-14


def test_rank1_fit_recovers_a_product_boundary():
    rng = np.random.default_rng(3)
    mats = []
    for _ in range(5):
        a = rng.normal(size=(3, 3))
        s = a @ a.T
        mats.append(s / np.linalg.norm(s))
    T = [m[None, :, :, None] * 2.5 for m in mats]
    fit = C.rank1_fit(T)
    for a, b in zip(fit, mats):
        assert np.max(np.abs(a - b)) < 1e-12


def test_rank1_fit_is_stationary_on_a_general_boundary():
    rng = np.random.default_rng(4)
    dims = [1, 3, 4, 3, 1]
    T = [rng.normal(size=(dims[i], 2, 2, dims[i + 1])) for i in range(4)]
    sig = C.rank1_fit(T)
    # dense boundary vector over (u0 v0 u1 v1 ...) and the overlap gradient
    full = T[0]
    for M in T[1:]:
        full = np.tensordot(full, M, axes=([full.ndim - 1], [0]))
    full = full[0, ..., 0]                   # end bonds have dimension 1
    for x in range(4):
        g = full
        for y in reversed(range(4)):
            if y == x:
                continue
            g = np.tensordot(g, sig[y], axes=([2 * y, 2 * y + 1], [0, 1]))
        g = g / np.linalg.norm(g)
        if np.trace(g) < 0:
            g = -g
        assert np.max(np.abs(g - sig[x])) < 1e-9
