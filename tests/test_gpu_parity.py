"""GPU parity: the CUDA path against the FP64 oracle, element by element.

Tolerance (FP64 path): 1e-10 on the relative error |x - x_ref| / max(|x_ref|, 1e-2)
of every expectation value and every normalised density-matrix entry, and 1e-10
absolute on ln|<psi|psi>| (relative on the norm itself).
"""
import numpy as np
import pytest

from oracle import peps_oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def peps():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1311_6696_gb300 import peps as P
    return P


def _rel(a, b):
    a = np.asarray(a, dtype=float)
    b = np.asarray(b, dtype=float)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-2))) if a.size else 0.0


def _oracle_rhos(env, kind):
    key = {"site": "rho_site", "hbond": "rho_h", "vbond": "rho_v"}[kind]
    out = []
    for row in env[key]:
        for r in row:
            k = int(round(np.sqrt(r.size)))
            m = r.reshape(k, k)
            out.append(m / np.trace(m))
    return np.array(out)


def _compare(genv, oenv, with_norm=True, tol=TOL, kinds=("site", "hbond", "vbond")):
    for kind in kinds:
        g = genv.rho(kind)
        if g.size == 0:
            continue
        g = g / np.trace(g, axis1=1, axis2=2)[:, None, None]
        assert _rel(g, _oracle_rhos(oenv, kind)) < tol, kind
    for kind, op in (("site", O.SZ), ("site", O.SX), ("hbond", O.SDOTS), ("vbond", O.SDOTS)):
        if kind not in kinds:
            continue
        assert _rel(genv.expect(kind, op), O.expect_all(oenv, kind, op)) < tol, kind
    if with_norm:
        ln, sg = genv.ln_norm()
        assert abs(ln - oenv["ln_norm"]) < tol and sg == oenv["sign"]


@pytest.mark.parametrize("mode", ["svd", "var"])
def test_4x4_D2_exact(peps, mode):
    from paper_1311_6696_gb300 import synth
    A = synth.workload("4x4_D2")
    _compare(peps.env_full(A, chi=16, mode=mode), O.env_full(A, chi=16, mode=mode))


@pytest.mark.parametrize("shape,D,chi,mode", [((4, 5), 2, 16, "svd"), ((3, 3), 3, 9, "svd"),
                                              ((5, 4), 2, 5, "svd"), ((5, 6), 2, 6, "var"),
                                              ((6, 6), 3, 8, "var"), ((3, 7), 3, 7, "var")])
def test_full_env_parity(peps, shape, D, chi, mode):
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(shape[0], shape[1], 2, D, seed=100 + D + chi)
    _compare(peps.env_full(A, chi=chi, mode=mode, seed=7), O.env_full(A, chi=chi, mode=mode, seed=7))


def test_var_three_half_sweeps(peps):
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(5, 5, 2, 3, seed=31)
    _compare(peps.env_full(A, chi=6, mode="var", sweeps=3, seed=3),
             O.env_full(A, chi=6, mode="var", sweeps=3, seed=3))


def test_10x10_D4_chi16_var(peps):
    """The 10x10 D=4 workload at its smallest chi, compared everywhere."""
    from paper_1311_6696_gb300 import synth
    A = synth.workload("10x10_D4")
    _compare(peps.env_full(A, chi=16, mode="var"), O.env_full(A, chi=16, mode="var"))


def test_f32_input_matches_f64_of_same_values(peps):
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(4, 4, 2, 2, seed=5).astype(np.float32)
    _compare(peps.env_full(A, chi=8, mode="var"), O.env_full(A.astype(np.float64), chi=8, mode="var"))


def test_device_input(peps):
    import torch
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(4, 4, 2, 2, seed=6)
    At = torch.from_numpy(A).cuda()
    _compare(peps.env_full(At, chi=8, mode="svd"), O.env_full(A, chi=8, mode="svd"))


def test_product_state(peps):
    from paper_1311_6696_gb300 import synth
    A = synth.peps_product(3, 4, 2, seed=5)
    _compare(peps.env_full(A, chi=4, mode="var"), O.env_full(A, chi=4, mode="var"))


def test_norm_call(peps):
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(6, 5, 2, 3, seed=9)
    for mode in ("svd", "var"):
        ln, sg = peps.norm(A, chi=7, mode=mode)
        lo, so = O.norm(A, chi=7, mode=mode)
        assert abs(ln - lo) < TOL and sg == so


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_cluster_parity(peps, n):
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(5, 5, 2, 2, seed=40 + n)
    kinds = ("site",) if n == 1 else ("site", "hbond", "vbond")   # n = 1 windows hold no bond
    _compare(peps.env_cluster(A, n=n, chi=6, mode="var"),
             O.env_cluster(A, n=n, chi=6, mode="var"), with_norm=False, kinds=kinds)


def test_cluster_covering_lattice_equals_full_on_gpu(peps):
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(4, 4, 2, 2, seed=7)
    f = peps.env_full(A, chi=6, mode="var")
    c = peps.env_cluster(A, n=8, chi=6, mode="var")
    for kind in ("site", "hbond", "vbond"):
        np.testing.assert_array_equal(f.rho(kind), c.rho(kind))


def test_obc_violation_is_einval(peps):
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(3, 3, 2, 2, seed=1)
    A[0, 0, 0, 1, 0, 0, 0] = 0.5          # up leg of the top row must be index 0 only
    with pytest.raises(peps.PepsError) as e:
        peps.env_full(A, chi=4)
    assert e.value.code == peps.EINVAL


def test_bad_args_are_einval(peps):
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(3, 3, 2, 2, seed=1)
    for kw in (dict(chi=0), dict(chi=4, mode=7), dict(chi=4, precision=9)):
        with pytest.raises(peps.PepsError) as e:
            peps.env_full(A, **kw)
        assert e.value.code == peps.EINVAL
    with pytest.raises(peps.PepsError) as e:
        peps.env_cluster(A, n=0, chi=4)
    assert e.value.code == peps.EINVAL


def test_cluster_svd_mode_parity(peps):
    """svd compression inside batched windows (batched QR sweep + Jacobi SVD)."""
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(5, 5, 2, 2, seed=57)
    _compare(peps.env_cluster(A, n=2, chi=4, mode="svd"),
             O.env_cluster(A, n=2, chi=4, mode="svd"), with_norm=False)


def test_cluster_large_batched_group(peps):
    """8x8 lattice, n=3: 36 interior windows share one shape and run as one batch."""
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(8, 8, 2, 2, seed=58)
    _compare(peps.env_cluster(A, n=3, chi=6, mode="var", seed=4),
             O.env_cluster(A, n=3, chi=6, mode="var", seed=4), with_norm=False)
