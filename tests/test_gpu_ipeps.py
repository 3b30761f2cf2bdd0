"""Infinite PEPS by the cluster update (Section 5.4) on the GPU against the
FP64 oracle: the four infinite separable boundaries and the density matrices
of an n x n cluster of copies."""
import numpy as np
import pytest

from oracle import peps_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def peps():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1311_6696_gb300 import peps as P
    return P


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-2)))


def _tensor(D, seed):
    from paper_1311_6696_gb300 import synth
    return synth.peps_gauss(3, 3, 2, D, seed=seed)[1, 1].copy()


@pytest.mark.parametrize("D,n,chi", [(2, 1, 4), (2, 3, 8), (3, 4, 9), (3, 5, 6)])
def test_ipeps_cluster_fp64_matches_the_oracle(peps, D, n, chi):
    A = _tensor(D, 20 + D + n)
    g = peps.ipeps_cluster(A, n=n, chi=chi, mode="var")
    r = O.ipeps_cluster(A, n, chi)
    for k in range(4):
        assert np.max(np.abs(g["sigma"][k] - r["sigma"][k])) < 1e-12, k
    gs = g["rho_site"] / np.trace(g["rho_site"])
    assert _rel(gs, r["rho_site"] / np.trace(r["rho_site"])) < 1e-10
    if n > 1:
        for key in ("rho_h", "rho_v"):
            gm = g[key] / np.trace(g[key])
            rm = r[key].reshape(4, 4)
            assert _rel(gm, rm / np.trace(rm)) < 1e-10, key


def test_ipeps_cluster_tensor_cores_and_device_input(peps):
    import torch
    A = _tensor(3, 31)
    g = peps.ipeps_cluster(torch.from_numpy(A).cuda(), n=4, chi=9, mode="var", precision="tf32x3")
    r = O.ipeps_cluster(A, 4, 9)
    assert _rel(O.expect(g["rho_site"], O.SZ), O.expect(r["rho_site"], O.SZ)) < 1e-4
    for key in ("rho_h", "rho_v"):
        assert _rel(O.expect(g[key], O.SDOTS), O.expect(r[key], O.SDOTS)) < 1e-4


def test_ipeps_boundary_that_never_settles_is_econverge(peps):
    """A zero-mean random tensor has no settling separable boundary here: the
    bounded iteration reports PEPS_ECONVERGE (the oracle raises too)."""
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(3, 3, 2, 2, seed=3, mean=0.0, std=1.0)[1, 1].copy()
    with pytest.raises(O.OracleNotConverged):
        O.cu0_infinite(A, max_iter=5000)
    with pytest.raises(peps.PepsError) as e:
        peps.ipeps_cluster(A, n=2, chi=4)
    assert e.value.code == peps.ECONVERGE
