"""Failure detection without faulting the GPU: every error path is forced
from the host (PEPS_FAULT, iteration caps) or by a bounded wait that is
certain to run out, and each test checks the status code and that the next
plain call on the same context still succeeds."""
import os

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


@pytest.fixture()
def lattice():
    from paper_1311_6696_gb300 import synth
    return synth.peps_gauss(4, 4, 2, 2, seed=61)


def _still_works(peps, A):
    e = peps.env_full(A, chi=6, mode="var")
    ref = O.env_full(A, chi=6, mode="var")
    assert np.max(np.abs(e.expect("site", O.SZ) - np.array(O.expect_all(ref, "site", O.SZ)))) < 1e-10


@pytest.fixture()
def fault(monkeypatch):
    def set_(mode):
        monkeypatch.setenv("PEPS_FAULT", mode)
    yield set_
    os.environ.pop("PEPS_FAULT", None)


def test_injected_allocation_failure_is_enomem(peps, lattice, fault):
    fault("alloc")
    for call in (lambda: peps.env_full(lattice, chi=6, mode="var"),
                 lambda: peps.env_cluster(lattice, n=2, chi=6, mode="var"),
                 lambda: peps.norm(lattice, chi=6, mode="var")):
        with pytest.raises(peps.PepsError) as e:
            call()
        assert e.value.code == peps.ENOMEM and "PEPS_FAULT=alloc" in str(e.value)
    os.environ.pop("PEPS_FAULT")
    _still_works(peps, lattice)


@pytest.mark.parametrize("on_device", [False, True])
def test_injected_nan_is_einval_and_leaves_the_input_alone(peps, lattice, fault, on_device):
    import torch
    A = torch.from_numpy(lattice).cuda() if on_device else lattice.copy()
    fault("nan")
    with pytest.raises(peps.PepsError) as e:
        peps.env_full(A, chi=6, mode="var")
    assert e.value.code == peps.EINVAL and "non-finite" in str(e.value)
    got = A.cpu().numpy() if on_device else A
    assert np.array_equal(got, lattice)                 # planted in the library's own copy
    os.environ.pop("PEPS_FAULT")
    _still_works(peps, lattice)


def test_nonfinite_input_is_einval(peps, lattice):
    A = lattice.copy()
    A[1, 1, 0, 0, 0, 0, 0] = np.inf
    with pytest.raises(peps.PepsError) as e:
        peps.env_full(A, chi=6, mode="var")
    assert e.value.code == peps.EINVAL and "non-finite" in str(e.value)


def test_injected_convergence_failure(peps, lattice, fault):
    fault("converge")
    with pytest.raises(peps.PepsError) as e:       # CU_0 needs more than one half-sweep
        peps.env_cluster(lattice, n=2, chi=6, mode="var")
    assert e.value.code == peps.ECONVERGE
    with pytest.raises(peps.PepsError) as e:       # so does the Jacobi SVD of svd mode
        peps.env_full(lattice, chi=3, mode="svd")
    assert e.value.code == peps.ECONVERGE
    os.environ.pop("PEPS_FAULT")
    _still_works(peps, lattice)


def test_iteration_caps_force_econverge_and_restore(peps, lattice):
    try:
        peps.set_iteration_caps(cu0_half_sweeps=2)
        with pytest.raises(peps.PepsError) as e:
            peps.env_cluster(lattice, n=2, chi=6, mode="var")
        assert e.value.code == peps.ECONVERGE and "half-sweep cap" in str(e.value)
        peps.set_iteration_caps(jacobi_sweeps=1)
        with pytest.raises(peps.PepsError) as e:
            peps.env_full(lattice, chi=3, mode="svd")
        assert e.value.code == peps.ECONVERGE and "Jacobi" in str(e.value)
    finally:
        peps.set_iteration_caps(0, 0)
    c = peps.env_cluster(lattice, n=2, chi=6, mode="var")
    ref = O.env_cluster(lattice, n=2, chi=6, mode="var")
    assert np.max(np.abs(c.expect("site", O.SZ) - np.array(O.expect_all(ref, "site", O.SZ)))) < 1e-10


def test_bounded_wait_returns_etimeout(peps, lattice):
    import time
    t0 = time.perf_counter()
    with pytest.raises(peps.PepsError) as e:
        peps.wait_selftest(budget_us=20000)
    assert e.value.code == peps.ETIMEOUT
    assert time.perf_counter() - t0 < 10.0
    _still_works(peps, lattice)
