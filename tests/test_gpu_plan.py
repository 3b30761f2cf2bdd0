"""Recorded plans (CUDA graphs): a replay computes what the plain call computes.

A plan is recorded once for a device lattice and replayed; the tensors are
overwritten in place between replays.  Each replay is compared with the FP64
oracle on the tensors it saw (1e-10, as the plain FP64 path) and with the plain
call on the same tensors (1e-12: same kernels, same inputs).
"""
import numpy as np
import pytest

from oracle import peps_oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-10
SAME = 1e-12


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


def _obs(env, kinds=("site", "hbond", "vbond")):
    out = {}
    for kind, op in (("site", O.SZ), ("site", O.SX), ("hbond", O.SDOTS), ("vbond", O.SDOTS)):
        if kind in kinds:
            out[(kind, id(op))] = env.expect(kind, op)
    return out


def _oracle_obs(oenv, kinds=("site", "hbond", "vbond")):
    out = {}
    for kind, op in (("site", O.SZ), ("site", O.SX), ("hbond", O.SDOTS), ("vbond", O.SDOTS)):
        if kind in kinds:
            out[(kind, id(op))] = O.expect_all(oenv, kind, op)
    return out


def _close(a, b, tol):
    for k in a:
        assert _rel(a[k], b[k]) < tol, (k, _rel(a[k], b[k]))


@pytest.mark.parametrize("mode,chi", [("svd", 16), ("var", 8)])
def test_full_plan_replays_match_oracle_after_in_place_update(peps, mode, chi):
    import torch
    from paper_1311_6696_gb300 import synth
    A1 = synth.peps_gauss(5, 5, 2, 2, seed=61)
    A2 = synth.peps_gauss(5, 5, 2, 2, seed=62)
    At = torch.from_numpy(A1).cuda()
    plan = peps.Plan(At, chi=chi, mode=mode, seed=3)
    assert plan.launches > 0
    for A in (A1, A2, A1):
        At.copy_(torch.from_numpy(A))
        env = plan.run()
        oenv = O.env_full(A, chi=chi, mode=mode, seed=3)
        _close(_obs(env), _oracle_obs(oenv), TOL)
        ln, sg = env.ln_norm()
        assert abs(ln - oenv["ln_norm"]) < TOL and sg == oenv["sign"]
        _close(_obs(env), _obs(peps.env_full(At, chi=chi, mode=mode, seed=3)), SAME)


def test_full_plan_tensor_core_path_equals_plain_call(peps):
    import torch
    from paper_1311_6696_gb300 import synth
    A = torch.from_numpy(synth.workload("10x10_D4")).cuda()
    plan = peps.Plan(A, chi=16, mode="var", precision="tf32x3")
    env = plan.run()
    _close(_obs(env), _obs(peps.env_full(A, chi=16, mode="var", precision="tf32x3")), SAME)


@pytest.mark.parametrize("n", [2, 3])
def test_cluster_plan_matches_oracle(peps, n):
    import torch
    from paper_1311_6696_gb300 import synth
    A1 = synth.peps_gauss(5, 5, 2, 2, seed=70 + n)
    A2 = synth.peps_gauss(5, 5, 2, 2, seed=80 + n)
    At = torch.from_numpy(A1).cuda()
    plan = peps.Plan(At, chi=6, mode="var", cluster_n=n)
    for A in (A1, A2):
        At.copy_(torch.from_numpy(A))
        env = plan.run()
        _close(_obs(env), _oracle_obs(O.env_cluster(A, n=n, chi=6, mode="var")), TOL)


def test_plan_needs_device_lattice(peps):
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(3, 3, 2, 2, seed=1)
    inp = peps._Input(A)
    o = peps._opts(4, "svd", 2, "fp64", 1, 0)
    import ctypes as C
    h = C.c_void_p()
    rc = peps.lib.peps_plan_create(C.byref(inp.lat), C.byref(o), 0, C.byref(h), None)
    assert rc == peps.EINVAL and not h.value


def test_plan_rejects_obc_violation(peps):
    import torch
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(3, 3, 2, 2, seed=1)
    A[0, 0, 0, 1, 0, 0, 0] = 0.5
    with pytest.raises(peps.PepsError) as e:
        peps.Plan(torch.from_numpy(A).cuda(), chi=4)
    assert e.value.code == peps.EINVAL


def test_tuned_plan_matches_oracle(peps):
    """The autotuner's choice changes only the launch configuration."""
    import torch
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(5, 5, 2, 2, seed=91)
    At = torch.from_numpy(A).cuda()
    plan = peps.Plan(At, chi=8, mode="var", seed=3, tune=True)
    assert plan.lanes in (2, 4, 8) and plan.qr_cluster in (4, 8, 16)
    env = plan.run()
    _close(_obs(env), _oracle_obs(O.env_full(A, chi=8, mode="var", seed=3)), TOL)


def test_tuned_cluster_plan_matches_oracle(peps):
    """Tuning a cluster plan (lanes, windows per batch, QR cluster cap) keeps the results."""
    import torch
    from paper_1311_6696_gb300 import synth
    A = synth.peps_gauss(6, 6, 2, 2, seed=93)
    At = torch.from_numpy(A).cuda()
    plan = peps.Plan(At, chi=6, mode="var", cluster_n=3, tune=True)
    env = plan.run()
    _close(_obs(env), _oracle_obs(O.env_cluster(A, n=3, chi=6, mode="var")), TOL)


@pytest.mark.parametrize("precision,cluster_n", [("fp64", 0), ("tf32x3", 0), ("tf32x3", 3)])
def test_profiler_counts_every_kernel_of_a_replay(peps, precision, cluster_n):
    """One replay adds to the per-class launch counters exactly the kernel
    nodes of the recorded graph: every kernel is counted once."""
    import torch
    from paper_1311_6696_gb300 import synth
    A = torch.from_numpy(synth.peps_gauss(6, 6, 2, 3, seed=95)).cuda()
    kw = dict(chi=12, mode="var", precision=precision)
    if cluster_n:
        kw["cluster_n"] = cluster_n
    plan = peps.Plan(A, **kw)
    assert plan.launches > 0
    torch.cuda.synchronize()
    peps.profile_reset()
    plan.run()
    torch.cuda.synchronize()
    counted = sum(v["launches"] for v in peps.profile_read().values())
    assert counted == plan.launches
