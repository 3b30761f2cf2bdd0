"""Checkpoint and resume: environment handles and closure-network training
state survive a round trip through a file, a training run split over calls
equals one run, and malformed files are rejected."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import peps_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1311_6696_gb300 import peps
    return torch, peps


@pytest.mark.parametrize("cluster", [False, True])
def test_environment_round_trip(env, tmp_path, cluster):
    torch, peps = env
    from paper_1311_6696_gb300 import synth
    A = synth.peps_simple_update(4, 5, 2, seed=3, steps=40)
    e = peps.env_cluster(A, n=2, chi=8, mode="var") if cluster else peps.env_full(A, chi=16, mode="var")
    path = str(tmp_path / "env.peps")
    peps.env_save(e, path)
    g = peps.env_load(path)
    for kind, op in (("site", O.SZ), ("hbond", O.SDOTS), ("vbond", O.SDOTS)):
        assert np.array_equal(e.expect(kind, op), g.expect(kind, op)), kind
        assert np.array_equal(e.rho(kind), g.rho(kind)), kind
    if not cluster:
        assert e.ln_norm() == g.ln_norm()


def test_training_split_over_calls_and_a_checkpoint_equals_one_run(env, tmp_path):
    torch, peps = env
    from paper_1311_6696_gb300 import synth
    D = 2
    X, Y = peps.closure_data(synth.peps_simple_update(5, 5, D, seed=300, steps=60), chi=16, mode="svd")
    w0 = peps.mlp_init(2, D, peps.CLOSURE_WIDTH, seed=4)
    # one run of 60 steps, with the stateless call and with caller-held state
    w_a = w0.clone()
    peps.mlp_train(w_a, X, Y, 2, D, steps=60, batch=64, lr=1e-3, seed=9)
    w_b = w0.clone()
    st_b = peps.AdamState(w_b)
    peps.mlp_train_state(w_b, st_b, X, Y, 2, D, steps=60, batch=64, lr=1e-3, seed=9)
    assert torch.equal(w_a, w_b) and st_b.step == 60
    # 20 steps, a checkpoint, a fresh process state, 40 more
    w_c = w0.clone()
    st_c = peps.AdamState(w_c)
    peps.mlp_train_state(w_c, st_c, X, Y, 2, D, steps=20, batch=64, lr=1e-3, seed=9)
    path = str(tmp_path / "mlp.peps")
    peps.mlp_save(path, w_c, 2, D, state=st_c)
    w_d = torch.zeros_like(w0)
    st_d = peps.AdamState(w_d)
    peps.mlp_load(path, w_d, 2, D, state=st_d)
    assert st_d.step == 20 and torch.equal(w_d, w_c)
    peps.mlp_train_state(w_d, st_d, X, Y, 2, D, steps=40, batch=64, lr=1e-3, seed=9)
    assert torch.equal(w_d, w_b) and st_d.step == 60
    # weights alone: no optimizer state in the file, zero moments on load
    peps.mlp_save(path, w_d, 2, D)
    st_e = peps.AdamState(w_d)
    st_e.m += 1.0
    peps.mlp_load(path, w_d, 2, D, state=st_e)
    assert st_e.step == 0 and float(st_e.m.abs().max()) == 0.0


def test_malformed_checkpoints_are_rejected(env, tmp_path):
    torch, peps = env
    from paper_1311_6696_gb300 import synth
    e = peps.env_full(synth.peps_gauss(3, 3, 2, 2, 1), chi=8)
    good = str(tmp_path / "env.peps")
    peps.env_save(e, good)
    w = peps.mlp_init(2, 2, peps.CLOSURE_WIDTH, seed=1)
    mlp = str(tmp_path / "mlp.peps")
    peps.mlp_save(mlp, w, 2, 2)
    with pytest.raises(peps.PepsError):
        peps.env_load(mlp)                                  # another format
    with pytest.raises(peps.PepsError):
        peps.mlp_load(mlp, torch.zeros(peps.mlp_param_count(2, 3, peps.CLOSURE_WIDTH), device="cuda"), 2, 3)
    short = str(tmp_path / "short.peps")
    with open(good, "rb") as f, open(short, "wb") as g:
        g.write(f.read()[:-8])                              # truncated body
    with pytest.raises(peps.PepsError):
        peps.env_load(short)
    with pytest.raises(peps.PepsError):
        peps.env_load(str(tmp_path / "missing.peps"))
    # the context is still usable
    assert np.isfinite(peps.env_load(good).expect("site", O.SZ)).all()
