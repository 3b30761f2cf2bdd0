"""The operation count behind bench.py's CPU baseline (set_cost_model)
against the oracle's own call structure: every absorb chain and open site the
oracle runs for one environment set of a lattice whose every absorb
truncates, counted by wrapping the oracle's chain functions."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


@pytest.mark.parametrize("L", [4, 5])
def test_set_cost_model_counts_the_oracles_steps(monkeypatch, L):
    import bench
    from oracle import peps_oracle as O
    from paper_1311_6696_gb300 import synth
    calls = {"chain": 0, "open": 0}
    chain_left, chain_right, open_site = O.chain_left, O.chain_right, O._open_site

    def cl(*a):
        calls["chain"] += 1
        return chain_left(*a)

    def cr(*a):
        calls["chain"] += 1
        return chain_right(*a)

    def op(*a):
        calls["open"] += 1
        return open_site(*a)

    monkeypatch.setattr(O, "chain_left", cl)
    monkeypatch.setattr(O, "chain_right", cr)
    monkeypatch.setattr(O, "_open_site", op)
    A = synth.peps_gauss(L, L, 2, 2, seed=3, mean=0.0, std=1.0)
    O.env_full(A, chi=2, mode="var")      # chi = 2 < D^2: every absorb is a variational fit
    # one unit of t_step per chain call and of t_open per open site, minus the
    # norm's closing row (L chain calls), which the model leaves out
    model = bench.set_cost_model(L, 1.0, 0.0)
    assert calls["chain"] - L == model
    # open sites: the model's L per pass; the oracle opens every site once and
    # every bond's left site again
    assert bench.set_cost_model(L, 0.0, 1.0) == 2 * L * L
    assert calls["open"] == 2 * L * L + 2 * L * (L - 1)
