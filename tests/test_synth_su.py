"""The simple-update input generator against the paper's Table 2 (Appendix A),
evaluated by exact (brute-force) contraction of the generated 4x4 states."""
import os

import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import peps_oracle as O
from paper_1311_6696_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "su_heisenberg_4x4_table2.txt")


def _rows():
    out = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            t = line.split()
            out.append((int(t[1]), float(t[3]), float(t[5])))
    return out


@pytest.mark.parametrize("D,e_paper,tol", _rows())
def test_su_energy_matches_table2(D, e_paper, tol):
    A = synth.peps_simple_update(4, 4, D, seed=3, tau=0.01, steps=400)
    psi = BF.state_vector(BF.dense_lattice(A))
    dims = [2] * 16
    bonds = [(y * 4 + x, y * 4 + x + 1) for y in range(4) for x in range(3)] + \
            [(y * 4 + x, (y + 1) * 4 + x) for y in range(3) for x in range(4)]
    e = sum(BF.expect_bond(psi, dims, i, j, O.SDOTS) for i, j in bonds) / 16
    assert abs(e - e_paper) < tol, e
    assert e > -0.57432544      # variational bound: above the exact ground state (Appendix A)


def test_su_state_respects_obc_and_norm():
    A = synth.peps_simple_update(3, 5, 3, seed=9, steps=20)
    for y in range(3):
        for x in range(5):
            du, dl, dd, dr = synth.site_dims(3, 5, y, x, 3)
            m = np.ones(A[y, x].shape, dtype=bool)
            m[:, :du, :dl, :dd, :dr] = False
            assert np.count_nonzero(A[y, x][m]) == 0
            assert abs(np.linalg.norm(A[y, x]) - 1.0) < 1e-12
