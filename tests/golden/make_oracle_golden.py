"""Writes the stored oracle results for the large workloads (test infrastructure).

Calls only the FP64 CPU oracle (``oracle/``) and the seeded input generators
(``paper_1311_6696_gb300/synth.py``); no value comes from the CUDA path.

The full environment set of the 20x20 D=8 simple-update lattice costs the
oracle hours, so what is stored is the part one top-down sweep yields
(Section 2, sandwich contraction): ln|<psi|psi>| and the last row's local
quantities -- <sigma_z> on its 20 sites and <S.S> on its 19 bonds -- which in
the full method use the top boundary above the last row and the bottom
closure, exactly as here.

Usage:  python tests/golden/make_oracle_golden.py c4 [--chi 128] [--refresh-input]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import peps_oracle as O  # noqa: E402
from paper_1311_6696_gb300 import synth  # noqa: E402


def fingerprint(A: np.ndarray) -> dict:
    """sha256 of the bytes and a weighted sum (identical generator and
    platform), and the gauge-invariant gram4 (same state on any platform)."""
    w = synth.uniform01(99, A.size).reshape(A.shape) - 0.5
    return {"sha256": hashlib.sha256(np.ascontiguousarray(A).tobytes()).hexdigest(),
            "wsum": float(np.sum(A * w)), "sum": float(np.sum(A)), "sumsq": float(np.sum(A * A)),
            "gram4": synth.gram4(A)}


def last_row_and_norm(A: np.ndarray, chi: int, mode: str = "var", sweeps: int = 2, seed: int = 0,
                      log=print) -> dict:
    lat = O.lattice_from_dense(A)
    Ly, Lx = lat.Ly, lat.Lx
    T = O.closure_mps(lat.top)
    lns = [0.0]
    t0 = time.time()
    for y in range(Ly - 1):
        T, ln = O.absorb_compress(T, lat, y, chi, mode, sweeps, seed, 0)
        lns.append(ln)
        log(f"row {y} absorbed ({time.time() - t0:.0f} s)")
    ln_norm, sign = O._norm_from_top(lat, T, lns)
    y = Ly - 1
    rs, rh = O._row_rhos(lat, T, O.closure_mps(lat.bottom), y)
    sz = [O.expect(rs[x], O.SZ) for x in range(Lx)]
    ss = [O.expect(rh[x], O.SDOTS) for x in range(Lx - 1)]
    return {"ln_norm": ln_norm, "sign": sign, "row": y, "sz": sz, "sdots_h": ss,
            "oracle_seconds": round(time.time() - t0, 1)}


WORKLOADS = {
    "c4": dict(name="20x20_D8_su", desc="20x20 OBC PEPS d=2 D=8 from the seeded simple-update Heisenberg "
                                        "generator (tau=0.01, 400 steps, seed 4)"),
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=sorted(WORKLOADS))
    ap.add_argument("--chi", type=int, default=128)
    ap.add_argument("--out", default=None)
    ap.add_argument("--refresh-input", action="store_true",
                    help="rewrite only the input fingerprint of an existing file, after checking that the "
                         "generator still gives the same bytes it was computed from")
    a = ap.parse_args()
    w = WORKLOADS[a.workload]
    A = synth.workload(w["name"])
    out = a.out or os.path.join(HERE, f"oracle_{w['name']}_chi{a.chi}.json")
    if a.refresh_input:
        res = json.load(open(out))
        fp = fingerprint(A)
        if fp["sha256"] != res["input"]["sha256"]:
            sys.exit("the generator's output changed: recompute the oracle result instead")
        res["input"] = fp
        with open(out, "w") as f:
            json.dump(res, f, indent=1)
        print("refreshed", out)
        return
    res = {"workload": w["desc"], "chi": a.chi, "mode": "var", "sweeps": 2, "seed": 0,
           "input": fingerprint(A), "what": "oracle (FP64 CPU): ln|<psi|psi>| by the top-down sweep and the "
                                            "last row's <sigma_z> (sites) and <S.S> (horizontal bonds)"}
    res.update(last_row_and_norm(A, a.chi, log=lambda m: print(m, flush=True)))
    with open(out, "w") as f:
        json.dump(res, f, indent=1)
    print("wrote", out)


if __name__ == "__main__":
    main()
