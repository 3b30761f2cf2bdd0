#!/usr/bin/env python
"""Benchmark: full boundary-MPS environments of a 20x20 OBC PEPS (d=2, D=8).

Workload (one step): every site environment of the 20x20 D=8 lattice made by
the seeded simple-update Heisenberg generator (tau=0.01, 400 steps), boundary
bond chi=128, variational (2 half-sweep) compression -- four directional
sweeps, the row and column environments, every site / bond density matrix --
followed by <S.S> on every one of the 760 nearest-neighbour bonds.  One step
yields Ly*Lx = 400 site environments; the metric is environments per second.

The absorb contractions run on the tensor cores in split BF16 (bf16x3: three
BF16 products per FP32 operand pair, FP32 accumulation) with FP64 QR, gauge
and rescaling.  Each step replays the recorded plan (one CUDA graph for the
whole environment set) and evaluates <S.S>.  The line also reports

* the accuracy of the step's own output against the FP64 oracle on the same
  tensors (ln N and the last row's observables, stored by
  tests/golden/make_oracle_golden.py);
* the FP64 GPU path on a bounded part of the same lattice (the norm sweep of
  its top rows) against the headline precision on the same part;
* the FP64 oracle on the host cores (a bounded sample, costed up to the whole
  environment set by operation count).

The roofline is that of the kernel class with the largest share of
exclusive device time in a launch list of one replay (the FP64 QR at this
workload); the absorb contractions are reported beside it, against the BF16
peak and against HBM.

``--workload c2`` runs the 10x10 D=4 chi=64 lattice instead (entries
0.5 + 0.1 N(0,1)), with the FP64 path timed on the whole set.  ``--cluster``
adds the cluster scheme on the 14x14 D=6 lattice (all 196 windows at chi=36,
n = 2, 4, 6); ``--fidelity`` the boundary distance 1 - f of Fig. Fid on the
20x20 D=4 simple-update lattice; ``--update`` the tensor update's Trotter
steps (full update and CU_0 .. CU_3) on that lattice beside the boundary
step time t_B.  ``--rows R`` runs only the norm sweep of the top R rows (a
small case for profiler captures) and exits.

Launch: ``python bench.py [--gpus N --steps K --warmup W]``; for N > 1 run
under ``torch.distributed.run`` with one process per GPU.  The full
environment does not shard, so every rank computes its own replica (seed +
rank): weak scaling, no collective on the data path.

``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "c4": dict(name="20x20_D8_su", Ly=20, Lx=20, d=2, D=8, chi=128, precision="bf16x3",
               desc="20x20 OBC PEPS d=2 D=8 from the seeded simple-update Heisenberg generator "
                    "(tau=0.01, 400 steps, seed 4), unit-norm tensors",
               golden="oracle_20x20_D8_su_chi128.json", fp64_rows=4,
               # largest share of device time in the serialised launch list of a replay
               dominant="qr_f64"),
    "c2": dict(name="10x10_D4", Ly=10, Lx=10, d=2, D=4, chi=64, precision="tf32x3",
               desc="10x10 OBC PEPS d=2 D=4, entries 0.5+0.1N(0,1), unit-norm tensors",
               golden=None, fp64_rows=None, dominant=None),
}
L2_BYTES = 129 * 2 ** 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it
# stands, keyed by (workload, class); an entry is dropped whenever its kernel changes.
TRAFFIC = {
    # (workload, class): (dram read + write bytes per launch, source)
    ("c4", "qr_f64"): (4.54e6, "ncu --set full, mean of the 2 captured k_qr_cluster launches (stacked R "
                               "0.61 MB, tall-skinny leaves 8.47 MB) of the chi=128 fit; "
                               "profiles/k_qr_cluster_rows3_20x20_D8_chi128.md"),
}

# Dense FP64 and TF32 peaks: measured at start-up by _measure_peaks (torch
# matmul 8192^3 on this GPU); these values (one earlier measurement on a GB300,
# best of 5) stand in if that fails.
FP64_PEAK_TFLOPS = 1.0996
TF32_PEAK_TFLOPS = 1008.8


def _clock_sampler():
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None


def _clock_summary(proc, gpu_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sms, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9 or f[0] != str(gpu_index):
            continue
        try:
            sms.append(float(f[1]))
            mx = max(mx, float(f[2]))
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sms:
        return None
    return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sms)}


def load_input(name: str, seed_offset: int = 0):
    """The named synthetic lattice (synth.workload); the simple-update lattices
    take a minute or two to generate, so they are kept in the temp directory
    keyed by the generator's source and the seed (a later process on the same
    machine reuses them)."""
    import hashlib
    import tempfile

    import numpy as np

    from paper_1311_6696_gb300 import synth
    w = synth.WORKLOADS[name]
    seed = w["seed"] + seed_offset
    if w["gen"] != "su":
        return synth.workload(name, seed=seed)
    src = open(synth.__file__, "rb").read()
    key = hashlib.sha256(src + f"{name}:{seed}".encode()).hexdigest()[:16]
    path = os.path.join(tempfile.gettempdir(), f"peps_input_{name}_{key}.npy")
    if os.path.exists(path):
        try:
            return np.load(path)
        except (OSError, ValueError):
            pass
    A = synth.workload(name, seed=seed)
    tmp = f"{path}.{os.getpid()}.tmp.npy"
    np.save(tmp, A)
    os.replace(tmp, path)
    return A


def _timed(fn, st, n, flush=None):
    """Device times (ms) of n calls of fn on stream st, CUDA events around each."""
    import torch
    out = []
    for _ in range(n):
        if flush is not None:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def _rel(a, b):
    import numpy as np
    a = np.asarray(a, dtype=float)
    b = np.asarray(b, dtype=float)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-2)))


def run_ours(args, rank, world, dist):
    import numpy as np
    import torch

    from paper_1311_6696_gb300 import peps

    W = WORKLOADS[args.workload]
    chi = args.chi or W["chi"]
    prec = args.precision or W["precision"]
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    st = torch.cuda.current_stream()
    A = load_input(W["name"], seed_offset=rank)
    At = torch.from_numpy(A).to(dev)
    Ah = torch.from_numpy(A).pin_memory()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    kw = dict(chi=chi, mode=args.mode, sweeps=2, precision=prec, stream=st)
    Ly, Lx = W["Ly"], W["Lx"]
    envs = Ly * Lx

    # ---- one replay of a plan with every kernel class timed inside the graph
    # (event nodes run back to back with the kernels): the class with the most
    # device time is the one whose roofline is reported.
    prof1 = None
    dom = args.dominant or (None if args.probe else W.get("dominant"))
    if dom is None:
        peps.profile_enable(-1)
        probe = peps.Plan(At, **kw)
        peps.profile_enable(0)
        peps.profile_reset()
        probe.run()
        prof1 = peps.profile_read()
        probe.free()
        del probe
        dom = max((k for k in prof1 if prof1[k]["launches"]), key=lambda k: prof1[k]["ms"])
    absorb = "gemm_tc" if prec != "fp64" else "gemm_f64"

    # ---- the step as a user runs it repeatedly: the recorded plan (one CUDA
    # graph launch for the whole environment set), then <S.S> on every bond.
    # The dominant class is timed inside every replay (event nodes around its
    # launches).
    t0 = time.perf_counter()
    # the roofline's class and the absorb contractions' class, timed by event
    # nodes around their launches inside every replay
    peps.profile_enable((1 << peps.class_index(dom)) | (1 << peps.class_index(absorb)))
    plan = peps.Plan(At, **kw, tune=args.tune)
    peps.profile_enable(0)
    t_plan = time.perf_counter() - t0
    env = plan.env

    def step():
        plan.run()
        return env.expect("hbond", SD), env.expect("vbond", SD)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    peps.profile_reset()
    clocks = _clock_sampler() if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    times = _timed(step, st, args.steps, flush)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = _clock_summary(clocks, local) if rank == 0 else None
    prof = peps.profile_read()
    launches = sum(v["launches"] for v in prof.values())
    h1, v1 = step()
    out_site = env.expect("site", SZ)
    ln_step = env.ln_norm()

    # ---- end to end: pinned host tensors in (H2D into the plan's lattice),
    # replay, observables out (D2H), timed on the host
    etimes = []
    for _ in range(max(1, min(args.steps, args.e2e_steps))):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        At.copy_(Ah, non_blocking=True)
        step()
        etimes.append((time.perf_counter() - t1) * 1e3)

    # ---- accuracy of the step's own output against the FP64 oracle
    accuracy = None
    gpath = os.path.join(ROOT, "tests", "golden", W["golden"]) if W["golden"] else None
    if gpath and os.path.exists(gpath) and args.mode == "var" and rank == 0:
        g = json.load(open(gpath))
        from paper_1311_6696_gb300 import synth
        same = "gram4" in g["input"] and abs(synth.gram4(A) - g["input"]["gram4"]) < 1e-9 * abs(g["input"]["gram4"])
        if not same or g["chi"] != chi:
            accuracy = {"vs": "FP64 oracle", "skipped": "the stored oracle result is for another input or chi"}
        else:
            y = g["row"]
            sz = out_site.reshape(Ly, Lx)[y]
            ss = h1.reshape(Ly, Lx - 1)[y]
            accuracy = {"vs": "FP64 oracle on the same tensors (stored: " + os.path.relpath(gpath, ROOT) + ")",
                        "max_rel_err": max(_rel(sz, g["sz"]), _rel(ss, g["sdots_h"])),
                        "observables": f"<sigma_z> on the {Lx} sites and <S.S> on the {Lx - 1} bonds of row {y}",
                        "ln_norm_abs_err": abs(ln_step[0] - g["ln_norm"]),
                        "metric": "|x-x_ref|/max(|x_ref|,1e-2); absolute on ln N"}

    # ---- the plain FP64 GPU path
    fp64 = None
    if prec != "fp64" and not args.no_fp64_compare:
        if W["fp64_rows"]:
            # bounded: the norm sweep (Section 2) of the lattice's top rows, both precisions
            R = W["fp64_rows"]
            part = np.array(A[:R])
            part[R - 1, :, :, :, :, 1:, :] = 0.0        # the part's last row: down legs closed (OBC)
            sub = torch.from_numpy(part).to(dev)
            for p_ in ("fp64", prec):
                peps.norm(sub, chi=chi, mode=args.mode, precision=p_, stream=st)   # warm
            tf = _timed(lambda: peps.norm(sub, chi=chi, mode=args.mode, precision="fp64", stream=st), st, 1)
            tp = _timed(lambda: peps.norm(sub, chi=chi, mode=args.mode, precision=prec, stream=st), st, 2)
            fp64 = {"part": f"norm sweep of the top {R} rows of the same lattice ({R - 1} absorbs at chi={chi}; "
                            "the part's last row closed at index 0 of its down legs)",
                    "fp64_ms": round(min(tf), 1), f"{prec}_ms": round(min(tp), 1),
                    "speedup": round(min(tf) / min(tp), 3)}
        else:
            p64 = peps.Plan(At, **dict(kw, precision="fp64"))
            e64 = p64.env
            tms = _timed(lambda: (p64.run(), e64.expect("hbond", SD)), st, max(1, min(3, args.steps)), flush)
            h0, v0 = e64.expect("hbond", SD), e64.expect("vbond", SD)
            ms64 = min(tms)
            fp64 = {"part": "whole environment set", "value": round(world * envs / (ms64 * 1e-3), 3),
                    "unit": "envs/s", "ms_per_step": round(ms64, 3),
                    "max_rel_err_vs_fp64_path": _rel(np.concatenate([h1, v1]), np.concatenate([h0, v0]))}
            del e64, p64

    cluster = cluster_section(args, peps, torch, st, flush) if args.cluster else None
    fidelity = fidelity_section(peps, torch, st) if args.fidelity and rank == 0 else None
    update = update_section(args, peps, torch, st) if args.update and rank == 0 else None

    ms_step, e_ms, value, e2e = aggregate(sum(times) / len(times), sum(etimes) / len(etimes), envs, world,
                                          dist, dev)
    if rank != 0:
        return None

    pk = _peaks()

    def roof(cls, src=None):
        d = (src or prof)[cls]
        timed = ("CUDA events recorded inside the replayed graph (timed steps)" if src is None else
                 "CUDA events recorded inside one replay of a graph timing every class")
        if cls == "pack":
            achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9 if d["ms"] > 0 else 0.0
            peak = pk.get("hbm_gbs", 6765.0)
            return {"bound": "hbm", "kernel": cls, "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 5), "traffic": None, "launches": d["launches"],
                    "avg_launch_us": round(1e3 * d["ms"] / max(1, d["launches"]), 3),
                    "peak_source": "of measured HBM copy bandwidth (MEASURED_PEAKS.json)", "timed": timed}
        achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12 if d["ms"] > 0 else 0.0
        if cls == "gemm_tc":
            if prec.startswith("bf16"):
                peak = pk.get("bf16_tflops_sustained", 1716.1)
                note = ("of measured bf16 dense, sustained (cuBLAS, MEASURED_PEAKS.json)" if pk else
                        "of measured bf16 dense, sustained (cuBLAS; this pool's earlier MEASURED_PEAKS.json "
                        "value, the file being absent)")
            else:
                peak, note = TF32_PEAK_TFLOPS, "of measured tf32 dense (torch matmul 8192^3, best of 5)"
            bound = "tensor"
        else:
            peak, bound = FP64_PEAK_TFLOPS, "alu"
            note = "of measured FP64 dense (torch matmul 8192^3, best of 5)"
        tr = TRAFFIC.get((args.workload, cls)) if src is None else None
        r = {"bound": bound, "kernel": cls, "achieved": round(achieved, 4), "peak": round(peak, 4),
             "unit": "TFLOP/s", "frac": round(achieved / peak, 5), "traffic": tr[0] if tr else None,
             "traffic_source": tr[1] if tr else None,
             "launches": d["launches"], "avg_launch_us": round(1e3 * d["ms"] / max(1, d["launches"]), 3),
             "algorithmic_flops_per_launch": round(d["flops"] / max(1, d["launches"]), 1),
             "peak_source": note, "timed": timed}
        if cls == "gemm_tc" and d["bytes"] > 0 and d["ms"] > 0:
            # the same launches against HBM: packed operands read once, output written once
            gbs = d["bytes"] / (d["ms"] * 1e-3) / 1e9
            hbm = pk.get("hbm_gbs", 6765.0)
            r["hbm_view"] = {"achieved": round(gbs, 2), "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 5),
                             "algorithmic_bytes_per_launch": round(d["bytes"] / max(1, d["launches"]), 1),
                             "flops_per_byte": round(d["flops"] / d["bytes"], 2),
                             "peak_source": "of measured HBM copy bandwidth (MEASURED_PEAKS.json)" if pk else
                             "of measured HBM copy bandwidth (this pool's earlier MEASURED_PEAKS.json value, "
                             "the file being absent)"}
        return r

    h2d = int(A.nbytes)
    d2h = 8 * (Ly * (Lx - 1) + (Ly - 1) * Lx)
    res = {
        "metric": "PEPS site environments/sec (full boundary-MPS envs + <S.S> on all bonds)",
        "value": round(value, 3),
        "unit": "envs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": max(3, args.warmup),
        "ms_per_step": round(ms_step, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "tf32": "tf32", "bf16": "bf16", "tf32x3": "tf32x3+f64",
                  "bf16x3": "bf16x3+f64"}[prec],
        "data": "synthetic",
        "config": {"workload": W["desc"], "chi": chi, "mode": args.mode, "sweeps": 2, "precision": prec,
                   "envs_per_step": envs,
                   "l2": "flushed between steps (256 MiB write); the step's working set is far above L2",
                   "launch": f"recorded plan (CUDA graph of {plan.launches} kernels) replayed per step",
                   "tuned": {"lanes": plan.lanes, "qr_cluster_max": plan.qr_cluster} if args.tune else None,
                   "plan_create_s": round(t_plan, 1), "parallelism": f"replicas x{world}"},
        "e2e": {"value": round(e2e, 3), "unit": "envs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": len(etimes)},
        "gpu_launches": int(launches),
        "roofline": roof(dom),
        "roofline_absorb": roof(absorb) if (absorb != dom and prof[absorb]["launches"]) else None,
        "replay_kernel_ms": {k: round(v["ms"], 3) for k, v in prof1.items() if v["launches"]} if prof1 else None,
        "wall_s_timed": round(t_wall, 3),
    }
    if accuracy is not None:
        res["accuracy"] = accuracy
    if fp64 is not None:
        res["fp64_path"] = fp64
        if "ms_per_step" in fp64:
            res["speedup_vs_fp64_path"] = round(fp64["ms_per_step"] / ms_step, 3)
    if cluster is not None:
        res["cluster"] = cluster
    if fidelity is not None:
        res["fidelity"] = fidelity
    if update is not None:
        res["update"] = update
    if clk:
        res["clocks"] = clk
    if not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_sample(args, budget_s=args.cpu_budget)
    return res


SD = [[0.25, 0, 0, 0], [0, -0.25, 0.5, 0], [0, 0.5, -0.25, 0], [0, 0, 0, 0.25]]
SZ = [[1.0, 0.0], [0.0, -1.0]]


def cluster_section(args, peps, torch, st, flush):
    """Cluster environments of the 14x14 D=6 lattice (all 196 windows, chi=36,
    n in {2, 4, 6}) as recorded plans, with their deviation from the full
    chi=64 environments on sigma_z and <S.S> (every site and bond)."""
    import numpy as np
    prec = "tf32x3"
    A = torch.from_numpy(load_input("14x14_D6")).cuda()
    SZm = np.diag([1.0, -1.0])

    def obs(e):
        return np.concatenate([e.expect("site", SZm), e.expect("hbond", SD), e.expect("vbond", SD)])

    ref = peps.env_full(A, chi=64, mode="var", precision=prec, stream=st)
    r = obs(ref)
    ref.free()
    out = {"workload": "14x14 OBC PEPS d=2 D=6, entries 0.5+0.1N(0,1), 196 windows, chi=36, var, "
                       f"{prec}; reference: full environments at chi=64",
           "per_n": {}}
    for n in (2, 4, 6):
        t0 = time.perf_counter()
        plan = peps.Plan(A, chi=36, mode="var", precision=prec, cluster_n=n, stream=st, tune=args.tune)
        t_create = time.perf_counter() - t0
        env = plan.env
        plan.run()
        tms = _timed(lambda: (plan.run(), obs(env)), st, 2, flush)
        ms = min(tms)
        o = obs(env)
        out["per_n"][str(n)] = {"envs_per_s": round(196 / (ms * 1e-3), 2), "ms": round(ms, 2),
                                "launches": plan.launches, "max_rel_dev_vs_full_chi64": _rel(o, r),
                                "plan_create_s": round(t_create, 1)}
        del env
        plan.free()
    return out


def fidelity_section(peps, torch, st):
    """Section 5.2 / Fig. Fid on the paper's setting: 1 - f of the left-most
    column's environment of a 20x20 simple-update Heisenberg PEPS (D=4),
    clusters of delta = 1..4 columns and the full contraction at D' in
    {4, 8, 16, 32, 64}, against the full contraction at D' = 100 (FP64)."""
    A = torch.from_numpy(load_input("20x20_D4_su")).cuda()
    out = {"workload": "20x20 OBC PEPS d=2 D=4, seeded simple-update Heisenberg generator (tau=0.01, 400 steps); "
                       "var, FP64; reference: full contraction at D'=100", "one_minus_f": {}}
    t0 = time.perf_counter()
    for delta in (1, 2, 3, 4, 19):
        key = "full" if delta == 19 else f"delta={delta}"
        out["one_minus_f"][key] = {str(chi): peps.boundary_fidelity(A, delta, chi=chi, chi_ref=100, stream=st)
                                   for chi in (4, 8, 16, 32, 64)}
    out["seconds"] = round(time.perf_counter() - t0, 1)
    return out


def update_section(args, peps, torch, st):
    """The tensor update (Section 2) under the parallel schedule, timed per
    Trotter set: the full update and the cluster updates CU_delta, beside the
    time t_B of one boundary step (the quantities of the paper's timing model,
    Section 5.4: sequential FU 2(L-2) t_B + L t_U per set, parallel CU_delta
    2(delta-1) t_B + t_U per row)."""
    import numpy as np
    from paper_1311_6696_gb300 import synth
    name, chi, prec = "20x20_D4_su", 16, "bf16x3"
    A0 = torch.from_numpy(synth.workload(name)).to("cuda")
    Ly = int(A0.shape[0])
    h = np.array([[0.25, 0, 0, 0], [0, -0.25, 0.5, 0], [0, 0.5, -0.25, 0], [0, 0, 0, 0.25]])
    w, v = np.linalg.eigh(h)
    G = (v * np.exp(-0.01 * w)) @ v.T
    sets = peps.trotter_sets(Ly, int(A0.shape[1]))
    kw = dict(chi=chi, mode="var", precision=prec, iters=8, stream=st)
    peps.norm(A0, chi=chi, mode="var", precision=prec, stream=st)
    t_sweep = min(_timed(lambda: peps.norm(A0, chi=chi, mode="var", precision=prec, stream=st), st, 2))
    out = {"workload": f"{name} (20x20 D=4 simple-update Heisenberg, seed 6), chi={chi}, var, {prec}, "
                       "gate exp(-0.01 h), 8 ALS rounds; every schedule starts from the same state",
           "t_B_ms": round(t_sweep / (Ly - 1), 3), "sweep_ms": round(t_sweep, 2), "per_schedule": {}}
    for name_s, delta in [("FU", None), ("CU_0", 0), ("CU_1", 1), ("CU_2", 2), ("CU_3", 3)]:
        A = A0.clone()
        peps.bond_update(A.clone(), G, sets[0], delta=delta, **kw)       # warm
        times = [min(_timed(lambda: peps.bond_update(A, G, s_, delta=delta, **kw), st, 1)) for s_ in sets]
        out["per_schedule"][name_s] = {"set_ms": [round(t, 2) for t in times],
                                       "step_ms": round(sum(times), 2)}
    fu = out["per_schedule"]["FU"]["step_ms"]
    for k, v_ in out["per_schedule"].items():
        v_["fu_over_this"] = round(fu / v_["step_ms"], 3)
    return out


def aggregate(ms_step, e_ms, envs_per_rank, world, dist=None, device=None):
    """Whole-job throughput of weak-scaled replicas: the slowest rank's step
    time (max over ranks) bounds the job; every rank processed envs_per_rank."""
    if dist is not None:
        import torch
        t = torch.tensor([ms_step, e_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step, e_ms = float(t[0]), float(t[1])
    value = world * envs_per_rank / (ms_step * 1e-3)
    e2e = world * envs_per_rank / (e_ms * 1e-3)
    return ms_step, e_ms, value, e2e


def set_cost_model(L: int, t_step: float, t_open: float) -> float:
    """Seconds of one environment set of an L x L lattice (var mode, two
    half-sweeps) from the time of one site step of a fit (absorb chain,
    closing contraction, QR, environment update) and of one site's density
    matrices (site + right bond).  Each absorbed row costs (L-1) right
    environments to start the fit and L site steps per half-sweep; each of the
    2L row / column passes costs 2(L-1) environment steps and L open sites.
    Every site is costed as an interior one (an upper bound: edge sites have
    smaller bonds)."""
    absorb = (L - 1) + 2 * L
    return 4 * (L - 1) * absorb * t_step + 2 * L * (2 * (L - 1) * t_step + L * t_open)


_OPEN_SITE_S = {}


def cpu_sample(args, budget_s=20.0):
    """The FP64 oracle as it stands on a bounded sample of the same workload.

    Sample: single site steps of the variational fit at the centre of an
    interior row (absorb chain, closing contraction, QR, environment update)
    and one open site (its density matrix and its right bond's), on the
    workload's own site tensors with boundary and environment tensors of the
    interior shapes (chi, D, D, chi) drawn at random -- the cost of a step
    depends on the shapes only.  set_cost_model turns the times into the time
    of the whole environment set.
    """
    import numpy as np

    from oracle import peps_oracle as O

    W = WORKLOADS[args.workload]
    chi = args.chi or W["chi"]
    A = load_input(W["name"])
    lat = O.lattice_from_dense(A)
    L, Dv = W["Ly"], W["D"]
    t_all = time.perf_counter()
    y, x = L // 2, L // 2
    Ay = lat.A[y]
    rng = np.random.default_rng(0)

    def bt():
        return rng.standard_normal((chi, Dv, Dv, chi))

    M, M2, Lenv, Renv, Bm, Bm2 = bt(), bt(), bt(), bt(), bt(), bt()
    steps = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        X3 = O.chain_left(Lenv, M, Ay[x])
        b = O.close_left(X3, Renv)
        cc, n, o, e = b.shape
        Q, _ = np.linalg.qr(b.reshape(cc * n * o, e))
        O.lenv_next(X3, Q.reshape(cc, n, o, Q.shape[1]))
        steps.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > 0.6 * budget_s or len(steps) >= 5:
            break
    # the open site's cost depends on the shapes only: timed once per process
    key = (args.workload, chi)
    if key not in _OPEN_SITE_S:
        t0 = time.perf_counter()
        O.rho_site(Lenv, Renv, M, Ay[x], Bm)
        O.rho_hbond(Lenv, Renv, M, Ay[x], Bm, M2, Ay[x + 1], Bm2)
        _OPEN_SITE_S[key] = time.perf_counter() - t0
    t_open = _OPEN_SITE_S[key]
    t_step = float(np.median(steps))
    t_set = set_cost_model(L, t_step, t_open)
    cores = _blas_threads()
    return {"value": round(L * L / t_set, 6), "unit": "envs/s", "cores": cores, "kind": "oracle",
            "set_seconds": round(t_set, 1), "sample_wall_s": round(time.perf_counter() - t_all, 1),
            "sample": f"{len(steps)} interior site steps of the variational fit (median {t_step:.2f} s: "
                      f"absorb chain, closing contraction, QR, environment update) and one open site "
                      f"({t_open:.2f} s, timed once per process) of the same {L}x{L} D={Dv} chi={chi} "
                      f"{args.mode} workload, "
                      f"costed up to the whole environment set by operation count "
                      f"(bench.set_cost_model: every site as an interior one)"}


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def run_reference(args):
    W = WORKLOADS[args.workload]
    chi = args.chi or W["chi"]
    vals, cb = [], None
    t_wall = time.perf_counter()
    for i in range(args.warmup + args.steps):
        cb = cpu_sample(args, budget_s=args.ref_budget)
        if i >= args.warmup:
            vals.append(cb["value"])
    v = statistics.mean(vals)
    envs = W["Ly"] * W["Lx"]
    return {
        "impl": "reference",
        "metric": "PEPS site environments/sec (full boundary-MPS envs + <S.S> on all bonds)",
        "value": round(v, 6), "unit": "envs/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * envs / v, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": W["desc"], "chi": chi, "mode": args.mode, "sweeps": 2, "precision": "fp64",
                   "step": "one whole environment set, costed from a timed sample (see cpu_baseline)"},
        "cpu_baseline": {"value": round(v, 6), "unit": "envs/s", "cores": cb["cores"], "kind": "oracle",
                         "sample": cb["sample"]},
        "e2e": {"value": round(v, 6), "unit": "envs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": round(time.perf_counter() - t_wall, 1),
    }


def _measure_peaks():
    """FP64 and TF32 dense peaks of this GPU (torch matmul 8192^3, best of 3,
    CUDA events); the BF16 peak is MEASURED_PEAKS.json's."""
    import torch
    global FP64_PEAK_TFLOPS, TF32_PEAK_TFLOPS
    try:
        n = 8192
        old = torch.backends.cuda.matmul.allow_tf32
        for dt, tf32 in ((torch.float64, False), (torch.float32, True)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device="cuda", dtype=dt)
            b = torch.randn(n, n, device="cuda", dtype=dt)
            a @ b
            best = min(_timed(lambda: a @ b, torch.cuda.current_stream(), 3))
            tf = 2 * n ** 3 / (best * 1e-3) / 1e12
            if dt == torch.float64:
                FP64_PEAK_TFLOPS = tf
            else:
                TF32_PEAK_TFLOPS = tf
            del a, b
        torch.backends.cuda.matmul.allow_tf32 = old
        torch.cuda.empty_cache()
    except Exception:
        pass


def rows_case(args):
    """The norm sweep (Section 2) of the workload's top rows: the same absorb
    chains, fits and QR shapes as a full set, few enough launches for a
    profiler capture."""
    import numpy as np
    import torch

    from paper_1311_6696_gb300 import peps
    W = WORKLOADS[args.workload]
    chi = args.chi or W["chi"]
    prec = args.precision or W["precision"]
    R = args.rows
    A = load_input(W["name"])
    part = np.array(A[:R])
    part[R - 1, :, :, :, :, 1:, :] = 0.0        # the part's last row: down legs closed (OBC)
    sub = torch.from_numpy(part).cuda()
    st = torch.cuda.current_stream()
    peps.norm(sub, chi=chi, mode=args.mode, precision=prec, stream=st)     # warm
    t = _timed(lambda: peps.norm(sub, chi=chi, mode=args.mode, precision=prec, stream=st), st, 1)
    return {"case": f"norm sweep of the top {R} rows of {W['name']} ({R - 1} absorbs at chi={chi}, {prec})",
            "ms": round(min(t), 2)}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c4", choices=sorted(WORKLOADS))
    ap.add_argument("--chi", type=int, default=None, help="default: the workload's")
    ap.add_argument("--mode", default="var", choices=["var", "svd"])
    ap.add_argument("--precision", default=None, choices=["fp64", "tf32", "bf16", "tf32x3", "bf16x3"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--dominant", default=None, help="kernel class timed for the roofline (skips the probe replay)")
    ap.add_argument("--probe", action="store_true",
                    help="choose the roofline's class by one replay timing every class (concurrent lanes)")
    ap.add_argument("--rows", type=int, default=0,
                    help="small case for profilers: only the norm sweep of the workload's top ROWS rows "
                         "(last of them closed), at the headline precision, then exit")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cluster", action="store_true", help="add the 14x14 D=6 cluster section")
    ap.add_argument("--fidelity", action="store_true", help="add the boundary-fidelity section (Fig. Fid)")
    ap.add_argument("--update", action="store_true",
                    help="add the tensor-update section: FU and CU_delta Trotter sets on the 20x20 D=4 lattice")
    ap.add_argument("--tune", action="store_true", help="choose the plan's launch configuration by measurement")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--ref-budget", type=float, default=20.0)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        dist = tdist
    if args.rows > 0:
        if rank == 0:
            print(json.dumps(rows_case(args)), flush=True)
        return
    _measure_peaks()
    res = run_ours(args, rank, world, dist)
    if res is not None:
        print(json.dumps(res), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
