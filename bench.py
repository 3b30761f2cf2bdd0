#!/usr/bin/env python
"""Benchmark: full boundary-MPS environments of a 10x10 OBC PEPS (d=2, D=4).

Workload (one step): every site environment of a 10x10 PEPS with d=2, D=4,
entries 0.5 + 0.1*N(0,1) (unit-norm tensors, seeded), boundary bond chi=64,
variational (2 half-sweep) compression -- four directional sweeps, the row
and column environments, every site / bond density matrix -- followed by
<S.S> on every one of the 180 nearest-neighbour bonds.  One step yields
Ly*Lx = 100 site environments; the metric is environments per second.

The headline path computes the absorb contractions on the tensor cores in
split TF32 (tf32x3) with FP64 QR / gauge / rescaling; the same line reports
the plain FP64 GPU path's throughput and the largest relative deviation of
the 180 bond observables between the two.  Each step replays the recorded
plan (one CUDA graph for the whole environment set) and evaluates <S.S>.

A "cluster" object adds the cluster scheme on the 14x14 D=6 lattice (all 196
windows at chi=36, n = 2, 4, 6) with its deviation from the full chi=64
environments.

Launch: ``python bench.py [--gpus N --steps K --warmup W]``; for N > 1 run
under ``torch.distributed.run`` with one process per GPU.  The full
environment does not shard, so every rank computes its own replica (seed 2 +
rank): weak scaling, no collective on the data path.

``--impl reference`` times the FP64 CPU oracle on the host cores instead
(a bounded sample of the same workload, extrapolated by operation count).
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

WORKLOAD = dict(name="10x10_D4", Ly=10, Lx=10, d=2, D=4, seed=2)
L2_BYTES = 129 * 2 ** 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it
# stands (profiles/<kernel>_bench_10x10_D4_chi64.md); update or drop an entry
# whenever that kernel changes.
TRAFFIC = {
    "qr_f64": (595456, "ncu dram__bytes_read.sum + dram__bytes_write.sum of one 1024x64 k_qr_cluster "
                       "launch (profiles/k_qr_cluster_bench_10x10_D4_chi64.md); the matrix read once"),
}

# FP64 ALU peak of GB300 from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


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


def run_ours(args, rank, world, dist):
    import numpy as np
    import torch

    from paper_1311_6696_gb300 import peps, synth

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    st = torch.cuda.current_stream()
    A = synth.peps_gauss(WORKLOAD["Ly"], WORKLOAD["Lx"], WORKLOAD["d"], WORKLOAD["D"], WORKLOAD["seed"] + rank)
    At = torch.from_numpy(A).to(dev)
    Ah = torch.from_numpy(A).pin_memory()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    kw = dict(chi=args.chi, mode=args.mode, sweeps=2, precision=args.precision, stream=st)

    # ---- one replay of a plan with every kernel class timed inside the graph
    # (event nodes run back to back with the kernels, so small kernels are not
    # charged the host's launch gaps): the class with the most device time is
    # the one whose roofline is reported; the absorb class is reported from
    # the same replay.
    peps.profile_enable(-1)
    probe = peps.Plan(At, **kw)
    peps.profile_enable(0)
    probe.run()
    torch.cuda.synchronize()
    peps.profile_reset()
    probe.run()
    prof1 = peps.profile_read()
    probe.free()
    del probe
    dom = args.dominant or max((k for k in prof1 if prof1[k]["launches"]), key=lambda k: prof1[k]["ms"])
    absorb = "gemm_tc" if args.precision != "fp64" else "gemm_f64"

    # ---- the step as a user runs it repeatedly: the recorded plan (one CUDA
    # graph launch for the whole environment set), then <S.S> on every bond.
    # The dominant class is timed inside every replay (event nodes around its
    # launches); the absorb class's figure comes from the probe replay above.
    peps.profile_enable(1 << peps.class_index(dom))
    plan = peps.Plan(At, **kw, tune=not args.no_tune)
    peps.profile_enable(0)
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
    times = []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        h1, v1 = step()
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = _clock_summary(clocks, local) if rank == 0 else None
    prof = peps.profile_read()
    launches = sum(v["launches"] for v in prof.values())

    # ---- end to end: pinned host tensors in (H2D into the plan's lattice), replay, observables out
    etimes = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        At.copy_(Ah, non_blocking=True)
        step()
        etimes.append((time.perf_counter() - t0) * 1e3)

    # ---- the plain FP64 GPU path (also recorded) on the same input, and the deviation between the two
    cmp_ms, dev_err, others = None, None, {}
    if args.precision != "fp64" and not args.no_fp64_compare:
        p64 = peps.Plan(At, **dict(kw, precision="fp64"))
        e64 = p64.env
        p64.run()
        tms = []
        for _ in range(max(1, min(3, args.steps))):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            p64.run()
            h0, v0 = e64.expect("hbond", SD), e64.expect("vbond", SD)
            e1.record(st)
            e1.synchronize()
            tms.append(e0.elapsed_time(e1))
        cmp_ms = sum(tms) / len(tms)
        a = np.concatenate([h1, v1])
        b = np.concatenate([h0, v0])
        dev_err = float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-2)))
        del e64, p64
        # every other tensor-core precision on the same input, against the FP64 path
        for prec in ("bf16x3", "tf32", "bf16"):
            if prec == args.precision:
                continue
            pp = peps.Plan(At, **dict(kw, precision=prec), tune=not args.no_tune)
            ep = pp.env
            pp.run()
            tms = []
            for _ in range(max(1, min(3, args.steps))):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                pp.run()
                hp, vp = ep.expect("hbond", SD), ep.expect("vbond", SD)
                e1.record(st)
                e1.synchronize()
                tms.append(e0.elapsed_time(e1))
            ms_p = min(tms)
            c = np.concatenate([hp, vp])
            others[prec] = {"value": round(world * WORKLOAD["Ly"] * WORKLOAD["Lx"] / (ms_p * 1e-3), 2),
                            "ms_per_step": round(ms_p, 2),
                            "max_rel_err_vs_fp64_path": float(np.max(np.abs(c - b) / np.maximum(np.abs(b), 1e-2)))}
            del ep, pp

    cluster = None if args.no_cluster else cluster_section(args, peps, synth, torch, st, flush)

    total_ms = sum(times)
    envs = WORKLOAD["Ly"] * WORKLOAD["Lx"]
    ms_step, e_ms, value, e2e = aggregate(total_ms / len(times), sum(etimes) / len(etimes), envs, world,
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
            bf = pk.get("bf16_tflops_sustained", 1720.0)
            if args.precision.startswith("bf16"):
                peak, note = bf, "of measured bf16 sustained (cuBLAS, MEASURED_PEAKS.json)"
            else:
                peak, note = bf / 2.0, "of measured bf16 sustained x 1/2 (nominal tf32:bf16 dense ratio)"
            bound = "tensor"
        else:
            peak, bound = FP64_PEAK_TFLOPS, "alu"
            note = "FP64 ALU peak derived from 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"
        tr = TRAFFIC.get(cls) if src is None else None
        return {"bound": bound, "kernel": cls, "achieved": round(achieved, 4), "peak": round(peak, 4),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 5), "traffic": tr[0] if tr else None,
                "traffic_source": tr[1] if tr else None,
                "launches": d["launches"], "avg_launch_us": round(1e3 * d["ms"] / max(1, d["launches"]), 3),
                "algorithmic_flops_per_launch": round(d["flops"] / max(1, d["launches"]), 1),
                "peak_source": note, "timed": timed}

    h2d = int(A.nbytes)
    d2h = 8 * (WORKLOAD["Ly"] * (WORKLOAD["Lx"] - 1) + (WORKLOAD["Ly"] - 1) * WORKLOAD["Lx"])
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
                  "bf16x3": "bf16x3+f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": "10x10 OBC PEPS d=2 D=4, entries 0.5+0.1N(0,1), unit-norm tensors",
                   "chi": args.chi, "mode": args.mode, "sweeps": 2, "precision": args.precision,
                   "envs_per_step": envs, "l2": "flushed between steps (256 MiB write)",
                   "launch": f"recorded plan (CUDA graph of {plan.launches} kernels) replayed per step",
                   "tuned": {"lanes": plan.lanes, "qr_cluster_max": plan.qr_cluster} if not args.no_tune else None,
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": round(e2e, 3), "unit": "envs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": roof(dom),
        "roofline_absorb": roof(absorb, prof1) if absorb != dom else None,
        "replay_kernel_ms": {k: round(v["ms"], 3) for k, v in prof1.items() if v["launches"]},
        "wall_s_timed": round(t_wall, 3),
    }
    if cmp_ms is not None:
        res["fp64_path"] = {"value": round(world * envs / (cmp_ms * 1e-3), 3), "unit": "envs/s",
                            "ms_per_step": round(cmp_ms, 3)}
        res["speedup_vs_fp64_path"] = round(cmp_ms / ms_step, 3)
        res["accuracy"] = {"max_rel_err_vs_fp64_path": dev_err, "observables": 180,
                           "metric": "|x-x_ref|/max(|x_ref|,1e-2) over <S.S> on every bond"}
        res["other_precisions"] = others
    if cluster is not None:
        res["cluster"] = cluster
    if clk:
        res["clocks"] = clk
    if not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_sample(args, budget_s=args.cpu_budget)
    return res


SD = [[0.25, 0, 0, 0], [0, -0.25, 0.5, 0], [0, 0.5, -0.25, 0], [0, 0, 0, 0.25]]


def cluster_section(args, peps, synth, torch, st, flush):
    """Cluster environments of the 14x14 D=6 lattice (all 196 windows, chi=36,
    n in {2, 4, 6}) as recorded plans, with their deviation from the full
    chi=64 environments on sigma_z and <S.S> (every site and bond)."""
    import numpy as np
    A = torch.from_numpy(synth.workload("14x14_D6")).cuda()
    SZ = np.diag([1.0, -1.0])

    def obs(e):
        return np.concatenate([e.expect("site", SZ), e.expect("hbond", SD), e.expect("vbond", SD)])

    ref = peps.env_full(A, chi=64, mode="var", precision=args.precision, stream=st)
    r = obs(ref)
    ref.free()
    out = {"workload": "14x14 OBC PEPS d=2 D=6, entries 0.5+0.1N(0,1), 196 windows, chi=36, var, "
                       f"{args.precision}; reference: full environments at chi=64",
           "per_n": {}}
    for n in (2, 4, 6):
        t0 = time.perf_counter()
        plan = peps.Plan(A, chi=36, mode="var", precision=args.precision, cluster_n=n, stream=st,
                         tune=not args.no_tune)
        t_create = time.perf_counter() - t0
        env = plan.env
        plan.run()
        tms = []
        for _ in range(2):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            plan.run()
            o = obs(env)
            e1.record(st)
            e1.synchronize()
            tms.append(e0.elapsed_time(e1))
        ms = min(tms)
        err = float(np.max(np.abs(o - r) / np.maximum(np.abs(r), 1e-2)))
        out["per_n"][str(n)] = {"envs_per_s": round(196 / (ms * 1e-3), 2), "ms": round(ms, 2),
                                "launches": plan.launches, "max_rel_dev_vs_full_chi64": err,
                                "tuned": {"lanes": plan.lanes, "qr_cluster_max": plan.qr_cluster}
                                if not args.no_tune else None, "plan_create_s": round(t_create, 1)}
        del env
        plan.free()
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


def cpu_sample(args, budget_s=20.0):
    """The FP64 oracle as it stands, on a bounded sample of the same workload.

    Sample: top-down absorb+compress steps of interior rows until the budget is
    spent, plus one row pass (row environments and all density matrices of that
    row, with the boundary above it standing in for the one below, which has the
    same shapes).  envs/s = Ly*Lx / (4 (L-1) t_absorb + 2 L t_row), i.e. the
    full environment set's operation count: four directional sweeps of L-1 rows
    and L row passes plus L column passes.
    """
    import numpy as np

    from oracle import peps_oracle as O
    from paper_1311_6696_gb300 import synth

    A = synth.peps_gauss(WORKLOAD["Ly"], WORKLOAD["Lx"], WORKLOAD["d"], WORKLOAD["D"], WORKLOAD["seed"])
    lat = O.lattice_from_dense(A)
    L = WORKLOAD["Ly"]
    T = O.closure_mps(lat.top)
    ts = []
    y = 0
    t_start = time.perf_counter()
    while y < L - 1:
        t0 = time.perf_counter()
        T, _ = O.absorb_compress(T, lat, y, args.chi, args.mode, 2, 0, 0)
        dt = time.perf_counter() - t0
        if y >= 1:
            ts.append(dt)
        y += 1
        if time.perf_counter() - t_start > budget_s and len(ts) >= 1:
            break
    t0 = time.perf_counter()
    O._row_rhos(lat, T, T, y)
    t_row = time.perf_counter() - t0
    t_abs = float(np.median(ts))
    t_set = 4 * (L - 1) * t_abs + 2 * L * t_row
    cores = _blas_threads()
    return {"value": round(L * L / t_set, 5), "unit": "envs/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(ts)} interior absorb+compress steps (median {t_abs:.2f} s) and one row pass "
                      f"({t_row:.2f} s) of the same 10x10 D=4 chi={args.chi} {args.mode} workload, "
                      f"extrapolated to the full environment set (4x{L-1} absorbs + {2*L} row passes)"}


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
    steps = []
    cb = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_sample(args, budget_s=args.ref_budget)
        if i >= args.warmup:
            steps.append((time.perf_counter() - t0, cb["value"]))
    v = statistics.mean(s[1] for s in steps)
    return {
        "impl": "reference",
        "metric": "PEPS site environments/sec (full boundary-MPS envs + <S.S> on all bonds)",
        "value": round(v, 5), "unit": "envs/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * statistics.mean(s[0] for s in steps), 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "10x10 OBC PEPS d=2 D=4, entries 0.5+0.1N(0,1), unit-norm tensors",
                   "chi": args.chi, "mode": args.mode, "sweeps": 2, "precision": "fp64"},
        "cpu_baseline": {"value": round(v, 5), "unit": "envs/s", "cores": cb["cores"], "kind": "oracle",
                         "sample": cb["sample"]},
        "e2e": {"value": round(v, 5), "unit": "envs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chi", type=int, default=64)
    ap.add_argument("--mode", default="var", choices=["var", "svd"])
    ap.add_argument("--precision", default="tf32x3", choices=["fp64", "tf32", "bf16", "tf32x3", "bf16x3"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--dominant", default=None, help="kernel class timed for the roofline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cluster", action="store_true", help="skip the 14x14 D=6 cluster section")
    ap.add_argument("--no-tune", action="store_true", help="record the plan with the default launch configuration")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--ref-budget", type=float, default=10.0)
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
    res = run_ours(args, rank, world, dist)
    if res is not None:
        print(json.dumps(res), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
