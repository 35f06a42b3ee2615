#!/usr/bin/env python3
"""Benchmark of the variational MPO-MPO fit on one GB300 (or N independent ones).

Workload (the timed configuration): two MPOs on L = 30 sites, local dims 2x2,
each a sum of 128 Kronecker products of 2x2 Gaussian factors with weights
0.8^k (bond 128 after exact trimming), fitted to chi_C = 128 with the
Gaussian-sketch randomized update (oversampling 10) until the relative change
of ||C||^2 between sweeps is <= 1e-8. A step is one complete fit: input
preparation, initial guess and right environments, sweeps until converged, and
the export of C. Metric: time-to-tol in seconds (lower is better), reported
with the local-update TFLOP/s of the contraction kernels against the measured
peak.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (a few bulk windows), scaled to the fit's window count.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MPO-MPO fit time-to-tol (s) & local-update TFLOP/s vs peak, L=30 χ=128"
WORKLOAD = "kron_L30_chi128"
L_SITES, CHI, OVERSAMPLE, TOL, MAX_SWEEPS = 30, 128, 10, 1e-8, 12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--precision", default=os.environ.get("TTFIT_BENCH_PRECISION", "fp32"))
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.p is None:
            return out
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# --------------------------------------------------------------------------- native arm
def native(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2606_23274_gb300 import ttfit
    from paper_2606_23274_gb300.synth import mpo_pair

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    ttfit.load()

    # inputs resident in HBM before the timed region; rank r fits its own pair
    A, B = mpo_pair(WORKLOAD, seed=rank)
    Ad = [torch.from_numpy(a).to(dev) for a in A]
    Bd = [torch.from_numpy(b).to(dev) for b in B]
    Ah = [torch.from_numpy(a).pin_memory() for a in A]
    Bh = [torch.from_numpy(b).pin_memory() for b in B]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    def one_fit(Ain, Bin, host=False):
        if host:
            Ain = [a.to(dev, non_blocking=True) for a in Ain]
            Bin = [b.to(dev, non_blocking=True) for b in Bin]
        f = ttfit.tt_fit_create(Ain, Bin, CHI, TOL, "site", update="rsvd", oversample=OVERSAMPLE, seed=rank,
                                precision=args.precision, device=dev, stream=stream)
        sweeps, rep = 0, None
        stages = {k: 0.0 for k in ("halves_ms", "join_ms", "env_finish_ms", "factorize_ms", "gauge_ms",
                                   "contraction_flops", "launches")}
        while sweeps < MAX_SWEEPS:
            rep = f.sweep(1)
            sweeps += 1
            st = f.stage_times()
            for k in stages:
                stages[k] += st[k]
            if rep["converged"]:
                break
        C = f.result()
        d2h = 0
        if host:
            Ch = [c.to("cpu", non_blocking=True) for c in C]
            d2h = sum(c.numel() * c.element_size() for c in Ch)
        f.destroy()
        return rep, sweeps, stages, C, d2h

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        one_fit(Ad, Bd)
        flush.zero_()
    barrier()
    clocks = ClockSampler(local)
    times, reps, stage_acc = [], [], []
    t_wall0 = time.time()
    for _ in range(args.steps):
        flush.zero_()                       # L2 flushed between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep, sweeps, stages, C, _ = one_fit(Ad, Bd)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        reps.append((rep, sweeps))
        stage_acc.append(stages)
    barrier()
    wall = time.time() - t_wall0
    clk = clocks.stop()
    t_step = statistics.mean(times)
    tmax = torch.tensor([t_step], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    t_step = float(tmax.item())

    e2e = None
    if not args.no_e2e:
        et = []
        h2d = sum(a.numel() * a.element_size() for a in Ah + Bh)
        d2h = 0
        for _ in range(max(1, min(args.steps, 2))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, _, _, _, d2h = one_fit(Ah, Bh, host=True)
            torch.cuda.synchronize()
            et.append(time.perf_counter() - t0)
        e2e = {"value": statistics.mean(et), "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # live per-stage times (CUDA events on the launching stream, inside the timed steps)
    agg = {k: statistics.mean(s[k] for s in stage_acc) for k in stage_acc[0]}
    contr_ms = agg["halves_ms"] + agg["join_ms"] + agg["env_finish_ms"]
    local_tflops = agg["contraction_flops"] / (contr_ms * 1e-3) / 1e12 if contr_ms > 0 else 0.0
    pk = peaks()
    stage_ms = {k: agg[k] for k in ("halves_ms", "join_ms", "env_finish_ms", "factorize_ms", "gauge_ms")}
    dominant = max(stage_ms, key=stage_ms.get)
    # plain FP32 CUDA-core contractions: ALU bound, peak = 152 SMs x 128 FP32 FMA x 2 x 2.07 GHz
    fp32_alu_peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    if args.precision in ("fp32", "fp64"):
        peak = fp32_alu_peak if args.precision == "fp32" else 152 * 2 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": round(local_tflops, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(local_tflops / peak, 4), "traffic": None,
                "kernel": "contraction chain (halves + two-site join + environment finish)",
                "peak_source": "derived: 152 SMs x FMA lanes x 2 x max SM clock"}
    else:
        peak = pk.get("bf16_tflops", 1900.0) / (2.0 if args.precision == "tf32" else 1.0)
        roof = {"bound": "tensor", "achieved": round(local_tflops, 3), "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(local_tflops / peak, 4), "traffic": None,
                "kernel": "contraction chain (halves + two-site join + environment finish)",
                "peak_source": "MEASURED_PEAKS.json bf16 burst" + (" / 2 (tf32 nominal ratio)" if args.precision == "tf32" else "")}
    last_rep, last_sweeps = reps[-1]
    out = {
        "metric": METRIC, "value": round(t_step, 4), "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_step * 1e3, 2), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "tf32": "tf32",
                                                           "bf16_split": "bf16x3"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: L=30, d=2x2, K=128 Kronecker terms (w=0.8^k), chi_A=chi_B=128, "
                               f"chi_C=128, randomized update k=chi_C+{OVERSAMPLE}, conv tol {TOL:g}, "
                               f"max {MAX_SWEEPS} sweeps, site gauge",
                   "precision": args.precision, "parallelism": f"replicas x{world} (independent MPO pairs)",
                   "l2": "flushed between timed steps (256 MB write)"},
        "local_update_tflops": round(local_tflops, 3),
        "sweeps_to_tol": last_sweeps, "converged": bool(last_rep["converged"]), "final_delta": last_rep["delta"],
        "stage_ms_per_fit": {k: round(v, 3) for k, v in stage_ms.items()}, "dominant_stage": dominant,
        "roofline": roof, "clocks": clk, "e2e": e2e,
        "gpu_launches": int(agg["launches"]), "fits_per_s": round(world / t_step, 4),
        "wall_s_timed": round(wall, 2),
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(last_sweeps)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------- oracle timing
def _oracle_windows(n_windows: int, seed: int = 0):
    """Time the oracle's per-window work (two-site tensor, randomized SVD, environment)
    on bulk-shaped tensors of the workload (chi = 128, d = 2)."""
    import numpy as np
    from oracle.fit import keep_rank, left_env, local_tensor, randomized_svd
    from oracle import philox
    rng = np.random.default_rng(seed)
    chi, d = CHI, 2
    Lenv = rng.standard_normal((chi, chi, chi))
    Renv = rng.standard_normal((chi, chi, chi))
    A1, A2, B1, B2 = (rng.standard_normal((chi, d, d, chi)) for _ in range(4))
    t0 = time.perf_counter()
    for w in range(n_windows):
        Th = local_tensor(Lenv, A1, B1, A2, B2, Renv)
        M = Th.reshape(chi * d * d, -1)
        U, S, Vt = randomized_svd(M, chi + OVERSAMPLE, 0, philox.omega_stream(0, w + 1))
        k = keep_rank(S, float(np.linalg.norm(M)), TOL, L_SITES, chi, 1e-13)
        Cl = U[:, :k].reshape(chi, d, d, k)
        left_env(Lenv, A1, B1, Cl)
    return (time.perf_counter() - t0) / n_windows


def cpu_baseline(sweeps: int):
    n = 2
    per_window = _oracle_windows(n)
    est = per_window * (L_SITES - 1) * sweeps
    return {"value": round(est, 2), "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} bulk windows (chi=128, d=2: two-site tensor, randomized SVD, environment) on random "
                      f"tensors of the workload's shapes, {per_window:.2f} s/window, scaled to "
                      f"{L_SITES - 1} windows x {sweeps} sweeps (input preparation not included)"}


def reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    times = []
    for _ in range(args.warmup):
        _oracle_windows(1)
    for _ in range(args.steps):
        times.append(_oracle_windows(1) * (L_SITES - 1) * 3)
    v = statistics.mean(times)
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v * 1e3, 1), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{WORKLOAD} (oracle, bounded sample)", "precision": "fp64"},
           "cpu_baseline": {"value": round(v, 3), "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"1 bulk window per step scaled to {L_SITES - 1} windows x 3 sweeps"},
           "e2e": {"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        reference(a)
    else:
        native(a)
