#!/usr/bin/env python3
"""Benchmark of the variational MPO-MPO fit on one GB300 (or N independent ones).

Workload (the timed configuration): two MPOs on L = 30 sites, local dims 2x2,
each a sum of 128 Kronecker products of 2x2 Gaussian factors with weights
0.8^k (bond 128 after exact trimming), fitted to chi_C = 128 with the
Gaussian-sketch randomized update (oversampling 10) until the relative change
of ||C||^2 between sweeps is <= 1e-8. A step is one complete fit: input
preparation, initial guess and right environments, sweeps until converged, and
the export of C. The default precision schedule runs cheap sweeps first and
exact ones last: one sweep of 3xTF32 tensor-core contractions with the FP32
factorisation, then FP64-class double-FP32
contractions (on the FP32 pipes) with the FP64-polished factorisation to
convergence. Metric: time-to-tol in seconds
(lower is better), reported with the local-update TFLOP/s and a roofline entry
for the dominant stage.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (bulk windows), scaled to the fit's window count.
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
L_SITES, CHI, OVERSAMPLE, TOL, MAX_SWEEPS = 30, 128, 10, 1e-8, 14
LO_SWEEPS = 1  # default: cheap sweeps before the FP64-class ones
SCHEDULE = "tf32x3>bf16_split"  # default precision schedule of the timed fit


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--precision", default=os.environ.get("TTFIT_BENCH_PRECISION", SCHEDULE),
                   help='a precision ("fp64", "df32", "fp32", "tf32x3", ...) or a schedule "lo>hi"')
    p.add_argument("--lo-sweeps", type=int, default=LO_SWEEPS,
                   help="sweeps (>= 1) in the cheap precision of a 'lo>hi' schedule before the switch")
    p.add_argument("--workload", default=WORKLOAD,
                   help="synthetic workload (default: the timed one); smaller ones serve profiling captures")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-accuracy", action="store_true", help="skip the (untimed) FP64 reference fit")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the measurements of the other configurations (segments, configs 2, 4, 5)")
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
def rel_frobenius(X, Y) -> float:
    """||X - Y||_F / ||Y||_F for two MPOs (torch, FP64 on their device): the direct-sum MPO
    X (+) (-Y) and Y are left-orthogonalised by QR and the norms read off their last cores."""
    import torch

    def norm_of(cores):
        R = None
        for l, c in enumerate(cores):
            D = c if R is None else torch.tensordot(R, c, dims=([1], [0]))
            if l == len(cores) - 1:
                return float(torch.linalg.norm(D))
            a0, d, dp, a1 = D.shape
            _, R = torch.linalg.qr(D.reshape(a0 * d * dp, a1))

    L = len(X)
    S = []
    for l in range(L):
        x, y = X[l].double(), Y[l].double()
        if l == 0:
            S.append(torch.cat([x, -y], dim=3))
        elif l == L - 1:
            S.append(torch.cat([x, y], dim=0))
        else:
            a0, d, dp, a1 = x.shape
            b0, _, _, b1 = y.shape
            Z = torch.zeros((a0 + b0, d, dp, a1 + b1), dtype=torch.float64, device=x.device)
            Z[:a0, :, :, :a1] = x
            Z[a0:, :, :, a1:] = y
            S.append(Z)
    return norm_of(S) / norm_of([y.double() for y in Y])


STAGES = ("halves_ms", "join_ms", "env_finish_ms", "factorize_ms", "gauge_ms", "contraction_flops", "launches",
          "tc_issued_flops", "cc_issued_flops")
# peaks of the plain CUDA-core pipes (ALU bound): 152 SMs x FMA lanes per SM x 2 flop x max SM clock
FMA_LANES = {"f64": 2, "f32": 128}
DF32_INSTR = 15  # FP32 instructions of one double-FP32 multiply-add (csrc/common.cuh, madd)


def run_fit(ttfit, Ain, Bin, schedule, seed, dev, stream, chi=CHI, lo_sweeps=LO_SWEEPS, init="random", ab_rank=0):
    """One complete fit. ``schedule`` is a precision name ("fp64", "df32", "tf32x3", ...) for a
    single-precision fit, or "lo>hi", e.g. "tf32x3>df32": sweeps in ``lo`` (FP32-factorised
    randomized update) for ``lo_sweeps`` sweeps, then FP64-class contractions in ``hi`` with the
    FP64-polished FP32 factorisation until converged."""
    import torch
    lo, hi = (schedule.split(">") + [None])[:2]
    ev = {k: torch.cuda.Event(enable_timing=True) for k in ("c0", "c1", "s0", "s1", "r0", "r1")}
    ev["c0"].record(stream)
    f = ttfit.tt_fit_create(Ain, Bin, chi, TOL, "site", update="rsvd", oversample=OVERSAMPLE, seed=seed,
                            precision=lo, device=dev, stream=stream, init=init, ab_rank=ab_rank)
    ev["c1"].record(stream)
    switched = False
    phases = {lo: {k: 0.0 for k in STAGES}}
    phase_sweeps = {lo: 0}
    cur, sweeps, rep = lo, 0, None
    history = []
    while sweeps < MAX_SWEEPS:
        rep = f.sweep(1)
        sweeps += 1
        history.append(rep["delta"])
        phase_sweeps[cur] += 1
        st = f.stage_times()
        ex = f.exec_flops()
        st["tc_issued_flops"], st["cc_issued_flops"] = ex["tensor_core"], ex["cuda_core"]
        for k in STAGES:
            phases[cur][k] += st[k]
        if rep["converged"] and (hi is None or cur == hi):
            break
        if hi is not None and cur == lo and sweeps >= lo_sweeps:
            ev["s0"].record(stream)
            f.set_precision(hi, fast_factor=True)
            ev["s1"].record(stream)
            switched = True
            cur = hi
            phases[hi] = {k: 0.0 for k in STAGES}
            phase_sweeps[hi] = 0
    ev["r0"].record(stream)
    C = f.result()
    ev["r1"].record(stream)
    ev["r1"].synchronize()
    rep["host_ms"] = {"create": ev["c0"].elapsed_time(ev["c1"]),
                      "switch": ev["s0"].elapsed_time(ev["s1"]) if switched else 0.0,
                      "export": ev["r0"].elapsed_time(ev["r1"])}
    launches = f.launch_count()
    rep["jacobi_max_sweeps"] = f.jacobi_sweeps()
    rep["bonds"] = f.bonds()
    f.destroy()
    rep["history"] = history
    return rep, sweeps, phase_sweeps, phases, C, launches


def dist_env():
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 when run alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, world, device):
    """The largest x over the ranks: a step takes as long as its slowest replica."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank):
    """Rank r fits its own, independent MPO pair: the workload drawn with seed r."""
    return int(rank)


def local_update_roof(flops, ms, pk, bf16_digits=False):
    """The local update (halves, join, environment finish: minimal algorithmic flops over their summed
    event time) against the dense TF32 tensor rate, half the measured (else fallback) sustained bf16
    rate; against the bf16 rate itself when the FP64-class sweeps put their digit products on the
    BF16 tensor cores. The DF32 sweeps count FP64-class flops, each of which takes 21 digit products."""
    if ms <= 0:
        return None
    src = "of measured" if "bf16_tflops_sustained" in pk else "of fallback (1.7 PFLOP/s bf16 sustained)"
    bf16 = pk.get("bf16_tflops_sustained", 1700.0)
    peak = bf16 if bf16_digits else bf16 / 2.0
    tf = flops / (ms * 1e-3) / 1e12
    return {"tflops": round(tf, 3), "peak": round(peak, 1), "unit": "TFLOP/s", "frac": round(tf / peak, 4),
            "peak_source": f"bf16 sustained, {src}" if bf16_digits else f"TF32 = bf16 sustained / 2, {src}"}


def native(args):
    import torch
    import torch.distributed as dist
    from paper_2606_23274_gb300 import ttfit
    from paper_2606_23274_gb300.synth import mpo_pair

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    ttfit.load()

    # inputs resident in HBM before the timed region; rank r fits its own pair
    from paper_2606_23274_gb300.synth import WORKLOADS
    chi = WORKLOADS[args.workload]["chi_C"]
    A, B = mpo_pair(args.workload, seed=replica_seed(rank))
    Ad = [torch.from_numpy(a).to(dev) for a in A]
    Bd = [torch.from_numpy(b).to(dev) for b in B]
    Ah = [torch.from_numpy(a).pin_memory() for a in A]
    Bh = [torch.from_numpy(b).pin_memory() for b in B]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        run_fit(ttfit, Ad, Bd, args.precision, rank, dev, stream, chi, args.lo_sweeps)
        flush.zero_()
    barrier()
    clocks = ClockSampler(local)
    times, results = [], []
    t_wall0 = time.time()
    for _ in range(args.steps):
        flush.zero_()                       # L2 flushed between timed steps
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = run_fit(ttfit, Ad, Bd, args.precision, rank, dev, stream, chi, args.lo_sweeps)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        results.append(res)
    barrier()
    wall = time.time() - t_wall0
    clk = clocks.stop()
    t_step = max_over_ranks(statistics.mean(times), world, dev)

    e2e = None
    if not args.no_e2e:
        # the public API end to end: pinned host inputs -> device, the fit, C -> host
        et, h2d, d2h = [], 0, 0
        for _ in range(max(1, min(args.steps, 2))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Ain = [a.to(dev, non_blocking=True) for a in Ah]
            Bin = [b.to(dev, non_blocking=True) for b in Bh]
            _, _, _, _, C, _ = run_fit(ttfit, Ain, Bin, args.precision, rank, dev, stream, chi, args.lo_sweeps)
            Ch = [c.to("cpu") for c in C]
            torch.cuda.synchronize()
            et.append(time.perf_counter() - t0)
            h2d = sum(a.numel() * a.element_size() for a in Ah + Bh)
            d2h = sum(c.numel() * c.element_size() for c in Ch)
        e2e = {"value": round(statistics.mean(et), 4), "unit": "s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # accuracy of the timed fit (untimed): relative Frobenius distance of its C to the FP64 fit (FP64
    # contractions and factorisation, the path pinned to the oracle) of the same inputs, seed and sweep
    # count, by the stable difference norm (direct-sum MPO, QR sweep in FP64 on the device)
    accuracy = None
    if not args.no_accuracy:
        _, sw_t, _, _, C_t, _ = results[-1]
        g = ttfit.tt_fit_create(Ad, Bd, chi, TOL, "site", update="rsvd", oversample=OVERSAMPLE, seed=rank,
                                precision="fp64", device=dev, stream=stream, conv_tol=0.0)
        g.sweep(sw_t)
        C_ref = g.result()
        g.destroy()
        accuracy = {"rel_frobenius_vs_fp64_fit": float(f"{rel_frobenius(C_t, C_ref):.3e}"),
                    "reference": f"FP64 contractions + FP64 factorisation fit, same inputs, seed and sweep count "
                                 f"({sw_t}); that path matches the FP64 oracle to ~1e-12 in ||C||^2 at this size",
                    "bound": 1e-6}

    # live per-stage times: CUDA events recorded by the library on the caller's stream, inside the
    # timed steps, accumulated per precision phase and averaged over the steps
    names = list(results[0][3].keys())
    agg = {p: {k: statistics.mean(r[3][p][k] for r in results) for k in STAGES} for p in names}
    pk = peaks()
    mhz = pk.get("sm_max_mhz", 2070.0)
    rows = []
    for p in names:
        a = agg[p]
        chain_ms = a["halves_ms"] + a["join_ms"] + a["env_finish_ms"]
        rows.append((chain_ms, p, "chain", a["contraction_flops"]))
        rows.append((a["factorize_ms"], p, "factorize", 0.0))
        rows.append((a["gauge_ms"], p, "gauge", 0.0))
    dom_ms, dom_phase, dom_stage, dom_flops = max(rows)
    if dom_stage == "chain":
        tflops = dom_flops / (dom_ms * 1e-3) / 1e12
        if dom_phase in ("fp64", "fp32"):
            dt = "f64" if dom_phase == "fp64" else "f32"
            peak = 152 * FMA_LANES[dt] * 2 * mhz * 1e6 / 1e12
            roof = {"bound": "alu", "achieved": round(tflops, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
                    "frac": round(tflops / peak, 4), "traffic": None,
                    "kernel": f"gemm_simt_kernel<{'double' if dt == 'f64' else 'float'}> (contraction chain, "
                              f"{dom_phase} phase)",
                    "peak_source": f"derived: 152 SMs x {FMA_LANES[dt]} {dt} FMA/clk x 2 x {mhz:.0f} MHz"}
        elif dom_phase == "df32":
            # a double-FP32 multiply-add issues DF32_INSTR FP32 instructions (exact product, cross terms,
            # two-sum, renormalisation); the ceiling is the FP32 issue rate divided by that
            peak = 152 * FMA_LANES["f32"] * 2 * mhz * 1e6 / DF32_INSTR / 1e12
            roof = {"bound": "alu", "achieved": round(tflops, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
                    "frac": round(tflops / peak, 4), "traffic": None,
                    "kernel": "gemm_simt_kernel<df32> (contraction chain, df32 phase)",
                    "peak_source": f"derived: 152 SMs x 128 FP32 lanes x {mhz:.0f} MHz / {DF32_INSTR} instructions "
                                   f"per multiply-add, x 2 flop"}
        else:
            bf16 = pk.get("bf16_tflops_sustained", 1700.0)
            ratio = 2.0 if dom_phase == "tf32" else 6.0       # TF32 is half the bf16 rate; 3xTF32 issues 3 MMAs
            peak = bf16 / ratio
            roof = {"bound": "tensor", "achieved": round(tflops, 3), "peak": round(peak, 1), "unit": "TFLOP/s",
                    "frac": round(tflops / peak, 4), "traffic": None,
                    "kernel": f"gemm_tf32_kernel (contraction chain, {dom_phase} phase)",
                    "peak_source": f"of measured: bf16 sustained / {ratio:g}"}
    elif dom_stage == "factorize":
        # algorithmic work of the randomized factorisation of one m x n window with sketch width k:
        # Y = M Omega and B^T = M^T Q (2 m n k each), Householder QR of Y and of B^T with Q formed
        # (4 m k^2 - 4/3 k^3 each), SVD of the k x k factor with both bases (~21 k^3, Golub-Kahan count),
        # U = Q Vr and V = Q2 Ur (2 m k^2 + 2 n k^2); windows with k >= min(m, n) take the exact SVD
        # (at most 4 per sweep, ends of the chain) and are not counted
        b = results[-1][0]["bonds"]
        ks = CHI + OVERSAMPLE
        per_sweep = 0.0
        for l in range(len(b) - 3):
            m, n = b[l] * 4, 4 * b[l + 2]
            if ks < min(m, n):
                per_sweep += 4.0 * m * n * ks + 4.0 * m * ks ** 2 + 4.0 * n * ks ** 2 - 8.0 / 3 * ks ** 3 \
                    + 21.0 * ks ** 3 + 2.0 * m * ks ** 2 + 2.0 * n * ks ** 2
        sweeps_in = statistics.mean(r[2][dom_phase] for r in results)
        tflops = per_sweep * sweeps_in / (dom_ms * 1e-3) / 1e12
        peak = 152 * FMA_LANES["f32"] * 2 * mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": round(tflops, 4), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(tflops / peak, 5), "traffic": None,
                "kernel": f"factorisation stage ({dom_phase} phase): qr_cluster_blocked_kernel<float> x2, "
                          "jacobi_cluster_kernel<float>, sketch GEMMs, per window",
                "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz (the cluster kernels occupy 8 "
                               "SMs and are bound by the latency of their sequential steps)"}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None, "traffic": None,
                "kernel": f"{dom_stage} ({dom_phase} phase)"}
    local_flops = sum(agg[p]["contraction_flops"] for p in names)
    tc_issued = sum(agg[p]["tc_issued_flops"] for p in names)
    cc_issued = sum(agg[p]["cc_issued_flops"] for p in names)
    local_ms = sum(agg[p]["halves_ms"] + agg[p]["join_ms"] + agg[p]["env_finish_ms"] for p in names)
    rep, sweeps, phase_sweeps, _, _, launches = results[-1]
    dtypes = {"fp64": "f64", "fp32": "f32", "tf32": "tf32", "tf32x3": "tf32x3", "df32": "f32x2",
              "bf16_split": "f32x2 (bf16 digit products)"}
    out = {
        "metric": METRIC, "value": round(t_step, 4), "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_step * 1e3, 2), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "+".join(dtypes.get(p, p) for p in names),
        "data": "synthetic",
        "config": {"workload": (f"{WORKLOAD}: L=30, d=2x2, K=128 Kronecker terms (w=0.8^k), chi_A=chi_B=128, "
                               f"chi_C=128, randomized update k=chi_C+{OVERSAMPLE}, conv tol {TOL:g} on the "
                               f"relative change of ||C||^2, max {MAX_SWEEPS} sweeps, site gauge") if args.workload == WORKLOAD else args.workload,
                   "schedule": args.precision + (f" ({args.lo_sweeps} cheap sweeps)" if ">" in args.precision else ""), "parallelism": f"replicas x{world} (independent MPO pairs)",
                   "l2": "flushed between timed steps (256 MB write)"},
        "sweeps_to_tol": sweeps, "sweeps_per_phase": phase_sweeps, "converged": bool(rep["converged"]),
        "final_delta": rep["delta"], "norm2_C": rep["norm2_C"],
        "delta_history": [float(f"{d:.3e}") if d != float("inf") else None for d in rep["history"]],
        "local_update_tflops": round(local_flops / (local_ms * 1e-3) / 1e12, 3) if local_ms > 0 else None,
        "local_update": local_update_roof(local_flops, local_ms, pk, bf16_digits="bf16_split" in names),
        "local_update_as_issued": {
            "algorithmic_tflop_per_fit": round(local_flops / 1e12, 4),
            "tensor_core_mma_tflop_per_fit": round(tc_issued / 1e12, 4),
            "cuda_core_tflop_per_fit": round(cc_issued / 1e12, 4),
            "issued_tensor_tflops": round(tc_issued / (local_ms * 1e-3) / 1e12, 2) if local_ms > 0 else None,
            "note": "MMA flops as the tensor cores executed them (128 x 128 tiles, K per k-block, 3 passes for "
                    "3xTF32, 21 digit pairs for the FP64-class digit split) over the same stage time as "
                    "local_update; the algorithmic count credits none of that"},
        "stage_ms_per_fit": {p: {k: round(agg[p][k], 2) for k in STAGES[:5]} for p in names},
        "create_switch_export_ms": {k: round(statistics.mean(r[0]["host_ms"][k] for r in results), 2)
                                    for k in ("create", "switch", "export")},
        "roofline": roof, "clocks": clk, "e2e": e2e, "gpu_launches": int(sum(r[5] for r in results)), "gpu_launches_per_step": int(launches),
        "fits_per_s": round(world / t_step, 4), "wall_s_timed": round(wall, 2),
        "jacobi_max_sweeps": rep.get("jacobi_max_sweeps"),
        "accuracy": accuracy,
    }
    if rank == 0 and not args.no_extras and args.workload == WORKLOAD:
        try:
            out["extras"] = extras(ttfit, dev, stream, out["norm2_C"])
        except Exception as e:  # the timed line stands on its own; report what stopped the extras
            out["extras"] = {"error": f"{type(e).__name__}: {e}"[:500]}
    if rank == 0 and not args.no_cpu_baseline and args.workload == WORKLOAD:
        out["cpu_baseline"] = cpu_baseline(sweeps)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------- other configurations
def _timed(stream, fn):
    """fn() bracketed by CUDA events on `stream` (seconds), and its result."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    r = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3, r


def _segment_fit(ttfit, A, B, dev, stream, n_seg, edge_extra=0, gauge="inverse"):
    """The timed workload, serial (n_seg = 1) or segment-parallel (Alg. 6): one cheap 3xTF32
    pass (a full set of local sweeps when segmented), then DF32 until delta <= TOL, with
    the FP32 factorisation in the inverse gauge and the FP64 one in the site gauge (whose
    segments are merged before the switch and at the end, Sec. 4.5)."""
    site = gauge == "site" and n_seg > 1

    def run():
        f = ttfit.tt_fit_create(A, B, CHI, TOL, gauge, update="rsvd", oversample=OVERSAMPLE, seed=0,
                                precision="tf32x3", device=dev, stream=stream, n_segments=n_seg,
                                edge_extra=edge_extra)
        per_set = 2 if n_seg > 1 else 1
        f.sweep(per_set)
        if site:
            f.merge()
        f.set_precision("df32", fast_factor=0 if site else 1)
        n, rep = per_set, None
        while n < MAX_SWEEPS * per_set:
            rep = f.sweep(1)
            n += 1
            if rep["converged"]:
                break
        if site:
            rep = f.merge()
        f.destroy()
        return rep, n
    run()  # warm-up
    t, (rep, n) = _timed(stream, run)
    return t, rep, n


def extras(ttfit, dev, stream, norm2_site):
    """One measured run each (after a warm-up) of: the segment-parallel fit of the timed
    workload (Sec. 4, Alg. 6); plain FP32 vs mixed precision at equal accuracy (config 2:
    L=20, chi=64); 32 uneven independent pairs plus an L=64, chi=128 chain in 8 segments
    (config 4); the adjoint at L=32, chi=96 (config 5)."""
    import numpy as np
    import torch
    from paper_2606_23274_gb300.synth import gaussian_mpo, kron_sum_mpo, mpo_pair
    out = {}
    # segment-parallel fit of the timed workload
    A, B = mpo_pair(WORKLOAD, seed=0)
    A = [torch.from_numpy(a).to(dev) for a in A]
    B = [torch.from_numpy(b).to(dev) for b in B]
    seg = {}
    for n_seg, ee in ((1, 0), (2, 0), (4, 2), (8, 2)):
        t, rep, n = _segment_fit(ttfit, A, B, dev, stream, n_seg, ee)
        seg[str(n_seg)] = {"time_to_tol_s": round(t, 4), "sweeps_or_phases": n, "converged": bool(rep["converged"]),
                           "delta": rep["delta"], "norm2_rel_to_site_fit": rep["norm2_C"] / norm2_site - 1.0,
                           "edge_extra": ee}
    seg["schedule"] = "tf32x3>df32 (TF32 digit planes)"
    out["segments_inverse_gauge_L30_chi128"] = seg
    seg = {}
    for n_seg, ee in ((2, 0), (4, 2), (8, 2)):
        t, rep, n = _segment_fit(ttfit, A, B, dev, stream, n_seg, ee, gauge="site")
        seg[str(n_seg)] = {"time_to_tol_s": round(t, 4), "phases": n, "converged": bool(rep["converged"]),
                           "delta": rep["delta"], "norm2_rel_to_site_fit": rep["norm2_C"] / norm2_site - 1.0,
                           "edge_extra": ee, "merges": 2}
    seg["schedule"] = "tf32x3>df32 (TF32 digit planes), FP64 factorisation after the switch"
    out["segments_site_gauge_L30_chi128"] = seg

    # config 2: plain FP32 (FP32 CUDA-core contractions, FP32 SVD) vs mixed (3xTF32, then DF32 with the
    # FP64 SVD), both the exact two-site update; error = relative Frobenius distance to the converged FP64 fit
    A2, B2 = mpo_pair("kron_L20_chi64", seed=0)
    A2 = [torch.from_numpy(a).to(dev) for a in A2]
    B2 = [torch.from_numpy(b).to(dev) for b in B2]
    g = ttfit.tt_fit_create(A2, B2, 64, 1e-8, "site", precision="fp64", device=dev, stream=stream, conv_tol=1e-13)
    g.sweep(14)
    C_ref = g.result()
    g.destroy()

    def trace(schedule):
        lo, hi = (schedule.split(">") + [None])[:2]
        f = ttfit.tt_fit_create(A2, B2, 64, 1e-8, "site", precision=lo, device=dev, stream=stream, conv_tol=0.0)
        t_cum, pts = 0.0, []
        for s in range(12):
            if hi is not None and s == 1:
                dt, _ = _timed(stream, lambda: f.set_precision(hi, fast_factor=0))
                t_cum += dt
            dt, _ = _timed(stream, lambda: f.sweep(1))
            t_cum += dt
            pts.append((t_cum, rel_frobenius(f.result(), C_ref)))
        f.destroy()
        return pts
    trace("fp32")  # warm-up
    plain = trace("fp32")
    mixed = trace("tf32x3>df32")
    best = min(e for _, e in plain)
    t_plain = next(t for t, e in plain if e <= 1.05 * best)
    t_mixed = next((t for t, e in mixed if e <= best), None)
    out["config2_plain_fp32_vs_mixed_L20_chi64"] = {
        "accuracy_target": float(f"{best:.3e}"), "note": "the plain FP32 fit's best relative Frobenius error "
        "(to the converged FP64 fit) over 12 sweeps; each fit timed until it first reaches it",
        "plain_fp32_s": round(t_plain, 4), "mixed_s": round(t_mixed, 4) if t_mixed else None,
        "speedup": round(t_plain / t_mixed, 2) if t_mixed else None,
        "mixed_final_error": float(f"{mixed[-1][1]:.3e}"),
        "plain_errors": [float(f"{e:.2e}") for _, e in plain], "mixed_errors": [float(f"{e:.2e}") for _, e in mixed]}

    # config 4: 32 pairs with uneven L and chi, and one L = 64, chi = 128 chain in 8 segments
    rng = np.random.default_rng(4)
    Ls = rng.integers(16, 65, size=32)
    chis = rng.choice([16, 32, 64, 96, 128], size=32)
    pairs = [([torch.from_numpy(a).to(dev) for a in kron_sum_mpo(int(L), int(c), 100 + i, 0)],
              [torch.from_numpy(b).to(dev) for b in kron_sum_mpo(int(L), int(c), 100 + i, 1)])
             for i, (L, c) in enumerate(zip(Ls, chis))]
    Ac = [torch.from_numpy(a).to(dev) for a in kron_sum_mpo(64, 128, 99, 0)]
    Bc = [torch.from_numpy(b).to(dev) for b in kron_sum_mpo(64, 128, 99, 1)]
    kw = dict(update="rsvd", oversample=OVERSAMPLE, seed=0, precision="tf32x3", device=dev, stream=stream)

    def batch():
        fits = ttfit.tt_fit_create_batched(pairs, [int(c) for c in chis], 0.0, "inverse", conv_tol=0.0, **kw)
        fits += ttfit.tt_fit_create_batched([(Ac, Bc)], [128], 0.0, "inverse", n_segments=8, edge_extra=3,
                                            conv_tol=0.0, **kw)
        t_s, reps = _timed(stream, lambda: ttfit.tt_fit_sweep_batched(fits, 4))
        flops = sum(f.stage_times()["contraction_flops"] for f in fits)
        for f in fits:
            f.destroy()
        return t_s, reps, flops
    batch()  # warm-up (fills the block cache)
    t_all, (t_s, reps, flops) = _timed(stream, batch)
    windows = int(sum(int(L) - 1 for L in Ls) * 4 + 63 * 2)
    out["config4_batched_32_pairs_plus_L64_chi128_8_segments"] = {
        "pairs": 32, "L": [int(x) for x in Ls], "chi": [int(x) for x in chis], "precision": "tf32x3 (FP32-class)",
        "gauge": "inverse", "sweeps": "4 per pair; 4 phases (2 full sets) for the segmented chain",
        "sweep_wall_s": round(t_s, 4), "create_sweep_destroy_s": round(t_all, 4),
        "windows_per_s": round(windows / t_s, 1),
        "contraction_tflops_last_call": round(flops / t_s / 1e12, 3),
        "concurrency": "one host thread and CUDA stream per handle (and per segment); no single persistent launch"}

    # config 5: the adjoint at L = 32, chi_A = chi_B = chi_C = 96, W of chi = 32, FP32
    A5 = [torch.from_numpy(a).to(dev) for a in kron_sum_mpo(32, 96, 5, 0)]
    B5 = [torch.from_numpy(b).to(dev) for b in kron_sum_mpo(32, 96, 5, 1)]
    C5 = [torch.from_numpy(c).to(dev) for c in gaussian_mpo(32, 2, 96, 5, 2)]
    W5 = [torch.from_numpy(w).to(dev) for w in gaussian_mpo(32, 2, 32, 5, 3)]
    res5 = {}
    for prec in ("fp32", "tf32x3"):
        for target, X in (("residual", C5), ("inner", W5)):
            ttfit.tt_mpo_grad(A5, B5, X, target, prec, 0, stream=stream)  # warm-up
            t, _ = _timed(stream, lambda: ttfit.tt_mpo_grad(A5, B5, X, target, prec, 0, stream=stream))
            res5[f"{target}_{prec}"] = round(t, 4)
    out["config5_adjoint_L32_chi96_s"] = res5

    # the zip-up contraction (Alg. 2) of the timed workload, alone and as the fit's initial guess
    # (Sec. 2.3.5), against the random guess of the timed fit
    zu = {}
    for prec in ("tf32x3", "fp64"):
        kwz = dict(update="rsvd", oversample=OVERSAMPLE, seed=0, precision=prec, stream=stream, device=dev)
        ttfit.tt_mpo_zipup(A, B, CHI, TOL, **kwz)  # warm-up
        t, Cz = _timed(stream, lambda: ttfit.tt_mpo_zipup(A, B, CHI, TOL, **kwz))
        zu[f"zipup_{prec}_s"] = round(t, 4)
        zu[f"zipup_{prec}_norm2_rel_to_site_fit"] = float(f"{sum_sq(Cz) / norm2_site - 1.0:.3e}")
    for init in ("zipup", "random"):
        run_fit(ttfit, A, B, SCHEDULE, 0, dev, stream, init=init)  # warm-up
        t, (rep, sweeps, _, _, _, _) = _timed(stream, lambda: run_fit(ttfit, A, B, SCHEDULE, 0, dev, stream,
                                                                       init=init))
        zu[f"fit_from_{init}"] = {"time_to_tol_s": round(t, 4), "sweeps": sweeps, "converged": bool(rep["converged"]),
                                  "norm2_rel_to_site_fit": float(f"{rep['norm2_C'] / norm2_site - 1.0:.3e}"),
                                  "delta_history": [float(f"{d:.3e}") if d != float("inf") else None
                                                    for d in rep["history"]]}
    out["zipup_L30_chi128"] = zu

    # randomized bond projection of A and B (Sec. 3.2) to rank k, the default schedule; error relative
    # to the unprojected fit of the same schedule
    _, _, _, _, C_full, _ = run_fit(ttfit, A, B, SCHEDULE, 0, dev, stream)
    pr = {}
    for k in (32, 64, 96):
        run_fit(ttfit, A, B, SCHEDULE, 0, dev, stream, ab_rank=k)  # warm-up
        t, (rep, sweeps, _, phases, C_k, _) = _timed(stream, lambda: run_fit(ttfit, A, B, SCHEDULE, 0, dev, stream,
                                                                             ab_rank=k))
        chain_ms = sum(ph["halves_ms"] + ph["join_ms"] + ph["env_finish_ms"] for ph in phases.values())
        pr[str(k)] = {"time_to_tol_s": round(t, 4), "sweeps": sweeps, "converged": bool(rep["converged"]),
                      "chain_ms": round(chain_ms, 2),
                      "rel_frobenius_vs_unprojected": float(f"{rel_frobenius(C_k, C_full):.3e}")}
    out["bond_projection_L30_chi128"] = pr
    return out


def sum_sq(C) -> float:
    """||C||_F^2 of an MPO on the device (FP64 left-orthogonalisation, QR per site)."""
    import torch
    M = None
    for c in C:
        c = c.double()
        a0, d, dp, a1 = c.shape
        X = c.reshape(a0, -1) if M is None else M @ c.reshape(a0, -1)
        X = X.reshape(-1, a1)
        _, R = torch.linalg.qr(X)
        M = R
    return float(torch.sum(M * M))


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


THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def _time_window_subprocess(threads):
    """Seconds of one bulk window of the oracle, in a fresh interpreter with `threads`
    BLAS/OpenMP threads (None: the library default, all cores)."""
    env = dict(os.environ)
    for v in THREAD_VARS:
        if threads is None:
            env.pop(v, None)
        else:
            env[v] = str(threads)
    code = "import sys; sys.path.insert(0, %r); import bench; print(bench._oracle_windows(1))" % ROOT
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return float(r.stdout.strip().splitlines()[-1])


def cpu_baseline(sweeps: int):
    """The oracle on the host cores: one bulk window (two-site tensor, randomized SVD,
    environment at chi = 128) timed with 1 thread and with all threads, scaled to the fit's
    windows x sweeps. `value` is the all-threads figure."""
    t1 = _time_window_subprocess(1)
    tn = _time_window_subprocess(None)
    n = os.cpu_count()
    scale = (L_SITES - 1) * sweeps
    return {"value": round(tn * scale, 2), "unit": "s", "cores": n, "kind": "oracle",
            "single_thread": {"value": round(t1 * scale, 2), "cores": 1},
            "sample": f"1 bulk window (chi=128, d=2: two-site tensor, randomized SVD, environment) on random "
                      f"tensors of the workload's shapes, timed once with 1 thread ({t1:.2f} s) and once with "
                      f"all {n} threads ({tn:.2f} s), scaled to {L_SITES - 1} windows x {sweeps} sweeps "
                      f"(factor {scale}); input preparation not included"}


def reference(args):
    """The FP64 oracle on the host cores. A step is one bulk window of the workload, measured;
    `value` is that window time scaled to a full fit (29 windows x 3 sweeps), and ms_per_step is
    the measured per-step time of the sample itself."""
    if dist_env()[1] != 0:  # under torchrun the other ranks exit without work
        return
    windows, sweeps = L_SITES - 1, 3
    for _ in range(args.warmup):
        _oracle_windows(1)
    t0 = time.perf_counter()
    per = [_oracle_windows(1) for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    w = statistics.mean(per)
    v = w * windows * sweeps
    n = os.cpu_count()
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(w * 1e3, 1), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{WORKLOAD} (oracle, one bulk window per step)", "precision": "fp64"},
           "extrapolation": {"measured_s_per_window": round(w, 3), "windows_per_sweep": windows, "sweeps": sweeps,
                             "factor": windows * sweeps, "timed_wall_s": round(wall, 2)},
           "cpu_baseline": {"value": round(v, 3), "unit": "s", "cores": n, "kind": "oracle",
                            "sample": f"1 bulk window per step (measured {w:.2f} s, all {n} threads), scaled to "
                                      f"{windows} windows x {sweeps} sweeps"},
           "e2e": {"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        reference(a)
    else:
        native(a)
