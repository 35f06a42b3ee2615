"""bench.py's host logic on CPU.

* The multi-GPU mode: one process per rank (gloo, world size 2, 127.0.0.1), each
  fitting its own pair, the step time taken as the maximum over the ranks, and the
  reference arm running on rank 0 only. The data path has no collective; these are
  the only cross-rank steps.
* The reference arm's JSON line.
* The roofline and accuracy helpers behind the bench line."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    from paper_2606_23274_gb300.synth import mpo_pair
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (world, rank, rank)
        # every rank reports its own step time; all of them see the slowest one
        t = bench.max_over_ranks(0.25 + 0.5 * rank, world, "cpu")
        # independent pairs: rank r draws the workload with seed r
        A, _ = mpo_pair("kron_L10_chi16", seed=bench.replica_seed(rank))
        sums = [None] * world
        dist.all_gather_object(sums, float(sum(np.abs(a).sum() for a in A)))
        dist.barrier()
        with open(os.path.join(outdir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{t} {sums[0]} {sums[1]}\n")
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_step_and_fit_distinct_pairs(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    rows = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(world)]
    for row in rows:
        assert float(row[0]) == pytest.approx(0.75)          # the max over ranks, on every rank
        assert float(row[1]) != float(row[2])               # the ranks' pairs differ
    assert rows[0][1:] == rows[1][1:]


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_env() == (1, 0, 0)
        assert bench.max_over_ranks(1.25, 1, "cpu") == 1.25
    finally:
        os.environ.update(env)


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    """Under torchrun the other ranks leave the reference arm without work or output."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    ns = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})()
    assert bench.reference(ns) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_the_contract_line(capsys, monkeypatch):
    """bench.py --impl reference on rank 0: one JSON line with the contract's keys, the oracle timed
    on a bounded sample (one bulk window per step)."""
    sys.path.insert(0, ROOT)
    import json
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    ns = type("A", (), {"steps": 1, "warmup": 0, "gpus": 1})()
    bench.reference(ns)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "s"
    assert d["higher_is_better"] is False and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_local_update_roofline_takes_the_peak_of_the_digit_type():
    """The local-update fraction is taken against the TF32 rate (half of bf16) unless the FP64-class
    sweeps run their digit products on the BF16 tensor cores; without a measured-peaks file the
    recipe's fallback is used and said."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.local_update_roof(1.7e12, 1000.0, {})          # 1.7 TFLOP/s
    assert r["peak"] == 850.0 and r["frac"] == round(1.7 / 850.0, 4) and "fallback" in r["peak_source"]
    r = bench.local_update_roof(1.7e12, 1000.0, {}, bf16_digits=True)
    assert r["peak"] == 1700.0 and r["frac"] == round(1.7 / 1700.0, 4)
    r = bench.local_update_roof(1.7e12, 1000.0, {"bf16_tflops_sustained": 1707.0})
    assert r["peak"] == 853.5 and "of measured" in r["peak_source"]
    assert bench.local_update_roof(1.0, 0.0, {}) is None


def test_accuracy_helpers_match_the_oracle():
    """The bench's accuracy figure (rel_frobenius) and its ||C||^2 check (sum_sq) run in torch on the
    tensors' device; on CPU tensors they agree with the oracle's pinned difference norm and norm."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from oracle.mpo import mpo_diff_norm, mpo_norm
    from paper_2606_23274_gb300.synth import gaussian_mpo
    X = gaussian_mpo(6, 2, 5, 0, 0)
    Y = [y + 1e-3 * x for x, y in zip(gaussian_mpo(6, 2, 5, 0, 1), X)]   # X near Y
    tX = [torch.from_numpy(x) for x in X]
    tY = [torch.from_numpy(y) for y in Y]
    want = mpo_diff_norm(X, Y) / mpo_norm(Y)
    assert abs(bench.rel_frobenius(tX, tY) - want) <= 1e-10 * want
    assert bench.rel_frobenius(tY, tY) <= 1e-14
    assert np.isclose(bench.sum_sq(tX), mpo_norm(X) ** 2, rtol=1e-12)
