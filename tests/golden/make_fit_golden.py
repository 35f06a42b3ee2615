"""Writes the FP64 oracle's reference values for the GPU parity tests of the
randomized fit at the timed configuration's window shapes.

Calls only ``oracle/`` and the seeded input generators of
``paper_2606_23274_gb300.synth`` (which hold none of the fit's arithmetic); no
value here comes from the CUDA path.

For each case it runs the oracle's fit (Alg. 5 with the randomized update of
Sec. 3.1, site gauge) sweep by sweep and records after every sweep:
``norm2`` (the kept weight at the orthogonality centre), ``delta`` and the
bonds; after the sweeps listed in ``--keep``: the kept singular values of every
inner bond and 256 sampled entries <x|C|y> of the fitted operator (row and
column multi-indices drawn from a fixed generator, x_1 most significant), with
||C||_F. Usage:

    python tests/golden/make_fit_golden.py kron_L10_chi128 --sweeps 4 --keep 3 4
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.fit import FitOracle  # noqa: E402
from oracle.mpo import mpo_norm  # noqa: E402
from paper_2606_23274_gb300.synth import WORKLOADS, mpo_pair  # noqa: E402

N_SAMPLES = 256


def sample_indices(L: int, d: int, n: int, seed: int = 12345):
    rng = np.random.default_rng(seed)
    return rng.integers(0, d, size=(n, L)), rng.integers(0, d, size=(n, L))


def entries(C, xs, ys):
    """<x|C|y> = C_1[:, x_1, y_1, :] C_2[:, x_2, y_2, :] ... C_L[:, x_L, y_L, :]."""
    out = []
    for x, y in zip(xs, ys):
        v = np.ones((1,))
        for l, c in enumerate(C):
            v = v @ c[:, x[l], y[l], :]
        out.append(float(v[0]))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--sweeps", type=int, default=4)
    ap.add_argument("--keep", type=int, nargs="+", default=[3, 4])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--oversample", type=int, default=10)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    chi = WORKLOADS[a.workload]["chi_C"]
    A, B = mpo_pair(a.workload, seed=a.seed)
    L = len(A)
    xs, ys = sample_indices(L, A[0].shape[1], N_SAMPLES)
    t0 = time.time()
    f = FitOracle(A, B, chi, a.tol, gauge="site", update="rsvd", oversample=a.oversample, seed=a.seed,
                  sv_cutoff=1e-13, conv_tol=0.0)
    rec = {"workload": a.workload, "chi_max": chi, "tol": a.tol, "oversample": a.oversample, "seed": a.seed,
           "gauge": "site", "update": "rsvd", "sv_cutoff": 1e-13, "sample_seed": 12345,
           "x": ["".join(map(str, x)) for x in xs], "y": ["".join(map(str, y)) for y in ys],
           "sweeps": [], "source": "oracle/fit.py FitOracle (FP64, numpy), written by tests/golden/make_fit_golden.py"}
    for s in range(1, a.sweeps + 1):
        f.sweep(1, stop_on_converge=False)
        h = f.st.history[-1]
        item = {"sweep": s, "norm2": h.norm2, "delta": None if not np.isfinite(h.delta) else h.delta,
                "bonds": h.bonds}
        if s in a.keep:
            C = f.result()
            item["lambdas"] = [lam.tolist() for lam in f.lambdas()]
            item["entries"] = entries(C, xs, ys)
            item["norm_C"] = mpo_norm(C)
        rec["sweeps"].append(item)
        print(f"sweep {s}: norm2 {h.norm2:.15e} delta {h.delta:.3e} ({time.time() - t0:.0f} s)", flush=True)
    out = a.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), f"fit_{a.workload}_rsvd_site.json")
    with open(out, "w") as fh:
        json.dump(rec, fh)
    print("wrote", out)


if __name__ == "__main__":
    main()
