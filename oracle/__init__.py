"""FP64 CPU oracle for the MPO-MPO fit contraction.

ORACLE: this package is test infrastructure. Only tests/, __graft_entry__.smoke()
and bench.py (its CPU-baseline and reference legs) may import it; the product
path (paper_2606_23274_gb300) never does, and shares no code with it.

Parity status per function (pins live in tests/test_oracle_*.py):
* naive_product, to_dense, canonical forms, mpo_diff_norm: pinned (dense brute
  force on tiny L, closed-form Kronecker norms, isometry invariants).
* philox: pinned (Random123 known-answer vectors in tests/golden/).
* fit (Algs. 3-5): pinned (exact product at chi_C >= chi_A chi_B, gauge
  equivalence, Pythagorean residual identity, monotone residual, dense
  brute-force projection optimality on a tiny window).
* randomized_svd: pinned (equals the exact SVD when the sketch spans the range;
  Gaussian moments of Omega).
"""
