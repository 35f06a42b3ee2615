"""GB300-native variational MPO-MPO fit (libttfit.so behind include/ttfit.h).

``paper_2606_23274_gb300.ttfit`` is the thin ctypes binding of the C ABI;
``paper_2606_23274_gb300.synth`` draws the seeded synthetic MPO workloads.
"""
