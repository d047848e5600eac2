"""GB300-native Neu-PiG optimisation hot path (sm_103a CUDA behind a C ABI).

``paper_2602_22212_gb300.npg`` is the thin ctypes binding of ``libnpg.so``;
``paper_2602_22212_gb300.inputs`` builds seeded synthetic sequences.
Submodules are imported lazily so that the input generators do not load the
CUDA library.
"""
