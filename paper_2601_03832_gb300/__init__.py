"""GB300 (sm_103a) iterative-Grover MPS simulator.

`paper_2601_03832_gb300.inputs` holds the seeded instance generators;
`paper_2601_03832_gb300.binding` is the thin ctypes binding over the C ABI of
libgrover_mps.so (include/grover_mps.h).  Importing this package loads
nothing; the binding raises on first use when the CUDA library is missing.
"""
