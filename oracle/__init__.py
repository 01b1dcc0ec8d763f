"""CPU oracle for iterative Grover on a matrix product state (MPS).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import anything
here.  The CUDA library under `paper_2601_03832_gb300/` never imports, links
or calls this package, and this package never imports the CUDA library: the
two share no code.  The only common input is the seeded instance generator
`paper_2601_03832_gb300.inputs`, which holds none of the method's arithmetic
(and which these modules do not import either: instances are passed in).

Everything is plain, slow and FP64 (complex128), written to be checked
against the paper by eye:

* `statevector` -- dense 2^n vector; the Grover operator of Sec. II applied
  by its definition (n <= 24), plus the reverse-mode adjoint of the phases.
* `reduced`     -- the two-dimensional invariant-plane model of Sec. II
  (Eqs. 1-3), the closed form (Eqs. 5-6) and the exact Schmidt spectrum of
  the state at every cut of the chain.
* `mps`         -- a plain MPS following the steps of Sec. III-B-2: MPO
  contraction, canonicalising QR sweep, truncated-SVD sweep, amplitudes and
  perfect sampling.
* `philox`      -- the Philox4x64-10 counter-based generator (Salmon et al.,
  SC'11) used to draw the sampler's uniforms on both sides.

Pins (tests/test_oracle_*.py) tie each function to something other than
itself: the closed form, brute-force dense operators, library routines
(numpy.linalg.svd, numpy.random.Philox) and finite differences.
"""
