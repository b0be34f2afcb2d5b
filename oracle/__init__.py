"""FP64 CPU oracle for the SCS-style ADMM hot path (test infrastructure).

This package is test infrastructure only: ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the product path never
does.  It is plain, slow, obviously-correct NumPy in float64 and shares no
code with the CUDA path (it does not import ``paper_1609_03488_b300``).

Modules:

* ``quant``  -- BF16 / FP8-e4m3 (+ per-row scale) operand rounding, from the
  formats' definitions.
* ``linop``  -- the structured linear operators of Section 3.1 (dense, CSR,
  1-D/2-D convolution, diagonal, Kronecker and their compositions): dense
  materialisation and matrix-free apply / adjoint (Section 4.1: adjoints by
  transformation of the operator graph).
* ``cones``  -- Euclidean projections onto the zero, nonnegative and
  second-order cones and their duals.
* ``cg``     -- conjugate gradient (the ``cg_solve`` routine of Section 4.2).
* ``scs``    -- the SCS iteration on the homogeneous self-dual embedding
  (Section 5.2 uses SCS as its solver; the steps follow the published SCS
  method, which the paper cites and does not restate).

Every function's docstring names the passage it follows.  Parity pins (the
checks that tie this code to something other than itself) live in
``tests/test_oracle_*.py``; functions without such a pin say "parity unpinned".
"""
