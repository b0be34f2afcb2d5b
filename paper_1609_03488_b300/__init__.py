"""B300-native SCS-style ADMM hot path of arxiv 1609.03488 (cvxflow).

* ``paper_1609_03488_b300.binding`` -- ctypes binding of the C ABI
  (``include/cvxb300.h``) over the CUDA kernels in ``csrc/`` (compiled by
  ``paper_1609_03488_b300.build``).  Import it explicitly; importing the
  package alone does not load the shared library.
* ``paper_1609_03488_b300.synth`` -- seeded synthetic cone programs shaped
  like the paper's workloads.
"""
