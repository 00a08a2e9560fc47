"""Plain, slow FP64 CPU oracle for the randomized truncated SVD (RSVD) hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or call
anything in this package.  The product path (the CUDA library and its Python
binding) never imports it, and the oracle never imports the product path: the
two share no code.  The only module both sides use is the seeded input
generator ``paper_1710_01463_gb300.inputs``, which holds none of the method's
arithmetic.

Everything here follows Kohn et al., "Probabilistic low-rank factorization
accelerates tensor network simulations of critical quantum many-body ground
states" (arXiv:1710.01463), written in the paper's order and notation, with
library primitives (matmul, LAPACK SVD / QR / eigh) used as steps:

* ``philox``  - Philox4x64-10 counter-based generator and the Gaussian test
  matrix Omega (Alg. RSVD step 1, Sec. II.B).
* ``rsvd``    - Alg. TSVD (Sec. II.A) and Alg. RSVD with the power iteration
  re-orthonormalised after every application of A or A^T (Sec. II.B).
* ``sectors`` - block-wise compression of a block-diagonal matrix with the
  global post-selection of the chi largest singular values (Sec. III.A).
* ``tebd``    - imaginary-time TEBD of the open spin-1/2 transverse-field Ising
  chain (Sec. III.A, III.B, III.C), its exact MPS energy, and the free-fermion
  closed form of the ground energy.
* ``grad``    - the derivative of a loss of the truncated factorization,
  through the full-SVD adjoint, and central finite differences.

Every function is pinned in ``tests/test_oracle_*.py`` against facts fixed by
the paper or by mathematics (closed forms, invariants, brute force, an
independent library generator), never against itself.
"""
