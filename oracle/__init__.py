"""FP64 CPU oracle for the shrink-and-expand block eigensolvers
(Liu, Ma & Shao, "On a shrink-and-expand technique for symmetric block
eigensolvers", arXiv:2409.05572).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
(the CUDA library and its Python binding) never imports, links or calls it,
and shares no code with it: the two meet only through the seeded inputs of
``paper_2409_05572_gb300.workloads``, which hold none of the method's
arithmetic.

The oracle is plain NumPy/SciPy in float64, written step by step in the order
of the paper's algorithms (Algorithms 1, 2, 3, 5, 6, 7; Eqs. conv, rk, ckslope,
ckslopek).  Library primitives (sparse matrix product, dense matmul,
triangular solve, symmetric eigensolver, Householder QR) serve as steps.

Modules:
  blocks    - block primitives: SpMM, Gram, CholeskyQR2, Rayleigh-Ritz,
              Hetmaniuk-Lehoucq basis selection, residual test (Eq. conv/rk),
              Chebyshev filter.
  strategy  - the warm-up gate (also its first-pair variant from the
              paper's closing remarks) and the fix / slope / slopek
              strategies (Algorithms 6 and 7).
  lobpcg    - LOBPCG with soft locking and shrink-and-expand (Algorithm 3).
  chebsi    - subspace iteration with shrink-and-expand (Algorithm 1), the
              shift-and-invert solve replaced by a Chebyshev filter.
  sd        - steepest descent with shrink-and-expand (Algorithm 2).

Parity pins: every function here is checked by the ``-m "not gpu"`` tests
against closed forms, brute force, printed values of the paper's worked
3x3 examples, invariants and special cases.  Iteration counts of whole solves
are "parity unpinned" (rounding differences can move a strategy decision that
sits on a threshold by an iteration or two).
"""
