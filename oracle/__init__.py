"""CPU oracle for sketch-preconditioned Riemannian CCA / Fisher LDA (FP64).

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct NumPy/SciPy code in
float64 that states what the method computes, section by section, following
Shustin & Avron, "Faster Randomized Methods for Orthogonality Constrained
Problems".  Only the test-suite, the smoke check and the CPU-baseline leg of
the benchmark may import this package; the library itself never does, and
shares no code with it.

Modules
  rng       counter-based generator (SplitMix64) and Feistel row permutation
  sketch    CountSketch (Sec. 3) and SRHT (App. A, Def. A.1)
  precond   R factor of [S Z; sqrt(lambda) I] (Sec. 3)
  cca       closed-form regularized CCA (Def. 4.1) by three routes
  lda       closed-form regularized FDA (Def. 5.1) by two routes
  geometry  generalized Stiefel components with metric M (Table 1)
  problems  CCA / FDA costs and Euclidean gradients (Eq. 4.2, Eq. 5.2 ...)
  fused     the per-iteration data products as explicit matrix products
  rcg       reference Riemannian CG and the ALS / power-method special cases

Parity status of each function is stated in its module header.
"""
