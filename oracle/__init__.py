"""FP64 CPU oracle for the polynomial-smoother AMG path.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct
reference that the CUDA path is checked against.  Only the test-suite, the
package entry's smoke check and the benchmark's CPU-baseline / reference arm may
import it; the product path never does, and this package imports nothing from
the product.  The one input module both sides share is the seeded problem
generator, which holds none of the method's arithmetic.

Contents (each function cites the paper passage it restates):

* :mod:`oracle.params`   - a_k* (Eq. optimalparameter), closed-form polynomials
  (4th-kind W_k, scaled 1st-kind tau_k^{[a,1]}), the gamma functional of
  Proposition 1, and the optimal 4th-kind weights beta_{j,k} (minimax problem
  Eq. prob1, solved here by a Remez exchange).
* :mod:`oracle.smoother` - l1-Jacobi diagonal (Eq. l1smooth), the 4th-kind
  recurrence (Eq. polsmoother) and its optimised-weight form
  (Eq. polsmootheropt), the 1st-kind acceleration (Algorithm 1), plain
  l1-Jacobi sweeps, and the power-iteration spectral estimate.
* :mod:`oracle.amg`      - symmetric V-cycle (Eq. amg), dense Cholesky coarse
  solve, preconditioned CG.
* :mod:`oracle.adjoint`  - reverse-mode derivatives of the smoother and of the
  V-cycle error-reduction loss.
* :mod:`oracle.mlp`      - FP64 reference of the weight-predicting MLP.
* :mod:`oracle.omp`      - the smoother, V-cycle and PCG loops restated in
  plain C with OpenMP row loops (``oracle/c/amg_omp.c``), for timing the
  oracle on every host core; checked against the numpy oracle.

Parity status: every function is pinned by tests against printed constants,
closed forms or brute force, except where its docstring says "parity unpinned".
"""
