"""CPU FP64 oracle for the sparse dual solvers of De Palma et al., "Scaling the Convex Barrier with
Sparse Dual Algorithms" (arXiv 2101.05844).

TEST INFRASTRUCTURE ONLY. This package is a plain, slow restatement of the paper's method, used to
check the CUDA library. Only the tests, the package smoke check and the benchmark's CPU-baseline
leg may import it; the library never does. It shares no code with the CUDA path: convolutions are
expanded into their dense linear operators, masks are dense 0/1 matrices produced by the
separation oracle (eq. 3), and every step follows the paper's formulas in the paper's order.

Modules:
  network     dense linear operators of the layers, interval bound propagation (App. E).
  relaxation  the interval matrices of Sec. 2.2, the separation oracle eq. (3), mask row sums.
  dual        f_k, g_k (eq. 6 / Sec. 4.1), closed-form inner minimisation (eqs. 7-8),
              supergradient (eq. 9), Lagrangian value (eqs. 5-6), constraint-form Lagrangian (App. D).
  active_set  Big-M solver (Alg. 3, App. B) and Active Set (Alg. 1) with Adam.
  saddle      Saddle Point (Alg. 2): sufficient statistics (eq. 10), caps (eq. 16), primal
              initialisation (App. C.2), conditional gradients (eqs. 11-12).
  lp          exact rational simplex and the LPs of problems (2), (4) and (17) for pins.
  envelope    gradient of the bound at fixed duals (Danskin).

Parity pins are listed in the tests; "parity unpinned" notes sit in the module that has them.
"""
