"""Plain FP64 CPU oracle for region multigrid (arXiv 2103.11962).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package. The GPU library never calls it, shares no code
with it and has no fallback to it.

The oracle forms the paper's objects literally, as scipy.sparse matrices, and applies the
paper's formulas to them, so each step can be checked against the text by eye:

* ``regions``   - the boolean map Psi (Sec. 3.1), multiplicities Psi Psi^T.
* ``split``     - non-invasive splitting of the composite matrix into region matrices (Sec. 4).
* ``transfer``  - 3:1 linear interpolation P, R = P^T, regional replicated-interface form
                  [[P]] = diag(Psi_k^T P Psibar_k) (Sec. 3.1, Sec. 3.2).
* ``hierarchy`` - composite and regional Galerkin hierarchies (Sec. 3.2, Theorem 1).
* ``smoothers`` - damped Jacobi, Chebyshev (Algorithm 2) and the power method (Sec. 3.4).
* ``cycle``     - the composite V-cycle and the regional V-cycle (Sec. 3.3, Sec. 3.6 figure).
* ``krylov``    - preconditioned conjugate gradients (the paper only mentions Krylov use).
* ``rng``       - SplitMix64 as a counter-based generator (for power-method start vectors).
* ``learned``   - operator-dependent weights, the learned prolongator's features and its small
                  MLP (forward, loss and gradient); no paper basis, pinned by closed forms.

Parity status of every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
lemmas of the paper and brute force; the exceptions are listed in ``UNPINNED``.
"""

# Every function is pinned. The power method is pinned to its closed form in the eigenpairs of
# D^-1/2 A D^-1/2 and to the bounds (0.85 lambda_max, lambda_max]. Its start vector and step
# count are readings (the paper leaves both open), not pins.
UNPINNED = {}
