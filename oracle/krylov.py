"""Preconditioned conjugate gradients (textbook form; Saad, Iterative Methods, Alg. 9.1).

The paper runs multigrid as a stand-alone solver and notes that applications normally call
it inside a Krylov method; here one V-cycle with zero initial guess is the preconditioner.
The stopping test is ||b - A x||_2 / ||b||_2 <= rtol on the recurrence residual, and the
iteration count is the number of products with A.
"""
from __future__ import annotations

import numpy as np


def pcg(A, b, precond, rtol=1e-10, maxit=200, x0=None, flexible=False):
    """Preconditioned CG; flexible=True takes the Polak-Ribiere form
    beta = r.(z - z_old) / r_old.z_old for a preconditioner that is not exactly symmetric."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    bnorm = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bnorm]
    if hist[-1] <= rtol:
        return x, 0, hist
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    for it in range(1, maxit + 1):
        q = A @ p
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        hist.append(np.linalg.norm(r) / bnorm)
        if hist[-1] <= rtol:
            break
        z_old = z
        z = precond(r)
        rz_new = float(r @ z)
        beta = (rz_new - float(r @ z_old)) / rz if flexible else rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, it, hist


def regional_preconditioner(mg):
    """Composite-in, composite-out wrapper of a regional V-cycle: z = avg(cycle(Psi^T r))."""
    lay = mg.levels[0].layout

    def apply(r):
        return lay.average_to_composite(mg.precondition(lay.to_regional(r)))
    return apply
