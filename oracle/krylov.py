"""Preconditioned conjugate gradients (textbook form; Saad, Iterative Methods, Alg. 9.1).

The paper runs multigrid as a stand-alone solver and notes that applications normally call
it inside a Krylov method (Sec. 6.2); here one V-cycle with zero initial guess is the
preconditioner. The stopping test is ||b - A x||_2 / ||b||_2 <= rtol, read as a property of
the returned iterate: it is first met on the recurrence residual, then checked on the true
residual b - A x, and if that one does not pass the iteration restarts from it. The iteration
count is the number of products with A inside the iteration.
"""
from __future__ import annotations

import numpy as np


def pcg(A, b, precond, rtol=1e-10, maxit=200, x0=None, flexible=False, counts=None):
    """Preconditioned CG; flexible=True takes the Polak-Ribiere form
    beta = r.(z - z_old) / r_old.z_old for a preconditioner that is not exactly symmetric.
    ``counts`` (a dict, optional) receives the number of preconditioner applications and of
    restarts."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    bnorm = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bnorm]
    ncyc = restarts = 0
    it = 0
    done = hist[-1] <= rtol
    while not done and it < maxit:
        z = precond(r)
        ncyc += 1
        p = z.copy()
        rz = float(r @ z)
        while it < maxit:
            it += 1
            q = A @ p
            alpha = rz / float(p @ q)
            x = x + alpha * p
            r = r - alpha * q
            hist.append(np.linalg.norm(r) / bnorm)
            if hist[-1] <= rtol:
                rt = b - A @ x
                if np.linalg.norm(rt) / bnorm <= rtol:
                    done = True
                else:
                    r = rt
                    restarts += 1
                break
            z_old = z
            z = precond(r)
            ncyc += 1
            rz_new = float(r @ z)
            beta = (rz_new - float(r @ z_old)) / rz if flexible else rz_new / rz
            rz = rz_new
            p = z + beta * p
    if counts is not None:
        counts.update(vcycles=ncyc, restarts=restarts)
    return x, it, hist


def regional_preconditioner(mg):
    """Composite-in, composite-out wrapper of a regional V-cycle: z = avg(cycle(Psi^T r))."""
    lay = mg.levels[0].layout

    def apply(r):
        return lay.average_to_composite(mg.precondition(lay.to_regional(r)))
    return apply
