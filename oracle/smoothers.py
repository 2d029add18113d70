"""Smoothers of Sec. 3.4 and the power-method eigenvalue estimate.

All functions are written against two callables so that the same formulas serve the
composite operator and the regional one:

* ``residual(u, b)`` returns b - A u (regional: [[b]] - Psi^T Psi [[A]] [[u]], eq.
  "regional residual"),
* ``dot(x, y)`` is the composite inner product.

``dinv`` is the inverse of the composite diagonal, in the layout of the vectors.
"""
from __future__ import annotations

import numpy as np


def jacobi(u, b, residual, dinv, omega, sweeps):
    """Damped Jacobi: u <- u + omega D~^-1 r with r recomputed before every sweep."""
    u = u.copy()
    for _ in range(sweeps):
        r = residual(u, b)
        u = u + omega * dinv * r
    return u


def gauss_seidel_colored(u, b, residual, local_apply, dinv, omega, sweeps, colours, order):
    """Region Gauss-Seidel of Algorithm 1 with the nodes of every region visited colour by
    colour (``colours`` gives each regional node its colour, ``order`` the colour sequence).

    Each sweep recomputes the regional residual r (with the interface sum), sets delta = 0,
    and then for every colour class: r_i <- r_i - sum_j A^(l)_ij delta_j with the region's
    own matrix (``local_apply`` = [[A]] delta, no interface sum), delta_i = omega r_i / d~_ii,
    u_i <- u_i + delta_i. Copies of an interface node are updated by their own regions and
    need not agree afterwards (as the paper notes for Algorithm 1).
    """
    u = u.copy()
    for _ in range(sweeps):
        r = residual(u, b)
        delta = np.zeros_like(u)
        for c in order:
            sel = colours == c
            rc = r[sel] - local_apply(delta)[sel]
            delta[sel] = omega * rc * dinv[sel]
            u[sel] = u[sel] + delta[sel]
    return u


def chebyshev_bounds(lam_max_est, eig_ratio=20.0, boost=1.1):
    """[alpha, beta] = [lambda~/eta, boost * lambda~] (Sec. 3.4, Ifpack2 convention)."""
    return lam_max_est / eig_ratio, boost * lam_max_est


def chebyshev(u, b, residual, dinv, alpha, beta, degree):
    """Chebyshev smoother of Algorithm 2 with ``degree`` updates of u.

    theta is the centre and delta = 2/(beta - alpha) the inverse half-width of [alpha, beta].
    The first direction is D~^-1 r / theta (the reading under which Algorithm 2 is the
    classical three-term Chebyshev acceleration); each further step recomputes the regional
    residual, updates rho and the direction d, and adds d to u.
    """
    theta = 0.5 * (alpha + beta)
    delta = 2.0 / (beta - alpha)
    rho = 1.0 / (theta * delta)
    r = residual(u, b)
    d = dinv * r / theta
    u = u + d
    for _ in range(degree - 1):
        r = residual(u, b)
        rho_old = rho
        rho = 1.0 / (2.0 * theta * delta - rho_old)
        d = rho * rho_old * d + 2.0 * rho * delta * dinv * r
        u = u + d
    return u


def power_method(matvec, dinv, dot, x0, iters=10):
    """lambda~_max(D^-1 A): ``iters`` normalised power steps from x0, then the Rayleigh
    quotient x^T D^-1 A x / x^T x of the last normalised iterate."""
    x = x0 / np.sqrt(dot(x0, x0))
    for _ in range(iters):
        y = dinv * matvec(x)
        x = y / np.sqrt(dot(y, y))
    y = dinv * matvec(x)
    return dot(x, y) / dot(x, x)
