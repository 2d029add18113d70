"""Composite and regional multigrid V-cycles (the two mgCycle figures of Sec. 3).

Regional cycle on level l with regional vectors [[u]], [[b]] (Sec. 3.3, Sec. 3.6 figure):

    [[u]] <- applySmoother([[u]], [[b]])                         (nu1 sweeps)
    [[r]] <- [[b]] - Psi^T Psi [[A]] [[u]]                         (regional residual)
    [[w]] <- Psibar^T Psibar [[R]] [[Psi Psi^T]]^-1 [[r]]          (regional restriction)
    [[ubar]] <- cycle(l + 1, 0, [[w]])
    [[u]] <- [[u]] + [[P]] [[ubar]]                               (regional interpolation)
    [[u]] <- applySmoother([[u]], [[b]])                         (nu2 sweeps)

On the coarsest level the regional right-hand side is averaged to the composite layout,
the composite system Abar = Psibar [[Abar]] Psibar^T is solved directly (Cholesky of the
unmasked block) and the solution is replicated back to the regions (Sec. 3.5).

The composite cycle is the same recursion with composite A, P, R = P^T and diag(A).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from . import smoothers
from .hierarchy import Level, coarse_composite_from_regional
from .rng import uniform_pm1


@dataclass
class Options:
    smoother: str = "jacobi"     # "jacobi", "chebyshev" or "gs" (region Gauss-Seidel)
    nu1: int = 2                 # pre-smoothing: Jacobi sweeps / Chebyshev applications
    nu2: int = 2                 # post-smoothing
    omega: float = 0.67
    degree: int = 3              # Chebyshev updates per smoothing step
    eig_ratio: float = 20.0
    boost: float = 1.1
    power_iters: int = 10
    power_seed_base: int = 10    # start vector of level l uses SplitMix64 stream seed_base + l


class CoarseSolver:
    """Dense Cholesky of the unmasked block of the coarsest composite operator."""

    def __init__(self, Abar, mask):
        self.free = np.flatnonzero(~np.asarray(mask, bool))
        dense = Abar.toarray()[np.ix_(self.free, self.free)]
        self.L = np.linalg.cholesky(dense)
        self.n = Abar.shape[0]

    def solve(self, rhs):
        x = np.zeros(self.n)
        y = sla.solve_triangular(self.L, rhs[self.free], lower=True)
        x[self.free] = sla.solve_triangular(self.L.T, y, lower=False)
        return x


def power_start(level: Level, l: int, opts: Options):
    """Composite start vector: SplitMix64 stream (seed_base + l) indexed by composite id."""
    x = uniform_pm1(opts.power_seed_base + l, level.layout.counter_ids())
    x[level.layout.mask] = 0.0
    return x


def gs_colours(level: Level):
    """Colour of every regional node for the multicolour region Gauss-Seidel: the parity of
    i + j + l (2 colours) when the level's operator couples only nodes that differ along one
    axis (5- and 7-point stencils), else the parities of i, j and l (4 colours in 2D, 8 in 3D:
    9- and 27-point stencils). Nodes of one colour are never coupled."""
    lay = level.layout
    i_all, j_all, l_all = [], [], []
    for (nx, ny, nz) in np.asarray(lay.region_dims):
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        i_all.append(x.ravel()); j_all.append(y.ravel()); l_all.append(z.ravel())
    i, j, l = np.concatenate(i_all), np.concatenate(j_all), np.concatenate(l_all)
    Ar = level.Ar.tocoo()
    B = level.Ar.shape[0] // i.shape[0]
    rr, cc = Ar.row % i.shape[0], Ar.col % i.shape[0]
    axes = ((i[rr] != i[cc]).astype(int) + (j[rr] != j[cc]).astype(int) +
            (l[rr] != l[cc]).astype(int))
    dim3 = bool(np.any(np.asarray(lay.region_dims)[:, 2] > 1))
    if not np.any(axes > 1):
        col = (i + j + l) & 1
        ncol = 2
    else:
        col = (i & 1) | ((j & 1) << 1) | ((l & 1) << 2)
        ncol = 8 if dim3 else 4
    return np.tile(col, B), ncol


class CompositeMG:
    def __init__(self, levels, opts: Options):
        self.levels, self.opts = levels, opts
        L = len(levels)
        for l, lev in enumerate(levels[:-1]):
            if opts.smoother == "chebyshev":
                dot = lambda x, y: float(x @ y)
                lev.lam = smoothers.power_method(lambda v, A=lev.A: A @ v, lev.Dinv, dot,
                                                 power_start(lev, l, opts), opts.power_iters)
        self.coarse = CoarseSolver(levels[-1].A, levels[-1].layout.mask)
        self.L = L

    def smooth(self, l, u, b, nu):
        lev, o = self.levels[l], self.opts
        res = lambda uu, bb, A=lev.A: bb - A @ uu
        if o.smoother == "jacobi":
            return smoothers.jacobi(u, b, res, lev.Dinv, o.omega, nu)
        a, bt = smoothers.chebyshev_bounds(lev.lam, o.eig_ratio, o.boost)
        for _ in range(nu):
            u = smoothers.chebyshev(u, b, res, lev.Dinv, a, bt, o.degree)
        return u

    def cycle(self, u, b, l=0):
        if l == self.L - 1:
            return self.coarse.solve(b)
        lev = self.levels[l]
        u = self.smooth(l, u, b, self.opts.nu1)
        r = b - lev.A @ u
        w = lev.P.T @ r
        ubar = self.cycle(np.zeros(lev.P.shape[1]), w, l + 1)
        u = u + lev.P @ ubar
        return self.smooth(l, u, b, self.opts.nu2)

    def precondition(self, r):
        return self.cycle(np.zeros_like(r), r)


class RegionalMG:
    def __init__(self, levels, opts: Options):
        self.levels, self.opts = levels, opts
        self.L = len(levels)
        for l, lev in enumerate(levels[:-1]):
            if opts.smoother == "chebyshev":
                lay = lev.layout
                mv = lambda v, lev=lev: lev.layout.interface_sum(lev.Ar @ v)
                x0 = lay.to_regional(power_start(lev, l, opts))
                lev.lam_r = smoothers.power_method(mv, lev.Dinv_r, lay.dot, x0, opts.power_iters)
        last = levels[-1]
        self.Abar = coarse_composite_from_regional(last)
        self.coarse = CoarseSolver(self.Abar, last.layout.mask)

    def residual(self, l, u, b):
        lev = self.levels[l]
        return b - lev.layout.interface_sum(lev.Ar @ u)

    def smooth(self, l, u, b, nu, post=False):
        lev, o = self.levels[l], self.opts
        res = lambda uu, bb: self.residual(l, uu, bb)
        if o.smoother == "jacobi":
            return smoothers.jacobi(u, b, res, lev.Dinv_r, o.omega, nu)
        if o.smoother == "gs":
            colours, ncol = gs_colours(lev)
            order = list(range(ncol))[::-1] if post else list(range(ncol))
            return smoothers.gauss_seidel_colored(u, b, res, lambda d: lev.Ar @ d, lev.Dinv_r,
                                                  o.omega, nu, colours, order)
        a, bt = smoothers.chebyshev_bounds(lev.lam_r, o.eig_ratio, o.boost)
        for _ in range(nu):
            u = smoothers.chebyshev(u, b, res, lev.Dinv_r, a, bt, o.degree)
        return u

    def restrict(self, l, r):
        """[[w]] = Psibar^T Psibar [[R]] [[Psi Psi^T]]^-1 [[r]]."""
        lev, nxt = self.levels[l], self.levels[l + 1]
        scaled = r / lev.layout.regional_mult()
        return nxt.layout.interface_sum(lev.Pr.T @ scaled)

    def coarse_solve(self, b):
        lay = self.levels[-1].layout
        x = self.coarse.solve(lay.average_to_composite(b))
        return lay.to_regional(x)

    def cycle(self, u, b, l=0):
        if l == self.L - 1:
            return self.coarse_solve(b)
        lev = self.levels[l]
        u = self.smooth(l, u, b, self.opts.nu1)
        r = self.residual(l, u, b)
        w = self.restrict(l, r)
        ubar = self.cycle(np.zeros(lev.Pr.shape[1]), w, l + 1)
        u = u + lev.Pr @ ubar
        return self.smooth(l, u, b, self.opts.nu2, post=True)

    def precondition(self, r):
        return self.cycle(np.zeros_like(r), r)
