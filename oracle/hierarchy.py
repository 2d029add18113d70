"""Composite and regional multigrid hierarchies (Sec. 3.2; Theorem 1; Sec. 3.5).

Composite: A_{l+1} = R_l A_l P_l with R_l = P_l^T (the standard mgSetup figure).
Regional:  [[Abar]] = [[R]] [[A]] [[P]] computed block by block (eq.
"RegionalGalerkinProduct"), with [[P]] = diag(Psi_k^T P Psibar_k) and [[R]] = [[P]]^T.

Masked (Dirichlet) coarse nodes have zero rows and columns after the product because P has
zero columns there; they are reset to identity rows. In the regional form each of the mult
copies of a masked node receives 1/mult on the diagonal so that the composite sum is 1.

The coarse map Psibar ("inject") takes the regional nodes at local indices that are
multiples of 3 and the composite node co-located with them on the coarse grid.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .regions import Layout, make_layout, block_diag, block_layout
from .split import split_regional
from .transfer import composite_p, coarse_count, coarse_mask_from_fine, regional_p, stored_p


@dataclass
class Level:
    dims: tuple                       # composite grid nodes per axis
    layout: Layout                    # regional layout (Psi) on this level
    A: sp.csr_matrix                  # composite operator on this level
    Ar: sp.csr_matrix = None          # regional [[A]]
    P: sp.csr_matrix = None           # composite P to the next coarser level
    Pr: sp.csr_matrix = None          # regional [[P]]
    Dinv: np.ndarray = None           # composite 1/diag(A)
    Dinv_r: np.ndarray = None         # regional [[D~^-1]] with D~ = Psi^T Psi diag([[A]])
    lam: float = None                 # power-method estimate of lambda_max(D^-1 A)
    lam_r: float = None               # the same estimate computed in the regional form
    extra: dict = field(default_factory=dict)


def inject_layout(layout: Layout, dims) -> tuple:
    """Psibar: the coarse regional layout and the coarse composite grid (Sec. 3.2, inject)."""
    Nx, Ny, Nz = dims
    cdims = (coarse_count(Nx), coarse_count(Ny), coarse_count(Nz))
    cregion_dims, cgids = [], []
    for k in range(layout.m):
        nx, ny, nz = (int(v) for v in layout.region_dims[k])
        g = layout.region_gids[layout.offsets[k]:layout.offsets[k + 1]].reshape(nz, ny, nx)
        sz = slice(None, None, 3) if nz > 1 else slice(None)
        gc = g[sz, ::3, ::3]
        x = gc % Nx
        y = (gc // Nx) % Ny
        z = gc // (Nx * Ny)
        cg = x // 3 + cdims[0] * (y // 3 + cdims[1] * (z // 3 if Nz > 1 else z))
        cregion_dims.append((gc.shape[2], gc.shape[1], gc.shape[0]))
        cgids.append(cg.reshape(-1))
    cmask = coarse_mask_from_fine(dims, layout.mask)
    n_c = int(np.prod(cdims))
    return cdims, make_layout(np.asarray(cregion_dims), np.concatenate(cgids), n_c, cmask)


def _identity_on_mask(A: sp.csr_matrix, mask_diag_value: np.ndarray) -> sp.csr_matrix:
    """Add ``mask_diag_value`` on the diagonal (zero where nothing is to be added)."""
    return (A + sp.diags(mask_diag_value)).tocsr()


def build(problem_or_parts, nlevels: int, regional: bool = True, weights=None):
    """Build both hierarchies from a composite problem.

    ``problem_or_parts`` needs attributes global_dims, region_dims, region_gids, dirichlet, A.
    ``weights(l, level)``, if given, returns stored interpolation weights (3, n_l) for the
    transfer from level l (or None for linear interpolation); it is called once the level's
    operators exist. Returns a list of Level.
    """
    p = problem_or_parts
    dims = tuple(int(v) for v in p.global_dims)
    n = int(np.prod(dims))
    layout = make_layout(p.region_dims, p.region_gids, n, p.dirichlet)
    A = sp.csr_matrix(p.A)
    levels = [Level(dims=dims, layout=layout, A=A)]
    if regional:
        levels[0].Ar = split_regional(layout, A)
    for l in range(nlevels - 1):
        f = levels[l]
        cdims, clayout = inject_layout(f.layout, f.dims)
        wr = weights(l, f) if weights is not None else None
        if wr is None:
            P = composite_p(f.dims, f.layout.mask, clayout.mask)
        else:
            P = stored_p(f.dims, wr, f.layout.mask, clayout.mask)
        f.extra["wr"] = wr
        Ac = (P.T @ f.A @ P).tocsr()
        Ac = _identity_on_mask(Ac, clayout.mask.astype(float))
        f.P = P
        c = Level(dims=cdims, layout=clayout, A=Ac)
        if regional:
            f.Pr = regional_p(f.layout, clayout, P)
            Arc = (f.Pr.T @ f.Ar @ f.Pr).tocsr()
            rmask = clayout.regional_mask()
            rmult = clayout.regional_mult()
            c.Ar = _identity_on_mask(Arc, np.where(rmask, 1.0 / rmult, 0.0))
        levels.append(c)
    for lev in levels:
        lev.Dinv = 1.0 / lev.A.diagonal()
        if regional:
            dr = lev.layout.interface_sum(lev.Ar.diagonal())
            lev.Dinv_r = 1.0 / dr
    return levels


def node_major_to_component_major(n_nodes: int, B: int) -> np.ndarray:
    """Permutation: component-major entry c * n + g takes node-major dof g * B + c."""
    g = np.tile(np.arange(n_nodes), B)
    c = np.repeat(np.arange(B), n_nodes)
    return g * B + c


def build_block(p, nlevels: int):
    """Hierarchies of a B-dof operator (elasticity) in component-major ordering.

    The split acts on every B x B block A_cc' = A[c::B, c'::B] with the scalar rule (for the
    translations of the draft appendix's nullspace rule this is the scalar rule per block);
    the transfers are I_B (x) P with the scalar 3:1 interpolation; Galerkin products as usual.
    """
    B = p.dofs_per_node
    dims = tuple(int(v) for v in p.global_dims)
    n = int(np.prod(dims))
    slay = make_layout(p.region_dims, p.region_gids, n, p.dirichlet)
    perm = node_major_to_component_major(n, B)
    A = sp.csr_matrix(p.A)[perm][:, perm].tocsr()
    blocks = [[split_regional(slay, A[c * n:(c + 1) * n, c2 * n:(c2 + 1) * n])
               for c2 in range(B)] for c in range(B)]
    lay = block_layout(slay, B)
    lev0 = Level(dims=dims, layout=lay, A=A, Ar=sp.bmat(blocks, format="csr"))
    lev0.extra["slay"] = slay
    levels = [lev0]
    I = sp.identity(B, format="csr")
    for l in range(nlevels - 1):
        f = levels[l]
        fs = f.extra["slay"]
        cdims, cs = inject_layout(fs, f.dims)
        Pn = composite_p(f.dims, fs.mask, cs.mask)
        f.P = sp.kron(I, Pn).tocsr()
        f.Pr = sp.kron(I, regional_p(fs, cs, Pn)).tocsr()
        clay = block_layout(cs, B)
        Ac = _identity_on_mask((f.P.T @ f.A @ f.P).tocsr(), clay.mask.astype(float))
        Arc = (f.Pr.T @ f.Ar @ f.Pr).tocsr()
        rmask = clay.regional_mask()
        c = Level(dims=cdims, layout=clay, A=Ac,
                  Ar=_identity_on_mask(Arc, np.where(rmask, 1.0 / clay.regional_mult(), 0.0)))
        c.extra["slay"] = cs
        levels.append(c)
    for lev in levels:
        lev.Dinv = 1.0 / lev.A.diagonal()
        lev.Dinv_r = 1.0 / lev.layout.interface_sum(lev.Ar.diagonal())
    return levels


def coarse_composite_from_regional(level: Level) -> sp.csr_matrix:
    """Abar = Psibar [[Abar]] Psibar^T on the coarsest level (eq. CoarseCompositeOperator,
    with the trailing Psibar^T of Theorem 1 that the printed equation omits)."""
    Psi = level.layout.Psi
    return (Psi @ level.Ar @ Psi.T).tocsr()
