"""Structured 3:1 grid transfers (Sec. 3.2 and Sec. 6.1 of the paper).

Coarsening by a rate of 3 in each coordinate direction keeps every third node (index
multiples of 3) as a coarse node; linear interpolation fills the two fine nodes between two
coarse nodes with weights (2/3, 1/3) and (1/3, 2/3). In several dimensions the interpolation
is the tensor product of the 1D operators. R = P^T.

Dirichlet (masked) nodes take part neither as interpolation targets nor as sources: the rows
of masked fine nodes and the columns of masked coarse nodes are zero. This is the same as
eliminating the Dirichlet nodes before building the hierarchy.

The regional (replicated-interface) interpolation is eq. "region interp":
[[P]] = diag(Psi_k^T P Psibar_k).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .regions import Layout, block_diag


def coarse_count(n: int) -> int:
    if n == 1:
        return 1
    if (n - 1) % 3 != 0:
        raise ValueError(f"{n} nodes cannot be coarsened 3:1 (need 3k + 1)")
    return (n - 1) // 3 + 1


def linear_p_1d(n: int) -> sp.csr_matrix:
    """n x nc linear interpolation with coarse nodes at fine indices 0, 3, 6, ..."""
    nc = coarse_count(n)
    if n == 1:
        return sp.csr_matrix(np.ones((1, 1)))
    rows, cols, vals = [], [], []
    for i in range(n):
        c, rem = divmod(i, 3)
        if rem == 0:
            rows.append(i); cols.append(c); vals.append(1.0)
        else:
            w_right = rem / 3.0
            rows += [i, i]; cols += [c, c + 1]; vals += [1.0 - w_right, w_right]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, nc))


def composite_p(global_dims, fine_mask, coarse_mask) -> sp.csr_matrix:
    """P on the global grid (x fastest): kron(Pz, kron(Py, Px)), masked rows/columns zero."""
    Nx, Ny, Nz = global_dims
    P = sp.kron(linear_p_1d(Nz), sp.kron(linear_p_1d(Ny), linear_p_1d(Nx))).tocsr()
    keep_rows = sp.diags((~np.asarray(fine_mask, bool)).astype(float))
    keep_cols = sp.diags((~np.asarray(coarse_mask, bool)).astype(float))
    P = (keep_rows @ P @ keep_cols).tocsr()
    P.eliminate_zeros()
    return P


def stored_p(global_dims, wr, fine_mask, coarse_mask) -> sp.csr_matrix:
    """P with stored per-node weights (Table 4's "general grid transfers": the sparsity of 3:1
    linear interpolation with coefficients of choice).

    ``wr`` is (3, n_fine), FP32: the weight fine node f takes from its right coarse neighbour
    along axis a; the left neighbour gets 1 - wr; along an axis where f sits on a coarse index
    the weight is 1. The row is the tensor product of the three axis weights, formed in FP32
    as wz (wy wx) (the library's definition of a stored-weight P).
    """
    Nx, Ny, Nz = global_dims
    cNx, cNy, cNz = coarse_count(Nx), coarse_count(Ny), coarse_count(Nz)
    n = Nx * Ny * Nz
    wr = np.asarray(wr, dtype=np.float32)
    one = np.float32(1.0)
    g = np.arange(n)
    coord = [g % Nx, (g // Nx) % Ny, g // (Nx * Ny)]
    c0 = [c // 3 for c in coord]
    rem = [c - 3 * q for c, q in zip(coord, c0)]
    rows, cols, vals = [], [], []
    for sc in (0, 1):
        for sb in (0, 1):
            for sa in (0, 1):
                side = (sa, sb, sc)
                ok = np.ones(n, bool)
                w = None
                cc = []
                for a in range(3):
                    if side[a]:
                        ok &= rem[a] != 0
                        wa = np.where(rem[a] != 0, wr[a], np.float32(0.0)).astype(np.float32)
                    else:
                        wa = np.where(rem[a] != 0, one - wr[a], one).astype(np.float32)
                    cc.append(c0[a] + side[a])
                    w = wa if w is None else (wa * w).astype(np.float32)
                col = cc[0] + cNx * (cc[1] + cNy * cc[2])
                rows.append(g[ok]); cols.append(col[ok]); vals.append(w[ok].astype(np.float64))
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, cNx * cNy * cNz))
    keep_rows = sp.diags((~np.asarray(fine_mask, bool)).astype(float))
    keep_cols = sp.diags((~np.asarray(coarse_mask, bool)).astype(float))
    P = (keep_rows @ P @ keep_cols).tocsr()
    P.eliminate_zeros()
    return P


def coarse_dims(global_dims):
    return tuple(coarse_count(n) for n in global_dims)


def coarse_slabs(slabs):
    return tuple(tuple(coarse_count(n) for n in axis) for axis in slabs)


def coarse_mask_from_fine(global_dims, fine_mask):
    """Coarse nodes are co-located with fine nodes of index 3i; they inherit the mask."""
    Nx, Ny, Nz = global_dims
    f = np.asarray(fine_mask).reshape(Nz, Ny, Nx)
    sz = slice(None, None, 3) if Nz > 1 else slice(None)
    return f[sz, ::3, ::3].reshape(-1).copy()


def regional_p(layout_f: Layout, layout_c: Layout, P: sp.csr_matrix) -> sp.csr_matrix:
    """[[P]] = diag(Psi_k^T P Psibar_k)."""
    return block_diag([(Pf.T @ P @ Pc).tocsr()
                       for Pf, Pc in zip(layout_f.Psi_k, layout_c.Psi_k)])
