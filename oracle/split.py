"""Non-invasive splitting of the composite matrix into region matrices (Sec. 4).

Off-diagonal entries A_ij are shared by the q_ij regions that contain both i and j; each of
those regions receives A_ij / q_ij. The diagonal of each region matrix is then chosen so
that the region preserves the composite action on the constant vector: with z = A 1 moved
to the regional layout and divided by the multiplicity of each node (the nullspace rule of
the edge-based splitting scheme in the paper's draft appendix),

    A^(k)_ii = z_i / mult_i - sum_{j != i} A^(k)_ij .

For rows with zero row sum this is exactly the paper's "row sum of each region matrix is
identically zero"; for rows next to the Dirichlet boundary it still keeps sum_k A^(k) = A.
The result is returned in the block-diagonal regional form [[A]] = diag(Psi_k^T A^(k) Psi_k)
(eq. "block diagonal region matrix").
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .regions import Layout, block_diag


def share_counts(layout: Layout, A: sp.csr_matrix) -> sp.csr_matrix:
    """q_ij = number of regions containing both i and j, on the sparsity pattern of A.

    Every region k contributes a one at each entry (i, j) of A with i and j both in region k:
    Psi_k (Psi_k^T pattern(A) Psi_k) Psi_k^T, summed over k.
    """
    pattern = sp.csr_matrix(A, copy=True)
    pattern.data[:] = 1.0
    Q = None
    for Pk in layout.Psi_k:
        inside = (Pk @ (Pk.T @ pattern @ Pk) @ Pk.T).tocsr()
        Q = inside if Q is None else (Q + inside).tocsr()
    return Q


def split_blocks(layout: Layout, A: sp.csr_matrix):
    """Return the region blocks Psi_k^T A^(k) Psi_k (each n_k x n_k)."""
    A = sp.csr_matrix(A)
    Q = share_counts(layout, A)
    z = np.asarray(A @ np.ones(A.shape[0])).ravel()      # A applied to the constant vector
    blocks = []
    for k in range(layout.m):
        Pk = layout.Psi_k[k]                            # n x n_k
        Bk = (Pk.T @ A @ Pk).tocsr()                    # submatrix of A on region k
        Qk = (Pk.T @ Q @ Pk).tocsr()
        off = Bk - sp.diags(Bk.diagonal())
        off = off.tocsr()
        Qoff = (Qk - sp.diags(Qk.diagonal())).tocsr()
        # divide every off-diagonal by its share count (same sparsity as A's submatrix)
        off_split = off.multiply(_reciprocal_on_pattern(Qoff, off)).tocsr()
        zk = Pk.T @ z
        multk = Pk.T @ layout.mult
        offsum = np.asarray(off_split.sum(axis=1)).ravel()
        diag = zk / multk - offsum
        blocks.append((off_split + sp.diags(diag)).tocsr())
    return blocks


def _reciprocal_on_pattern(Q: sp.csr_matrix, pattern: sp.csr_matrix) -> sp.csr_matrix:
    """1/Q_ij on the nonzero pattern of ``pattern`` (Q_ij >= 1 wherever pattern is nonzero)."""
    P = pattern.copy().tocsr()
    P.data[:] = 1.0
    Qp = P.multiply(Q).tocsr()
    Qp.data = 1.0 / Qp.data
    return Qp


def split_regional(layout: Layout, A: sp.csr_matrix) -> sp.csr_matrix:
    """[[A]] = diag(Psi_k^T A^(k) Psi_k)."""
    return block_diag(split_blocks(layout, A))


def split_composite_pieces(layout: Layout, A: sp.csr_matrix):
    """The n x n split matrices A^(k) = Psi_k (block k) Psi_k^T (for Lemma 1 checks)."""
    return [(Pk @ Bk @ Pk.T).tocsr() for Pk, Bk in zip(layout.Psi_k, split_blocks(layout, A))]


def split_region_block(A: sp.csr_matrix, region_gids: np.ndarray, offsets: np.ndarray,
                       k: int) -> sp.csr_matrix:
    """Block Psi_k^T A^(k) Psi_k of a single region k, by the same rule as split_blocks
    (A_ij / q_ij off the diagonal, z_i / mult_i minus the split off-diagonal row sum on it),
    computed from region k and the regions that overlap it only. For operators too large for
    the whole-problem form; split_blocks is its check on small problems."""
    A = sp.csr_matrix(A)
    gids = np.asarray(region_gids, dtype=np.int64)
    n = A.shape[0]
    gk = gids[offsets[k]:offsets[k + 1]]
    mult = np.bincount(gids, minlength=n).astype(np.float64)
    # regions that hold any node of region k: every region whose node set meets gk
    inside = np.zeros(n, dtype=bool)
    inside[gk] = True
    region_of = np.repeat(np.arange(len(offsets) - 1), np.diff(offsets))
    neighbours = np.unique(region_of[inside[gids]])
    # membership of region k's nodes in each overlapping region, as bits of a mask
    bits = np.zeros(gk.shape[0], dtype=np.int64)
    for b, kk in enumerate(neighbours):
        member = np.zeros(n, dtype=bool)
        member[gids[offsets[kk]:offsets[kk + 1]]] = True
        bits |= member[gk].astype(np.int64) << b
    Bk = A[gk][:, gk].tocoo()
    off = Bk.row != Bk.col
    r, c, v = Bk.row[off], Bk.col[off], Bk.data[off]
    q = _popcount(bits[r] & bits[c])          # regions holding both i and j
    vs = v / q
    offsum = np.bincount(r, weights=vs, minlength=gk.shape[0])
    z = np.asarray(A[gk] @ np.ones(n)).ravel()
    diag = z / mult[gk] - offsum
    nk = gk.shape[0]
    M = sp.csr_matrix((np.concatenate([vs, diag]),
                       (np.concatenate([r, np.arange(nk)]), np.concatenate([c, np.arange(nk)]))),
                      shape=(nk, nk))
    return M


def _popcount(x: np.ndarray) -> np.ndarray:
    """Number of set bits of every entry (at most 63 overlapping regions)."""
    x = np.asarray(x, dtype=np.int64)
    count = np.zeros(x.shape, dtype=np.float64)
    while np.any(x):
        count += (x & 1)
        x = x >> 1
    return count
