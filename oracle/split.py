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
