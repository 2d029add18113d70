"""Region layout: the boolean map Psi and its properties (Sec. 3.1 of the paper).

Psi is n x n_r with a one at (i, j) when regional dof j is co-located with composite dof i.
The paper stores it implicitly; the oracle forms it as a sparse matrix so that the paper's
identities can be applied verbatim:

* Psi^T v        composite -> regional (replicate interface values),
* Psi [[v]]      regional  -> composite (sum co-located values),
* Psi^T Psi [[v]] interface summation,
* (Psi Psi^T)^-1 Psi [[v]] averaging,
* Psi Psi^T = diag(multiplicity).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Layout:
    region_dims: np.ndarray     # (m, 3) nodes per axis
    region_gids: np.ndarray     # (n_r,) composite id of every regional node
    n: int                      # composite nodes
    offsets: np.ndarray         # (m + 1,) start of every region in the regional vector
    Psi: sp.csr_matrix          # n x n_r
    Psi_k: list                 # column blocks Psi_k, each n x n_k
    mult: np.ndarray            # (n,) diagonal of Psi Psi^T
    mask: np.ndarray            # (n,) bool, Dirichlet (masked) composite nodes

    @property
    def n_r(self):
        return int(self.region_gids.shape[0])

    @property
    def m(self):
        return int(self.region_dims.shape[0])

    # -- the paper's operations, written with Psi -----------------------------------------
    def to_regional(self, v):
        """[[v]] = Psi^T v."""
        return self.Psi.T @ v

    def sum_to_composite(self, vr):
        """w = Psi [[v]]: sum of co-located regional values."""
        return self.Psi @ vr

    def interface_sum(self, vr):
        """[[w]] = Psi^T Psi [[v]]."""
        return self.Psi.T @ (self.Psi @ vr)

    def average_to_composite(self, vr):
        """w = (Psi Psi^T)^-1 Psi [[v]]."""
        return (self.Psi @ vr) / self.mult

    def regional_mult(self):
        """Diagonal of the interface version [[Psi Psi^T]] (multiplicity per regional dof)."""
        return self.Psi.T @ self.mult

    def regional_mask(self):
        return self.mask[self.region_gids]

    def dot(self, xr, yr):
        """Composite inner product of two consistent regional vectors: sum x y / mult."""
        return float(np.sum(xr * yr / self.regional_mult()))

    def counter_ids(self):
        """Composite dof id of every composite vector entry (the power-method counters)."""
        return np.arange(self.n)


def make_layout(region_dims, region_gids, n, mask) -> Layout:
    region_dims = np.asarray(region_dims, dtype=np.int64)
    gids = np.asarray(region_gids, dtype=np.int64)
    sizes = np.prod(region_dims, axis=1)
    offsets = np.zeros(len(sizes) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    assert offsets[-1] == gids.shape[0]
    n_r = gids.shape[0]
    Psi = sp.csr_matrix((np.ones(n_r), (gids, np.arange(n_r))), shape=(n, n_r))
    Psi_csc = Psi.tocsc()
    Psi_k = [Psi_csc[:, offsets[k]:offsets[k + 1]].tocsr() for k in range(len(sizes))]
    mult = np.asarray((Psi @ Psi.T).diagonal()).ravel()
    return Layout(region_dims, gids, n, offsets, Psi, Psi_k, mult,
                  np.asarray(mask).astype(bool))


def incidence(layout: Layout) -> sp.csr_matrix:
    """n x m node-region incidence M (M_ik = 1 when composite node i lies in region k)."""
    rows = layout.region_gids
    cols = np.repeat(np.arange(layout.m), np.diff(layout.offsets))
    return sp.csr_matrix((np.ones_like(rows, dtype=float), (rows, cols)),
                         shape=(layout.n, layout.m))


def block_diag(blocks):
    return sp.block_diag(blocks, format="csr")


@dataclass
class BlockLayout(Layout):
    """B dofs per node, vectors component-major (entry c * n + g): Psi_B = I_B (x) Psi."""
    B: int = 1
    scalar: Layout = None

    @property
    def n_r(self):
        return int(self.region_gids.shape[0]) * self.B

    def regional_mask(self):
        return np.tile(self.scalar.regional_mask(), self.B)

    def counter_ids(self):
        """Entry c * n + g is composite dof g * B + c (dofs numbered node-major)."""
        ns = self.scalar.n
        g = np.tile(np.arange(ns), self.B)
        c = np.repeat(np.arange(self.B), ns)
        return g * self.B + c


def block_layout(lay: Layout, B: int) -> BlockLayout:
    Psi = sp.kron(sp.identity(B, format="csr"), lay.Psi).tocsr()
    return BlockLayout(lay.region_dims, lay.region_gids, lay.n * B, lay.offsets, Psi, None,
                       np.tile(lay.mult, B), np.tile(lay.mask, B), B=B, scalar=lay)
