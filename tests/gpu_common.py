"""Shared helpers of the GPU parity tests (test-side glue, no method arithmetic)."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

OFFSETS = {
    7: [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)],
    5: [(0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0)],
    27: [(s % 3 - 1, (s // 3) % 3 - 1, s // 9 - 1) for s in range(27)],
    9: [(s % 3 - 1, s // 3 - 1, 0) for s in range(9)],
}


def region_offsets(region_dims):
    sizes = np.prod(np.asarray(region_dims, dtype=np.int64), axis=1)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    return off


def stencils_to_matrix(region_dims, coef, kind):
    """Block-diagonal regional matrix from slot-major region stencils."""
    off = region_offsets(region_dims)
    n_r = int(off[-1])
    coef = np.asarray(coef).reshape(kind, n_r)
    rows, cols, vals = [], [], []
    for k, (nx, ny, nz) in enumerate(np.asarray(region_dims)):
        nx, ny, nz = int(nx), int(ny), int(nz)
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        x, y, z = x.ravel(), y.ravel(), z.ravel()
        base = int(off[k])
        loc = np.arange(nx * ny * nz)
        for s, (dx, dy, dz) in enumerate(OFFSETS[kind]):
            ok = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny) & \
                 (z + dz >= 0) & (z + dz < nz)
            v = coef[s, base + loc[ok]]
            nb = (x + dx) + nx * ((y + dy) + ny * (z + dz))
            rows.append(base + loc[ok]); cols.append(base + nb[ok]); vals.append(v)
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n_r, n_r))
    return M


def rel_max(a, b):
    a, b = np.asarray(a), np.asarray(b)
    den = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / den)


def matrix_rel_diff(A, B):
    D = (A - B).tocsr()
    den = max(abs(B).max(), 1e-300)
    return float(abs(D).max() / den) if D.nnz else 0.0
