"""Region multigrid on one GB300 (sm_103a): the regional V-cycle of arXiv 2103.11962 as a
preconditioner, behind the C ABI in include/rmg.h.

``rmg`` is the ctypes binding of librmg.so; ``build`` compiles it. ``upload`` moves a problem
description (composite CSR, region map, mask, right-hand side) to device tensors.
"""
from __future__ import annotations

__all__ = ["upload", "DeviceProblem"]


class DeviceProblem:
    """Device copies of a problem's arrays (torch tensors on one CUDA device)."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def upload(problem, device="cuda:0", with_rhs=True):
    """Copy the arrays of ``problem`` (attributes A [scipy CSR], region_gids, dirichlet, b,
    region_dims, dim, stencil, n_nodes) to ``device`` as torch tensors."""
    import numpy as np
    import torch

    A = problem.A.tocsr()
    dp = DeviceProblem(
        dim=problem.dim,
        stencil=problem.stencil,
        n=problem.n_nodes,
        region_dims=np.asarray(problem.region_dims, dtype=np.int32),
        rowptr=torch.from_numpy(A.indptr.astype(np.int64)).to(device),
        col=torch.from_numpy(A.indices.astype(np.int64)).to(device),
        val=torch.from_numpy(A.data.astype(np.float64)).to(device),
        gids=torch.from_numpy(np.asarray(problem.region_gids, dtype=np.int64)).to(device),
        dirichlet=torch.from_numpy(np.asarray(problem.dirichlet, dtype=np.uint8)).to(device),
    )
    if with_rhs:
        dp.b = torch.from_numpy(np.asarray(problem.b, dtype=np.float64)).to(device)
    return dp
