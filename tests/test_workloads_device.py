"""The device-side workload generator (used for the full-size 3D Q1 Laplacian and elasticity
workloads) reproduces the numpy generators exactly: same CSR structure, same values, same
right-hand side (run here with torch on the CPU)."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")


def _same(p, d):
    A = p.A.tocsr()
    A.sort_indices()
    assert d.global_dims == tuple(p.global_dims)
    assert np.array_equal(d.region_dims, p.region_dims)
    assert np.array_equal(d.region_gids, p.region_gids)
    assert np.array_equal(d.dirichlet, p.dirichlet)
    assert np.array_equal(d.rowptr.numpy(), A.indptr)
    assert np.array_equal(d.col.numpy(), A.indices)
    assert np.array_equal(d.val.numpy(), A.data)          # bit for bit
    assert np.array_equal(d.b.numpy(), p.b)
    assert d.n_unknowns == p.n_unknowns and d.nnz == A.nnz
    rows = np.array([0, 5, A.shape[0] // 2, A.shape[0] - 1])
    R = d.rows(rows)
    assert abs(R[rows] - A[rows]).max() == 0.0


def test_q1_laplace3d_on_device_equals_numpy():
    from workloads import device as D
    p = W.q1_laplace3d(region_grid=(2, 2, 2), n=10, seed=2)
    d = D.q1_laplace3d(region_grid=(2, 2, 2), n=10, seed=2, device="cpu")
    _same(p, d)


def test_elasticity3d_on_device_equals_numpy():
    from workloads import device as D
    p = W.elasticity3d(region_grid=(2, 2, 2), choices=(10, 19), seed=4)
    d = D.elasticity3d(region_grid=(2, 2, 2), choices=(10, 19), seed=4, device="cpu")
    _same(p, d)


def test_diffusion3d_7pt_on_device_equals_numpy():
    from workloads import device as D
    p = W.diffusion3d_7pt(region_grid=(2, 3, 2), choices=(10, 19), seed=1)
    d = D.diffusion3d_7pt(region_grid=(2, 3, 2), choices=(10, 19), seed=1, device="cpu")
    _same(p, d)


def test_highcontrast3d_7pt_on_device_equals_numpy():
    from workloads import device as D
    p = W.highcontrast3d_7pt(region_grid=(3, 2, 2), choices=(10, 19), seed=3)
    d = D.highcontrast3d_7pt(region_grid=(3, 2, 2), choices=(10, 19), seed=3, device="cpu")
    _same(p, d)
