"""Piecewise-constant 3:1 transfers (Table 4 'Const') on the GPU against the oracle."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import matrix_rel_diff, rel_max, stencils_to_matrix

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]


@pytest.mark.parametrize("factory", [
    lambda: W.poisson2d_5pt(region_grid=(2, 3), n=28, seed=4),
    lambda: W.diffusion3d_7pt(region_grid=(2, 2, 2), choices=(10, 19), seed=5),
])
def test_piecewise_constant_transfers(factory):
    from oracle import cycle, hierarchy, krylov
    from paper_2103_11962_gb300 import rmg, upload
    p = factory()
    ctx = rmg.Context(0)
    dp = upload(p)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
    h = rmg.Hierarchy(lay, rmg.default_options(levels=3, smoother=rmg.CHEBYSHEV, nu1=1, nu2=1))
    n_r = lay.sizes()["n_regional"]
    wr = torch.empty(3 * n_r, dtype=torch.float32, device="cuda")
    h.constant_weights(0, wr)
    w = wr.view(3, n_r).cpu().numpy()
    Nx, Ny, Nz = p.global_dims
    g = p.region_gids
    coord = [g % Nx, (g // Nx) % Ny, g // (Nx * Ny)]
    for a in range(3):
        assert np.array_equal(w[a], (coord[a] % 3 == 2).astype(np.float32))
    h.set_transfer_weights(0, wr)
    h.setup_numeric()
    w0 = np.zeros((3, p.n_nodes), dtype=np.float32)
    w0[:, g] = w
    levels = hierarchy.build(p, 3, weights=lambda l, lev: w0 if l == 0 else None)
    mg = cycle.RegionalMG(levels, cycle.Options(smoother="chebyshev", nu1=1, nu2=1, degree=3))
    for l, lev in enumerate(levels):
        n_l, _, kind = h.level_sizes(l)
        coef = torch.empty(kind * n_l, dtype=torch.float64, device="cuda")
        h.level_export(l, coeffs=coef)
        M = stencils_to_matrix(lev.layout.region_dims, coef.cpu().numpy(), kind)
        assert matrix_rel_diff(M, lev.Ar) <= 1e-12
    L0 = levels[0].layout
    z = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
    h.vcycle(dp.b, z)
    expect = L0.average_to_composite(mg.precondition(L0.to_regional(p.b)))
    assert rel_max(z.cpu().numpy(), expect) <= 1e-10
    x_or, it_or, _ = krylov.pcg(p.A, p.b, krylov.regional_preconditioner(mg), rtol=1e-10)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    res = h.pcg(dp.b, x, rtol=1e-10, maxit=400)
    assert res["converged"] and abs(res["iterations"] - it_or) <= 1


def test_galerkin_recompute_and_setup_only_hierarchy():
    """rmg_hier_galerkin recomputes exactly the coarse operator of the numeric setup (linear
    and stored transfers); a hierarchy whose coarsest level exceeds the dense solver is built
    for setup and introspection while cycles fail with an error."""
    from paper_2103_11962_gb300 import rmg, upload
    from tests.gpu_common import matrix_rel_diff, stencils_to_matrix
    from oracle import hierarchy
    ctx = rmg.Context(0)
    p = W.q1_laplace2d_box(3 * 80 - 2, 3 * 70 - 2)          # coarse level 80 x 70 = 5600
    dp = upload(p)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(9, dp.rowptr, dp.col, dp.val)
    h = rmg.Hierarchy(lay, rmg.default_options(levels=2))
    n1, _, kind = h.level_sizes(1)
    a = torch.empty(kind * n1, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    h.level_export(1, coeffs=a)
    h.galerkin(0)
    h.level_export(1, coeffs=b)
    assert torch.equal(a, b)
    lev = hierarchy.build(p, 2)
    M = stencils_to_matrix(lev[1].layout.region_dims, b.cpu().numpy(), kind)
    assert matrix_rel_diff(M, lev[1].Ar) <= 1e-12
    wr = torch.empty(3 * p.n_regional_nodes, dtype=torch.float32, device="cuda")
    h.constant_weights(0, wr)
    h.set_transfer_weights(0, wr)
    h.setup_numeric()
    h.level_export(1, coeffs=a)
    h.galerkin(0)
    h.level_export(1, coeffs=b)
    assert torch.equal(a, b)
    h.close()
    # 3 x 3 regions of 136 nodes: coarsest composite level 136 x 136 (134^2 = 17956 unknowns
    # inside the Dirichlet boundary, above the dense solver's 16384)
    q = W.q1_laplace2d(region_grid=(3, 3), n=136)
    dq = upload(q)
    lq = rmg.Layout(ctx, q.dim, q.region_dims, dq.gids, q.n_nodes, dq.dirichlet)
    lq.operator_from_csr(9, dq.rowptr, dq.col, dq.val)
    hq = rmg.Hierarchy(lq, rmg.default_options(levels=2))
    hq.galerkin(0)
    z = torch.empty(q.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(rmg.RmgError):
        hq.vcycle(dq.b, z)
    with pytest.raises(rmg.RmgError):
        hq.pcg(dq.b, z, rtol=1e-10, maxit=10)
