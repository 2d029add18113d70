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
