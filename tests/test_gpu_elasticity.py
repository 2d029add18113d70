"""3D linear elasticity (3 dofs per node, 3x3-block 27-point stencils) on the GPU against the
block oracle (component-major regional vectors, node-major composite vectors)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from tests.gpu_common import matrix_rel_diff, rel_max, stencils_to_matrix

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]


# 10 power steps underestimate lambda_max(D^-1 A) of Q1 elasticity by more than the 1.1 boost,
# so the elasticity hierarchies take 30 (as the elasticity bench workload does)
POWER_ITERS = 30


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_11962_gb300 import rmg
    return rmg.Context(0)


@pytest.fixture(scope="module")
def case():
    from oracle import cycle, hierarchy
    p = W.elasticity3d(region_grid=(2, 2, 2), choices=(10, 19), seed=4)
    levels = hierarchy.build_block(p, 3)
    mg = cycle.RegionalMG(levels, cycle.Options(smoother="chebyshev", nu1=1, nu2=1, degree=3,
                                                power_iters=POWER_ITERS))
    return p, levels, mg


def _gpu(ctx, p, precision=0):
    from paper_2103_11962_gb300 import rmg, upload
    dp = upload(p)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_block_csr(27, 3, dp.rowptr, dp.col, dp.val)
    o = rmg.default_options(levels=3, smoother=rmg.CHEBYSHEV, nu1=1, nu2=1, cheb_degree=3,
                            precision=precision, power_iters=POWER_ITERS)
    return dp, lay, rmg.Hierarchy(lay, o)


def _block_matrix(region_dims, coef, kind, B=3):
    n_r = coef.size // (B * B * kind)
    blocks = coef.reshape(B * B, kind * n_r)
    return sp.bmat([[stencils_to_matrix(region_dims, blocks[c * B + c2], kind) for c2 in range(B)]
                    for c in range(B)], format="csr")


def test_block_hierarchy_operators(ctx, case):
    p, levels, mg = case
    dp, lay, h = _gpu(ctx, p)
    assert h.dofs_per_node() == 3
    for l, lev in enumerate(levels):
        n_r, _, kind = h.level_sizes(l)
        coef = torch.empty(9 * kind * n_r, dtype=torch.float64, device="cuda")
        dinv = torch.empty(3 * n_r, dtype=torch.float64, device="cuda")
        h.level_export(l, coeffs=coef, dinv=dinv)
        M = _block_matrix(lev.layout.region_dims, coef.cpu().numpy(), kind)
        assert matrix_rel_diff(M, lev.Ar) <= 1e-12, l
        assert rel_max(dinv.cpu().numpy(), lev.Dinv_r) <= 1e-12
        assert abs(h.lam(l) - (mg.levels[l].lam_r or 0)) <= 1e-12 * abs(mg.levels[l].lam_r or 1) \
            if l < len(levels) - 1 else True


def test_block_apply_vcycle_and_pcg(ctx, case):
    from oracle import hierarchy, krylov
    p, levels, mg = case
    dp, lay, h = _gpu(ctx, p)
    n = p.n_nodes
    perm = hierarchy.node_major_to_component_major(n, 3)
    L0 = levels[0].layout
    # regional apply
    x = np.random.default_rng(3).standard_normal(3 * n)
    xr = torch.empty(3 * lay.sizes()["n_regional"], dtype=torch.float64, device="cuda")
    yr = torch.empty_like(xr)
    lay.comp_to_reg(torch.from_numpy(x).cuda(), xr)
    lay.regional_apply(xr, yr)
    expect = L0.to_regional(levels[0].A @ x[perm])
    assert rel_max(yr.cpu().numpy(), expect) <= 1e-12
    # V-cycle (composite node-major in and out)
    z = torch.empty(3 * n, dtype=torch.float64, device="cuda")
    h.vcycle(dp.b, z)
    ez = L0.average_to_composite(mg.precondition(L0.to_regional(p.b[perm])))
    zc = np.empty(3 * n); zc[perm] = ez
    assert rel_max(z.cpu().numpy(), zc) <= 1e-10
    # PCG: identical iteration counts
    x_or, it_or, hist_or = krylov.pcg(levels[0].A, p.b[perm], krylov.regional_preconditioner(mg),
                                      rtol=1e-10)
    xg = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    res = h.pcg(dp.b, xg, rtol=1e-10, maxit=300)
    print("elasticity PCG: gpu", res["iterations"], ["%.3e" % v for v in res["history"][-4:]],
          "oracle", it_or, ["%.3e" % v for v in hist_or[-4:]])
    assert res["converged"] and res["true_relres"] <= 1.5e-10
    assert res["iterations"] == it_or
    assert np.abs(res["history"] / np.asarray(hist_or) - 1.0).max() <= 1e-6
    xo = np.empty(3 * n); xo[perm] = x_or
    assert np.linalg.norm(xg.cpu().numpy() - xo) <= 1e-8 * np.linalg.norm(xo)


def test_block_coarse_matrix(ctx, case):
    from oracle import hierarchy
    p, levels, mg = case
    dp, lay, h = _gpu(ctx, p)
    dense, ids = h.coarse_matrix()
    last = levels[-1]
    ns = last.extra["slay"].n
    free = np.flatnonzero(~last.extra["slay"].mask)
    assert np.array_equal(ids, free)
    Abar = hierarchy.coarse_composite_from_regional(last).toarray()
    # oracle: component-major (c * ns + g); GPU: dof cu * 3 + c over free nodes
    idx = np.array([c * ns + g for g in free for c in range(3)])
    assert rel_max(dense, Abar[np.ix_(idx, idx)]) <= 1e-12


def test_block_mixed_precision_reaches_fp64_tolerance(ctx, case):
    p, levels, mg = case
    for prec in (1, 2):
        dp, lay, h = _gpu(ctx, p, precision=prec)
        xg = torch.zeros(3 * p.n_nodes, dtype=torch.float64, device="cuda")
        res = h.pcg(dp.b, xg, rtol=1e-10, maxit=300)
        assert res["converged"] and res["true_relres"] <= 2e-10
