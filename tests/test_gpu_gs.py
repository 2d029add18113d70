"""Region Gauss-Seidel (Algorithm 1 in multicolour order) on the GPU against the oracle: the
V-cycle to 1e-10, flexible PCG with identical iteration counts, the mixed-precision cycle, and
the rejection of block operators."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import rel_max
from tests.test_gpu_parity import _problem

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

NAMES = ["c1_poisson2d", "poisson2d_uneven", "q1_2d", "diff3d_small", "q1_3d_small",
         "highcontrast_small"]


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_11962_gb300 import rmg
    return rmg.Context(0)


def _gpu(ctx, name, nu, omega, precision=0):
    from paper_2103_11962_gb300 import rmg, upload
    p, nlev = _problem(name)
    dp = upload(p)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
    o = rmg.default_options(levels=nlev, smoother=rmg.GAUSS_SEIDEL, nu1=nu, nu2=nu, omega=omega,
                            precision=precision)
    return p, nlev, dp, lay, rmg.Hierarchy(lay, o)


def _oracle(p, nlev, nu, omega):
    from oracle import cycle, hierarchy
    levels = hierarchy.build(p, nlev)
    return levels, cycle.RegionalMG(levels, cycle.Options(smoother="gs", nu1=nu, nu2=nu,
                                                          omega=omega))


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("nu,omega", [(1, 1.0), (2, 0.8)])
def test_gs_vcycle_matches_oracle(ctx, name, nu, omega):
    p, nlev, dp, lay, h = _gpu(ctx, name, nu, omega)
    levels, mg = _oracle(p, nlev, nu, omega)
    L0 = levels[0].layout
    z = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
    for seed in (0, 1):
        rhs = dp.b if seed == 0 else torch.from_numpy(
            np.random.default_rng(7).uniform(-1, 1, p.n_nodes) * (1 - p.dirichlet)).cuda()
        h.vcycle(rhs, z)
        expect = L0.average_to_composite(mg.precondition(L0.to_regional(rhs.cpu().numpy())))
        assert rel_max(z.cpu().numpy(), expect) <= 1e-10, (name, seed)


@pytest.mark.parametrize("name", ["c1_poisson2d", "diff3d_small", "q1_3d_small"])
def test_gs_pcg_matches_oracle(ctx, name):
    from oracle import krylov
    p, nlev, dp, lay, h = _gpu(ctx, name, 1, 1.0)
    levels, mg = _oracle(p, nlev, 1, 1.0)
    x_or, it_or, hist_or = krylov.pcg(p.A, p.b, krylov.regional_preconditioner(mg), rtol=1e-10,
                                      flexible=True)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    res = h.pcg(dp.b, x, rtol=1e-10, maxit=300)
    assert res["converged"] and res["true_relres"] <= 1.5e-10
    assert res["iterations"] == it_or
    assert np.abs(res["history"] / np.asarray(hist_or) - 1.0).max() <= 1e-6
    assert np.linalg.norm(x.cpu().numpy() - x_or) <= 1e-8 * np.linalg.norm(x_or)


@pytest.mark.parametrize("precision", [1, 2])
def test_gs_mixed_reaches_fp64_tolerance(ctx, precision):
    p, nlev, dp, lay, h = _gpu(ctx, "diff3d_small", 1, 1.0, precision)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    res = h.pcg(dp.b, x, rtol=1e-10, maxit=300)
    assert res["converged"] and res["true_relres"] <= 2e-10


def test_gs_rejects_block_operators(ctx):
    from paper_2103_11962_gb300 import rmg, upload
    p = W.elasticity3d(region_grid=(2, 2, 2), choices=(10, 19), seed=4)
    dp = upload(p)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_block_csr(27, 3, dp.rowptr, dp.col, dp.val)
    with pytest.raises(rmg.RmgError):
        rmg.Hierarchy(lay, rmg.default_options(levels=3, smoother=rmg.GAUSS_SEIDEL))
