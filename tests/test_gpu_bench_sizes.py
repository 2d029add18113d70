"""Oracle parity at the region sizes the benchmark times.

The full-size workloads (256 regions with 28/55/82 nodes per axis; 512 regions of 55^3) are too
large for the oracle, so these tests take 2 x 2 x 2-region samples built from the same
generators and seeds: regions of 28, 55 and 82 nodes per axis, hence many run tiles per region,
box tiles on the coarse levels, and the FP32 cycle's half planes at full region size. The
hierarchy options are the bench's (Chebyshev degree 3, nu 1/1, 4 levels, autotuned tiles).

Tolerances as in the small parity tests: V-cycle iterates 1e-10 relative (FP64), identical
PCG iteration counts; the FP32 cycle within 1e-4 of the FP64 oracle cycle (its coarse
operators and lambda are FP32 quantities, see test_gpu_mixed).
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import rel_max

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

CYCLE_TOL = 1e-10
FP32_CYCLE_TOL = 1e-4

SAMPLES = {
    # 2 x 2 x 2 regions, per-axis node counts drawn from {28, 55, 82} with the diffusion seed
    "diffusion3d_7pt_28_55_82": lambda: W.diffusion3d_7pt(region_grid=(2, 2, 2),
                                                          choices=(28, 55, 82), seed=1),
    # 2 x 2 x 2 regions of 55^3 nodes, Q1 27-point
    "q1_laplace3d_55": lambda: W.q1_laplace3d(region_grid=(2, 2, 2), n=55, seed=2),
}
_cache = {}


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_11962_gb300 import rmg
    return rmg.Context(0)


def _sample(name):
    if name not in _cache:
        from oracle import cycle, hierarchy
        p = SAMPLES[name]()
        levels = hierarchy.build(p, 4)
        mg = cycle.RegionalMG(levels, cycle.Options(smoother="chebyshev", nu1=1, nu2=1, degree=3))
        _cache[name] = (p, levels, mg)
    return _cache[name]


def _gpu(ctx, p, precision, tile_shape=-1):
    from paper_2103_11962_gb300 import rmg, upload
    dp = upload(p)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
    o = rmg.default_options(levels=4, precision=precision, tile_shape=tile_shape)
    o.smoother, o.nu1, o.nu2, o.cheb_degree = rmg.CHEBYSHEV, 1, 1, 3
    return dp, lay, rmg.Hierarchy(lay, o)


@pytest.mark.parametrize("name", list(SAMPLES))
def test_vcycle_at_bench_region_sizes(ctx, name):
    p, levels, mg = _sample(name)
    assert max(max(d) for d in p.region_dims) >= 55
    L0 = levels[0].layout
    expect = L0.average_to_composite(mg.precondition(L0.to_regional(p.b)))
    # the autotuned tiles, and a box shape forced on every level
    for shape in (-1, 8):
        dp, lay, h = _gpu(ctx, p, 0, shape)
        z = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
        h.vcycle(dp.b, z)
        err = rel_max(z.cpu().numpy(), expect)
        assert err <= CYCLE_TOL, (shape, err, [h.tile_shape(l) for l in range(4)])
        h.close()
        lay.close()


@pytest.mark.parametrize("name", list(SAMPLES))
def test_pcg_at_bench_region_sizes(ctx, name):
    from oracle import krylov
    p, levels, mg = _sample(name)
    x_or, it_or, hist_or = krylov.pcg(p.A, p.b, krylov.regional_preconditioner(mg), rtol=1e-10)
    dp, lay, h = _gpu(ctx, p, 0)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    res = h.pcg(dp.b, x, rtol=1e-10, maxit=300)
    assert res["converged"] and res["iterations"] == it_or, (res["iterations"], it_or)
    assert np.abs(res["history"] - np.asarray(hist_or)).max() <= 1e-8 * hist_or[0]
    xo = x.cpu().numpy()
    assert np.linalg.norm(xo - x_or) <= 1e-9 * np.linalg.norm(x_or)


@pytest.mark.parametrize("name", list(SAMPLES))
def test_fp32_cycle_at_bench_region_sizes(ctx, name):
    """The bench's headline cycle (FP32, half planes on level 0) against the FP64 oracle."""
    from oracle import krylov
    p, levels, mg = _sample(name)
    L0 = levels[0].layout
    expect = L0.average_to_composite(mg.precondition(L0.to_regional(p.b)))
    dp, lay, h = _gpu(ctx, p, 1)
    assert h.coef_planes(0) == (p.stencil + 1) // 2          # half planes in use
    z = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
    h.vcycle(dp.b, z)
    err = rel_max(z.cpu().numpy(), expect)
    assert err <= FP32_CYCLE_TOL, err
    x_or, it_or, _ = krylov.pcg(p.A, p.b, krylov.regional_preconditioner(mg), rtol=1e-10)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    res = h.pcg(dp.b, x, rtol=1e-10, maxit=300)
    assert res["converged"] and res["true_relres"] <= 1e-10
    assert res["iterations"] <= it_or + 3
    assert np.linalg.norm(x.cpu().numpy() - x_or) <= 1e-6 * np.linalg.norm(x_or)



@pytest.mark.parametrize("name", list(SAMPLES))
def test_fp32_tile_shapes_identical_at_bench_region_sizes(ctx, name):
    """Runs, box shapes and (27-point) the shared-memory staged columns give the same FP32
    cycle bit for bit at the bench's region sizes, with the half planes in use."""
    p, levels, mg = _sample(name)
    ref = None
    for shape in (0, 1, 8, 9):
        dp, lay, h = _gpu(ctx, p, 1, shape)
        assert h.coef_planes(0) == (p.stencil + 1) // 2
        if shape == 9:
            assert h.tile_shape(0) == ((32, 8, 0) if p.stencil == 27 else (0, 0, 0))
        z = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
        h.vcycle(dp.b, z)
        zc = z.cpu().numpy()
        if ref is None:
            ref = zc
        else:
            assert np.array_equal(zc, ref), shape
        h.close()
        lay.close()
