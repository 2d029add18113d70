"""The regional apply that allocates no device memory, against the regular entry point.

Callers whose device memory is owned by their own pool allocator, or that cannot afford the
synchronisation of a cudaMalloc, use rmg_regional_apply_static: it keeps its scratch in a
fixed device array inside the library. Its result must match rmg_regional_apply within the
operator tolerance of the parity tests, on two calls in a row (the second call reuses the
scratch left by the first, which must be cleared again). This file is collected last.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

OP_TOL = 1e-12


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("factory", [
    lambda: W.diffusion3d_7pt(region_grid=(2, 2, 2), choices=(10, 19, 28), seed=5),
    lambda: W.poisson2d_5pt(region_grid=(3, 2), n=28, seed=11),
    lambda: W.q1_laplace2d(region_grid=(2, 3), n=19, seed=12),
    lambda: W.q1_laplace3d(region_grid=(2, 2, 2), n=10, seed=6),
], ids=["7pt_3d", "5pt_2d", "9pt_2d", "27pt_3d"])
def test_static_apply_matches_regular_apply(factory):
    from paper_2103_11962_gb300 import rmg, upload
    p = factory()
    dp = upload(p)
    ctx = rmg.Context(0)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
    h = rmg.Hierarchy(lay, rmg.default_options(levels=3))
    n_r, _, kind = h.level_sizes(0)
    coef = torch.empty(kind * n_r, dtype=torch.float64, device="cuda")
    h.level_export(0, coeffs=coef)
    rng = np.random.default_rng(21)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        x = torch.from_numpy(rng.standard_normal(p.n_nodes)).cuda()
        u = torch.empty(n_r, dtype=torch.float64, device="cuda")
        lay.comp_to_reg(x, u)
        y_ref = torch.empty_like(u)
        lay.regional_apply(u, y_ref)
        y = torch.full_like(u, float("nan"))
        rmg.regional_apply_static(p.dim, p.region_dims, kind, coef, dp.gids, p.n_nodes, u, y,
                                  stream)
        torch.cuda.synchronize()
        yh, rh = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.isfinite(yh).all(), f"call {call}"
        assert _rel(yh, rh) <= OP_TOL, f"call {call}"


def test_static_apply_rejects_sizes_beyond_its_maximum():
    from paper_2103_11962_gb300 import rmg
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    gids = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(rmg.RmgError) as e:
        rmg.regional_apply_static(3, [[2, 2, 2]], 7, dummy, gids, (1 << 22) + 1, dummy, dummy)
    assert e.value.status == 1 and "4194304" in str(e.value)
