"""Mixed precision: FP32 V-cycle (FP32 or BF16 stencil coefficients) inside FP64 flexible CG.

The outer solve must still reach the FP64 relative residual 1e-10 and agree with the oracle's
FP64 solution; the V-cycle itself is compared against the FP64 oracle cycle with a tolerance
set by the arithmetic. A mixed hierarchy forms its coarse operators (Galerkin products) and its
Chebyshev lambda in FP32, so its operators carry relative errors up to 1e-5 (checked below),
which the coarse-grid correction passes to the cycle output at O(1): 1e-4 for the FP32 cycle.
BF16 coefficients carry 2^-9 relative rounding: 5e-2.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import rel_max
from tests.test_gpu_parity import _gpu, _oracle, _problem

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

VCYCLE_TOL = {1: 1e-4, 2: 5e-2}


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_11962_gb300 import rmg
    return rmg.Context(0)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("name", ["c1_poisson2d", "diff3d_small", "q1_3d_small"])
def test_mixed_vcycle_close_to_fp64_oracle(ctx, name, precision):
    smoother = "chebyshev"
    p, dp, lay, h = _gpu(ctx, name, smoother, precision=precision)
    levels, mg, _ = _oracle(name, smoother)
    L0 = levels[0].layout
    z = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
    h.vcycle(dp.b, z)
    expect = L0.average_to_composite(mg.precondition(L0.to_regional(p.b)))
    err = rel_max(z.cpu().numpy(), expect)
    assert err <= VCYCLE_TOL[precision], err


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("name", ["c1_poisson2d", "diff3d_small", "highcontrast_small"])
def test_mixed_pcg_reaches_fp64_tolerance(ctx, name, precision):
    from oracle import krylov
    smoother = "chebyshev"
    p, dp, lay, h = _gpu(ctx, name, smoother, precision=precision)
    levels, mg, _ = _oracle(name, smoother)
    x_or, it_or, _ = krylov.pcg(p.A, p.b, krylov.regional_preconditioner(mg), rtol=1e-10)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    res = h.pcg(dp.b, x, rtol=1e-10, maxit=300)
    assert res["converged"]
    assert res["true_relres"] <= 2e-10
    assert res["iterations"] <= it_or + (3 if precision == 1 else 8)
    xo = x.cpu().numpy()
    # both solutions satisfy the 1e-10 residual test; their difference is bounded by the
    # conditioning of A times that residual
    assert np.linalg.norm(xo - x_or) <= 1e-6 * np.linalg.norm(x_or)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("name", ["c1_poisson2d", "diff3d_small", "q1_3d_small"])
def test_mixed_hierarchy_galerkin_products_in_fp32(ctx, name, precision):
    """A mixed hierarchy forms its coarse operators in FP32 (they only enter the FP32 cycle):
    level 0 is the FP64 split exactly, coarser levels match the FP64 oracle's Galerkin products
    to FP32 accuracy (unit roundoff 6e-8 over sums of up to 11^3 terms)."""
    from tests.gpu_common import matrix_rel_diff, stencils_to_matrix
    p, dp, lay, h = _gpu(ctx, name, "chebyshev", precision=precision)
    levels, mg, _ = _oracle(name, "chebyshev")
    for l, lev in enumerate(levels):
        n_l, _, kind = h.level_sizes(l)
        coef = torch.empty(kind * n_l, dtype=torch.float64, device="cuda")
        h.level_export(l, coeffs=coef)
        M = stencils_to_matrix(lev.layout.region_dims, coef.cpu().numpy(), kind)
        err = matrix_rel_diff(M, lev.Ar)
        assert err <= (1e-12 if l == 0 else 1e-5), (l, err)
