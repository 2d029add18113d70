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


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_pcg_does_not_depend_on_rhs_scale(ctx, precision):
    """Every CG inner product is FP64 and the FP32 cycle sees the residual scaled by a power of
    two near 1/||b||: b times 2^-83 (about 1e-25) or 2^83 (about 1e25) gives the same
    iterations and the solution times the same power of two, bit for bit; b times 1e-25 or
    1e25 gives the same iterations and the same solution up to rounding."""
    p, dp, lay, h = _gpu(ctx, "diff3d_small", "chebyshev", precision=precision)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    ref = h.pcg(dp.b, x, rtol=1e-10, maxit=300)
    assert ref["converged"]
    x_ref = x.clone()
    for e in (-83, 83):
        f = 2.0 ** e
        x.zero_()
        res = h.pcg(dp.b * f, x, rtol=1e-10, maxit=300)
        assert res["converged"] and res["iterations"] == ref["iterations"], (e, res)
        assert torch.equal(x, x_ref * f), e
    for f in (1e-25, 1e25):
        x.zero_()
        res = h.pcg(dp.b * f, x, rtol=1e-10, maxit=300)
        assert res["converged"] and res["iterations"] == ref["iterations"], (f, res)
        assert res["true_relres"] <= 1e-10
        assert torch.linalg.norm(x / f - x_ref) <= 1e-9 * torch.linalg.norm(x_ref)


def test_converged_means_true_residual_passes(ctx):
    """A reported convergence always holds for the true FP64 residual b - A x of the returned
    iterate, in every precision."""
    for precision in (0, 1, 2):
        for name in ("c1_poisson2d", "diff3d_small", "highcontrast_small"):
            p, dp, lay, h = _gpu(ctx, name, "chebyshev", precision=precision)
            x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
            res = h.pcg(dp.b, x, rtol=1e-10, maxit=300)
            assert res["converged"] and res["true_relres"] <= 1e-10, (precision, name, res)
            r = p.b - p.A @ x.cpu().numpy()
            assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(p.b) * (1 + 1e-6)
