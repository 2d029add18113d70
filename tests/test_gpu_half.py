"""Half storage of the FP32 cycle's level-0 stencil (rmg_options.symmetric_storage).

Sec. 4 splits a symmetric composite matrix into symmetric region matrices, a(n, n+e) =
a(n+e, n). For such an operator the FP32 cycle reads only the centre and the slots after it
and takes each coefficient of the other half at the neighbour that owns its mirror. The half
form forms the same products in the same order as the full planes. So with the option on and
off, the cycle output, the Chebyshev lambda and the PCG iterates must agree bit for bit. An
operator whose FP32 pairs are not bitwise symmetric must keep the full planes.
"""
import numpy as np
import pytest

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


def _pair(ctx, p, nlev, A=None):
    """One layout, two FP32 hierarchies on it: symmetric storage on and off."""
    from paper_2103_11962_gb300 import rmg, upload
    dp = upload(p)
    if A is not None:
        A = A.tocsr()
        dp.rowptr = torch.from_numpy(A.indptr.astype(np.int64)).cuda()
        dp.col = torch.from_numpy(A.indices.astype(np.int64)).cuda()
        dp.val = torch.from_numpy(A.data.astype(np.float64)).cuda()
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
    hs = []
    for sym in (1, 0):
        o = rmg.default_options(levels=nlev, precision=rmg.FP32)
        o.smoother, o.nu1, o.nu2, o.cheb_degree = rmg.CHEBYSHEV, 1, 1, 3
        o.symmetric_storage = sym
        hs.append(rmg.Hierarchy(lay, o))
    return dp, lay, hs


def _bits(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("name", NAMES)
def test_half_form_is_bitwise_the_full_form(ctx, name):
    p, nlev = _problem(name)
    dp, lay, (hh, hf) = _pair(ctx, p, nlev)
    kind = p.stencil
    assert hh.coef_planes(0) == (kind + 1) // 2
    assert hf.coef_planes(0) == kind
    for l in range(1, nlev):
        assert hh.coef_planes(l) == hf.coef_planes(l) == hh.level_sizes(l)[2]
    for l in range(nlev - 1):
        assert hh.lam(l) == hf.lam(l)
    zh = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
    zf = torch.empty_like(zh)
    hh.vcycle(dp.b, zh)
    hf.vcycle(dp.b, zf)
    assert np.array_equal(_bits(zh), _bits(zf))
    xh = torch.zeros_like(zh)
    xf = torch.zeros_like(zh)
    rh = hh.pcg(dp.b, xh, rtol=1e-10, maxit=300)
    rf = hf.pcg(dp.b, xf, rtol=1e-10, maxit=300)
    assert rh["converged"] and rh["iterations"] == rf["iterations"]
    assert np.array_equal(_bits(xh), _bits(xf))


def _perturbed(p):
    """A with one off-diagonal entry inside region 0, between two single-copy free nodes, moved
    by 2^-10 relative (a[i, j] no longer a[j, i] in FP32)."""
    A = p.A.tocsr().copy()
    free = ~np.asarray(p.dirichlet, dtype=bool)
    gids = np.asarray(p.region_gids)
    mult = np.bincount(gids)[gids]          # copies of every regional node's composite node
    nx = int(p.region_dims[0][0])
    for n in range(nx + 1, len(gids) - 1):
        i, j = int(gids[n]), int(gids[n + 1])
        if mult[n] == 1 and mult[n + 1] == 1 and free[i] and free[j] and A[i, j] != 0:
            A[i, j] = A[i, j] * (1.0 + 2.0 ** -10)
            return A
    raise AssertionError("no interior pair found")


def test_asymmetric_operator_keeps_full_planes(ctx):
    p, nlev = _problem("diff3d_small")
    A = _perturbed(p)
    assert (A - A.T).count_nonzero() == 2
    dp, lay, (hh, hf) = _pair(ctx, p, nlev, A=A)
    assert hh.coef_planes(0) == hf.coef_planes(0) == 7
    zh = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
    zf = torch.empty_like(zh)
    hh.vcycle(dp.b, zh)
    hf.vcycle(dp.b, zf)
    assert np.array_equal(_bits(zh), _bits(zf))


def test_half_form_returns_after_the_operator_turns_symmetric_again(ctx):
    """The flag is recomputed at every numeric setup: the same hierarchy switches to the half
    form once the layout holds a symmetric operator again (same stencil, new values)."""
    p, nlev = _problem("diff3d_small")
    A = _perturbed(p)
    dp, lay, (hh, hf) = _pair(ctx, p, nlev, A=A)
    assert hh.coef_planes(0) == 7
    S = p.A.tocsr()
    dp.val.copy_(torch.from_numpy(S.data.astype(np.float64)))
    lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
    hh.setup_numeric()
    hf.setup_numeric()
    assert hh.coef_planes(0) == 4
    zh = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
    zf = torch.empty_like(zh)
    hh.vcycle(dp.b, zh)
    hf.vcycle(dp.b, zf)
    assert np.array_equal(_bits(zh), _bits(zf))


def test_coef_planes_of_other_precisions(ctx):
    from paper_2103_11962_gb300 import rmg, upload
    p, nlev = _problem("diff3d_small")
    dp = upload(p)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
    for prec in (rmg.FP64, rmg.FP32_BF16COEF):
        h = rmg.Hierarchy(lay, rmg.default_options(levels=nlev, precision=prec))
        assert h.coef_planes(0) == 7 and h.coef_planes(1) == 27
        with pytest.raises(Exception):
            h.coef_planes(nlev)


@pytest.mark.parametrize("perturb", [False, True])
def test_staged_sweep_matches_full_planes(ctx, perturb):
    """Tile shape 9 (27-point half planes staged through shared memory) against run tiles on
    the full planes: bitwise the same cycle for a symmetric operator, and for one whose FP32
    pairs differ (the staged kernel then reads the full planes itself)."""
    from paper_2103_11962_gb300 import rmg, upload
    p, nlev = _problem("q1_3d_small")
    dp = upload(p)
    if perturb:
        A = _perturbed(p)
        dp.val = torch.from_numpy(A.data.astype(np.float64)).cuda()
        dp.rowptr = torch.from_numpy(A.indptr.astype(np.int64)).cuda()
        dp.col = torch.from_numpy(A.indices.astype(np.int64)).cuda()
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
    out = []
    for sym, shape in ((1, 9), (0, 0)):
        o = rmg.default_options(levels=nlev, precision=rmg.FP32, tile_shape=shape)
        o.smoother, o.nu1, o.nu2, o.cheb_degree = rmg.CHEBYSHEV, 1, 1, 3
        o.symmetric_storage = sym
        h = rmg.Hierarchy(lay, o)
        assert h.tile_shape(0) == ((32, 8, 0) if sym else (0, 0, 0))
        assert h.coef_planes(0) == (27 if (perturb or not sym) else 14)
        z = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
        h.vcycle(dp.b, z)
        out.append((z, h.lam(0)))
        h.close()
    assert out[0][1] == out[1][1]
    assert np.array_equal(_bits(out[0][0]), _bits(out[1][0]))
