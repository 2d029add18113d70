"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (fixed for the plain FP64 path): every operator apply and every setup product to
1e-12 relative to the largest entry; V-cycle iterates to 1e-10 relative; identical PCG
iteration counts.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import matrix_rel_diff, rel_max, stencils_to_matrix

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

OP_TOL = 1e-12
CYCLE_TOL = 1e-10

CASES = {
    # name: (factory, levels)
    "c1_poisson2d": (lambda: W.config("c1_poisson2d"), 4),
    "poisson2d_uneven": (lambda: W.poisson2d_5pt(region_grid=(3, 2), n=28, seed=11), 3),
    "q1_2d": (lambda: W.q1_laplace2d(region_grid=(2, 3), n=19, seed=12), 3),
    "diff3d_small": (lambda: W.diffusion3d_7pt(region_grid=(2, 2, 2), choices=(10, 19, 28),
                                               seed=5), 3),
    "q1_3d_small": (lambda: W.q1_laplace3d(region_grid=(2, 2, 1), n=19, seed=6), 3),
    "single_region": (lambda: W.diffusion3d_7pt(region_grid=(1, 1, 1), choices=(28,), seed=7), 3),
    "highcontrast_small": (lambda: W.highcontrast3d_7pt(region_grid=(3, 2, 2), choices=(10, 19),
                                                        seed=13), 3),
}

_cache = {}


def _problem(name):
    if name not in _cache:
        f, nlev = CASES[name]
        _cache[name] = (f(), nlev)
    return _cache[name]


def _oracle(name, smoother):
    from oracle import cycle, hierarchy
    key = ("oracle", name, smoother)
    if key not in _cache:
        p, nlev = _problem(name)
        levels = hierarchy.build(p, nlev)
        opts = _oracle_opts(smoother)
        mg = cycle.RegionalMG(levels, opts)
        _cache[key] = (levels, mg, opts)
    return _cache[key]


def _oracle_opts(smoother):
    from oracle import cycle
    if smoother == "jacobi":
        return cycle.Options(smoother="jacobi", nu1=2, nu2=2, omega=0.67)
    return cycle.Options(smoother="chebyshev", nu1=1, nu2=1, degree=3)


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_11962_gb300 import rmg
    return rmg.Context(0)


def _gpu(ctx, name, smoother, precision=0, use_graph=1):
    from paper_2103_11962_gb300 import rmg, upload
    p, nlev = _problem(name)
    dp = upload(p)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
    o = rmg.default_options(levels=nlev, use_graph=use_graph, precision=precision)
    if smoother == "jacobi":
        o.smoother, o.nu1, o.nu2, o.omega = rmg.JACOBI, 2, 2, 0.67
    else:
        o.smoother, o.nu1, o.nu2, o.cheb_degree = rmg.CHEBYSHEV, 1, 1, 3
    h = rmg.Hierarchy(lay, o)
    return p, dp, lay, h


@pytest.mark.parametrize("name", list(CASES))
def test_layout_and_split(ctx, name):
    from oracle.split import split_regional
    p, dp, lay, h = _gpu(ctx, name, "jacobi")
    levels, _, _ = _oracle(name, "jacobi")
    L0 = levels[0].layout
    sz = lay.sizes()
    assert sz["n_regional"] == L0.n_r and sz["n_composite"] == p.n_nodes
    assert sz["n_groups"] == int((L0.mult > 1).sum())
    assert sz["n_group_slots"] == int(L0.mult[L0.mult > 1].sum())
    n_r, _, kind = h.level_sizes(0)
    coef = torch.empty(kind * n_r, dtype=torch.float64, device="cuda")
    h.level_export(0, coeffs=coef)
    M = stencils_to_matrix(p.region_dims, coef.cpu().numpy(), kind)
    assert matrix_rel_diff(M, levels[0].Ar) <= OP_TOL


@pytest.mark.parametrize("name", ["diff3d_small", "q1_2d"])
def test_host_csr_split_matches_device_csr(ctx, name):
    """rmg_operator_from_host_csr (host arrays: pageable, page-locked, and page-locked at an odd
    8-byte offset) gives the same region stencils, bit for bit, as the split of the same CSR
    from device memory."""
    from paper_2103_11962_gb300 import rmg, upload
    p, _ = _problem(name)
    dp = upload(p)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
    h = rmg.Hierarchy(lay, rmg.default_options(levels=2))
    n_r, _, kind = h.level_sizes(0)
    ref = torch.empty(kind * n_r, dtype=torch.float64, device="cuda")
    h.level_export(0, coeffs=ref)
    A = p.A.tocsr()
    host = [np.ascontiguousarray(A.indptr.astype(np.int64)),
            np.ascontiguousarray(A.indices.astype(np.int64)),
            np.ascontiguousarray(A.data.astype(np.float64))]
    pinned = [torch.from_numpy(a).pin_memory() for a in host]
    # page-locked arrays that start 8 bytes past a 16-byte boundary (the copy kernel's 8-byte
    # path)
    shifted = []
    for a in host:
        t = torch.empty(a.size + 1, dtype=torch.from_numpy(a).dtype, pin_memory=True)
        t[1:].copy_(torch.from_numpy(a))
        shifted.append(t[1:])
    assert all(t.data_ptr() % 16 == 8 for t in shifted)
    for arrays in (host, pinned, shifted):
        lay.operator_from_host_csr(p.stencil, 1, *arrays)
        got = torch.empty_like(ref)
        h.level_export(0, coeffs=got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
    with pytest.raises(rmg.RmgError):
        lay.operator_from_host_csr(p.stencil, 2, *host)


def _renumbered_split(ctx, p, A, seed=3):
    """Level-0 region stencils of the same operator under the original composite numbering
    and under a random renumbering (entries kept in their row order)."""
    from paper_2103_11962_gb300 import rmg
    A = A.tocsr()
    out = []
    for permute in (False, True):
        perm = (np.random.default_rng(seed).permutation(p.n_nodes) if permute
                else np.arange(p.n_nodes))
        inv = np.argsort(perm)
        counts = np.diff(A.indptr)[inv]
        rowptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        take = np.concatenate([np.arange(A.indptr[g], A.indptr[g + 1]) for g in inv])
        col = perm[A.indices[take]].astype(np.int64)
        val = A.data[take].astype(np.float64)
        gids = torch.from_numpy(perm[np.asarray(p.region_gids)].astype(np.int64)).cuda()
        dirn = np.zeros(p.n_nodes, dtype=np.uint8)
        dirn[perm] = np.asarray(p.dirichlet, dtype=np.uint8)
        lay = rmg.Layout(ctx, p.dim, p.region_dims, gids, p.n_nodes,
                         torch.from_numpy(dirn).cuda())
        lay.operator_from_csr(p.stencil, torch.from_numpy(rowptr).cuda(),
                              torch.from_numpy(col).cuda(), torch.from_numpy(val).cuda())
        h = rmg.Hierarchy(lay, rmg.default_options(levels=2))
        n_r, _, kind = h.level_sizes(0)
        coef = torch.empty(kind * n_r, dtype=torch.float64, device="cuda")
        h.level_export(0, coeffs=coef)
        torch.cuda.synchronize()
        out.append(coef.cpu().numpy())
        h.close()
        lay.close()
    return out


def test_split_skips_couplings_to_other_regions_on_both_paths(ctx):
    """A symmetric pair of entries between interior nodes of two different regions couples no
    node of either region's own matrix: both the arithmetic shortcut of affine regions and the
    general path skip it in the off-diagonals (the diagonal keeps it through A 1), so the two
    give the same region stencils bit for bit. The pair is added as the positive semi-definite
    edge matrix 0.25 [[1, -1], [-1, 1]], so A 1 and the hierarchy's coarse operators stay as
    they were."""
    import scipy.sparse as sp
    p, _ = _problem("diff3d_small")
    A = p.A.tolil(copy=True)
    gids = np.asarray(p.region_gids)
    dims = np.asarray(p.region_dims)
    off = np.concatenate([[0], np.cumsum(np.prod(dims, axis=1))])
    a = int(gids[off[0] + 2 + dims[0][0] * (2 + dims[0][1] * 2)])      # (2,2,2) of region 0
    last = len(dims) - 1
    b = int(gids[off[last] + 3 + dims[last][0] * (3 + dims[last][1] * 3)])
    A[a, b] = -0.25
    A[b, a] = -0.25
    A[a, a] += 0.25
    A[b, b] += 0.25
    fast, general = _renumbered_split(ctx, p, sp.csr_matrix(A))
    assert np.array_equal(fast, general)


@pytest.mark.parametrize("name", ["diff3d_small", "q1_3d_small", "q1_2d"])
def test_split_diagonal_of_single_copy_rows_is_the_matrix_diagonal(ctx, name):
    """For a node with one copy every in-region coupling enters both sums of the nullspace rule
    whole, so its split diagonal is A_ii plus its couplings to other regions (none in these
    box layouts): the split must return A_ii bit for bit, and every off-diagonal of such a row
    the matrix entry itself."""
    from paper_2103_11962_gb300 import rmg, upload
    p, _ = _problem(name)
    dp = upload(p)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
    h = rmg.Hierarchy(lay, rmg.default_options(levels=2))
    n_r, _, kind = h.level_sizes(0)
    coef = torch.empty(kind * n_r, dtype=torch.float64, device="cuda")
    h.level_export(0, coeffs=coef)
    C = coef.cpu().numpy().reshape(kind, n_r)
    gids = np.asarray(p.region_gids)
    single = np.bincount(gids, minlength=p.n_nodes)[gids] == 1
    A = p.A.tocsr()
    diag = A.diagonal()
    center = (kind - 1) // 2
    assert np.array_equal(C[center][single], diag[gids[single]])
    # off-diagonals of single-copy rows: the stencil entries are the matrix entries themselves
    M = stencils_to_matrix(p.region_dims, coef.cpu().numpy(), kind).tocoo()
    keep = single[M.row] & (M.row != M.col)
    r, c, v = M.row[keep], M.col[keep], M.data[keep]
    assert np.array_equal(v, np.asarray(A[gids[r], gids[c]]).ravel())
    h.close()
    lay.close()


@pytest.mark.parametrize("name", ["diff3d_small", "q1_3d_small", "q1_2d"])
def test_split_without_affine_numbering(ctx, name):
    """The split takes a shortcut for single-copy rows of regions whose composite ids are
    numbered lexicographically (an affine gid map). Renumbering the composite nodes at random
    (rows and columns of A, gids and Dirichlet flags alike, entries kept in their row order)
    leaves no region affine, so every row takes the general path: the region stencils must be
    the same bit for bit."""
    p, _ = _problem(name)
    fast, general = _renumbered_split(ctx, p, p.A)
    assert np.array_equal(fast, general)


@pytest.mark.parametrize("name", list(CASES))
def test_regional_apply_equals_composite(ctx, name):
    """Psi^T Psi [[A]] Psi^T x = Psi^T (A x) on the GPU (eq. regional residual)."""
    p, dp, lay, h = _gpu(ctx, name, "jacobi")
    rng = np.random.default_rng(3)
    x = rng.standard_normal(p.n_nodes)
    xd = torch.from_numpy(x).cuda()
    n_r = lay.sizes()["n_regional"]
    xr = torch.empty(n_r, dtype=torch.float64, device="cuda")
    yr = torch.empty_like(xr)
    lay.comp_to_reg(xd, xr)
    lay.regional_apply(xr, yr)
    yc = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
    lay.reg_to_comp(yr, yc, average=True)
    expect = p.A @ x
    assert rel_max(yc.cpu().numpy(), expect) <= OP_TOL
    # consistency: every copy of a shared node holds the same value
    from oracle.regions import make_layout
    L0 = make_layout(p.region_dims, p.region_gids, p.n_nodes, p.dirichlet)
    y = yr.cpu().numpy()
    assert rel_max(y, L0.to_regional(expect)) <= OP_TOL


@pytest.mark.parametrize("name", list(CASES))
def test_hierarchy_operators(ctx, name):
    """Every level's [[Abar]] (regional Galerkin product) and D~^-1 against the oracle."""
    p, dp, lay, h = _gpu(ctx, name, "jacobi")
    levels, _, _ = _oracle(name, "jacobi")
    for l, lev in enumerate(levels):
        n_r, ncomp, kind = h.level_sizes(l)
        assert n_r == lev.layout.n_r and ncomp == lev.layout.n
        coef = torch.empty(kind * n_r, dtype=torch.float64, device="cuda")
        dinv = torch.empty(n_r, dtype=torch.float64, device="cuda")
        gids = torch.empty(n_r, dtype=torch.int64, device="cuda")
        h.level_export(l, coeffs=coef, dinv=dinv, gids=gids)
        assert np.array_equal(gids.cpu().numpy(), lev.layout.region_gids)
        M = stencils_to_matrix(lev.layout.region_dims, coef.cpu().numpy(), kind)
        assert matrix_rel_diff(M, lev.Ar) <= OP_TOL, f"level {l}"
        assert rel_max(dinv.cpu().numpy(), lev.Dinv_r) <= OP_TOL


@pytest.mark.parametrize("name", ["c1_poisson2d", "diff3d_small", "q1_3d_small"])
def test_coarse_composite_matrix(ctx, name):
    from oracle import hierarchy
    p, dp, lay, h = _gpu(ctx, name, "jacobi")
    levels, mg, _ = _oracle(name, "jacobi")
    dense, ids = h.coarse_matrix()
    last = levels[-1]
    free = np.flatnonzero(~last.layout.mask)
    assert np.array_equal(ids, free)
    Abar = hierarchy.coarse_composite_from_regional(last).toarray()[np.ix_(free, free)]
    assert rel_max(dense, Abar) <= OP_TOL


@pytest.mark.parametrize("name", ["c1_poisson2d", "diff3d_small", "q1_2d", "highcontrast_small"])
def test_power_method_lambda(ctx, name):
    p, dp, lay, h = _gpu(ctx, name, "chebyshev")
    levels, mg, _ = _oracle(name, "chebyshev")
    for l in range(len(levels) - 1):
        assert h.lam(l) == pytest.approx(levels[l].lam_r, rel=1e-12)


@pytest.mark.parametrize("use_graph", [1, 0])
@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_matches_oracle(ctx, name, smoother, use_graph):
    p, dp, lay, h = _gpu(ctx, name, smoother, use_graph=use_graph)
    levels, mg, _ = _oracle(name, smoother)
    L0 = levels[0].layout
    z = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
    h.vcycle(dp.b, z)
    expect = L0.average_to_composite(mg.precondition(L0.to_regional(p.b)))
    assert rel_max(z.cpu().numpy(), expect) <= CYCLE_TOL
    # a second application on another right-hand side (graph replay, buffers reused)
    r2 = np.random.default_rng(9).uniform(-1, 1, p.n_nodes)
    r2[p.dirichlet.astype(bool)] = 0
    h.vcycle(torch.from_numpy(r2).cuda(), z)
    expect2 = L0.average_to_composite(mg.precondition(L0.to_regional(r2)))
    assert rel_max(z.cpu().numpy(), expect2) <= CYCLE_TOL


@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
@pytest.mark.parametrize("name", ["c1_poisson2d", "diff3d_small", "q1_3d_small",
                                  "highcontrast_small", "single_region"])
def test_pcg_matches_oracle(ctx, name, smoother):
    from oracle import krylov
    p, dp, lay, h = _gpu(ctx, name, smoother)
    levels, mg, _ = _oracle(name, smoother)
    x_or, it_or, hist_or = krylov.pcg(p.A, p.b, krylov.regional_preconditioner(mg), rtol=1e-10)
    x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
    res = h.pcg(dp.b, x, rtol=1e-10, maxit=200)
    assert res["converged"]
    assert res["iterations"] == it_or
    assert res["true_relres"] <= 1.5e-10
    assert rel_max(res["history"], np.asarray(hist_or)) <= 1e-6
    xo = x.cpu().numpy()
    assert np.linalg.norm(xo - x_or) <= 1e-8 * np.linalg.norm(x_or)


def test_setup_numeric_refresh(ctx):
    """New coefficients on the same mesh: the numeric setup and the captured graph follow."""
    from oracle import cycle, hierarchy
    from paper_2103_11962_gb300 import upload
    name = "diff3d_small"
    p, dp, lay, h = _gpu(ctx, name, "chebyshev")
    p2 = W.diffusion3d_7pt(region_grid=(2, 2, 2), choices=(10, 19, 28), seed=5, sigma=0.5)
    assert p2.global_dims == p.global_dims
    d2 = upload(p2)
    lay.operator_from_csr(p2.stencil, d2.rowptr, d2.col, d2.val)
    h.setup_numeric()
    levels = hierarchy.build(p2, 3)
    mg = cycle.RegionalMG(levels, _oracle_opts("chebyshev"))
    L0 = levels[0].layout
    z = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
    h.vcycle(d2.b, z)
    expect = L0.average_to_composite(mg.precondition(L0.to_regional(p2.b)))
    assert rel_max(z.cpu().numpy(), expect) <= CYCLE_TOL


def test_errors_are_reported(ctx):
    from paper_2103_11962_gb300 import rmg
    p = W.diffusion3d_7pt(region_grid=(2, 1, 1), choices=(10,), seed=1)
    gids = torch.from_numpy(p.region_gids.copy()).cuda()
    gids[5] = p.n_nodes + 3          # out of range
    with pytest.raises(rmg.RmgError) as e:
        rmg.Layout(ctx, 3, p.region_dims, gids, p.n_nodes, None)
    assert e.value.status == 2
    # region sizes that cannot be coarsened 3:1 are rejected at setup
    p = W.diffusion3d_7pt(region_grid=(2, 1, 1), choices=(9,), seed=1)
    from paper_2103_11962_gb300 import upload
    dp = upload(p)
    lay = rmg.Layout(ctx, 3, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(7, dp.rowptr, dp.col, dp.val)
    with pytest.raises(rmg.RmgError) as e:
        rmg.Hierarchy(lay, rmg.default_options(levels=2))
    assert e.value.status == 2
    # a 27-point matrix declared as 7-point fails the split
    q = W.q1_laplace3d(region_grid=(1, 1, 1), n=10)
    dq = upload(q)
    lay = rmg.Layout(ctx, 3, q.region_dims, dq.gids, q.n_nodes, dq.dirichlet)
    with pytest.raises(rmg.RmgError) as e:
        lay.operator_from_csr(7, dq.rowptr, dq.col, dq.val)
    assert e.value.status == 2
    # the context is still usable
    lay.operator_from_csr(27, dq.rowptr, dq.col, dq.val)


STAGED = (32, 8, 0)     # shared-memory staged columns: FP32 half planes of a 27-point level 0
SHAPES = [(0, 0, 0), (32, 8, 1), (64, 4, 1), (128, 2, 1), (16, 16, 1), (32, 4, 2), (16, 8, 2),
          (16, 4, 4), (8, 8, 4), STAGED]


@pytest.mark.parametrize("name", ["diff3d_small", "q1_3d_small", "c1_poisson2d"])
@pytest.mark.parametrize("precision", [0, 1])
def test_tile_shapes_give_identical_cycles(ctx, name, precision):
    """Every stencil-sweep tile shape (and the autotuned choice) computes each node's row with
    the same arithmetic, so V-cycles agree bit for bit; 2D levels take only tz = 1 boxes."""
    from paper_2103_11962_gb300 import rmg, upload
    p, nlev = _problem(name)
    dp = upload(p)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
    ref = None
    for k in [-1] + list(range(len(SHAPES))):
        o = rmg.default_options(levels=nlev, precision=precision, tile_shape=k)
        o.smoother, o.nu1, o.nu2, o.cheb_degree = rmg.CHEBYSHEV, 1, 1, 3
        h = rmg.Hierarchy(lay, o)
        for l in range(nlev - 1):
            got = h.tile_shape(l)
            if k >= 0 and SHAPES[k] == STAGED:
                want = STAGED if (precision == 1 and p.stencil == 27 and l == 0) else (0, 0, 0)
                assert got == want, (k, l, got)
            elif k >= 0:
                want = SHAPES[k] if (p.dim == 3 or SHAPES[k][2] == 1) else (0, 0, 0)
                assert got == want, (k, l, got)
            else:
                assert got in SHAPES
        assert h.tile_shape(nlev - 1) == (0, 0, 0)
        z = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
        h.vcycle(dp.b, z)
        zc = z.cpu().numpy()
        if ref is None:
            ref = zc
        else:
            assert np.array_equal(zc, ref), k
        h.close()


def test_tile_shapes_block_operator(ctx):
    """Box tiles on a 3-dof-per-node (elasticity) hierarchy give the run-tile cycle exactly."""
    from paper_2103_11962_gb300 import rmg, upload
    p = W.elasticity3d(region_grid=(2, 2, 2), choices=(10, 19), seed=4)
    dp = upload(p)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_block_csr(27, 3, dp.rowptr, dp.col, dp.val)
    ref = None
    for k in (0, 5, 8, -1):
        o = rmg.default_options(levels=3, smoother=rmg.CHEBYSHEV, nu1=1, nu2=1, cheb_degree=3,
                                power_iters=30, tile_shape=k)
        h = rmg.Hierarchy(lay, o)
        z = torch.empty(3 * p.n_nodes, dtype=torch.float64, device="cuda")
        h.vcycle(dp.b, z)
        zc = z.cpu().numpy()
        if ref is None:
            ref = zc
        else:
            assert np.array_equal(zc, ref), k
        h.close()


def test_bad_tile_shape_is_an_error(ctx):
    from paper_2103_11962_gb300 import rmg, upload
    p, nlev = _problem("diff3d_small")
    dp = upload(p)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
    with pytest.raises(rmg.RmgError):
        rmg.Hierarchy(lay, rmg.default_options(levels=nlev, tile_shape=len(SHAPES)))
