"""Learned prolongator on the GPU: operator-dependent weights, stored-weight transfers, the
MLP's forward and gradient against the oracle, and the trained network against the plain
method."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import matrix_rel_diff, rel_max, stencils_to_matrix

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]


@pytest.fixture(scope="module")
def ctx():
    from paper_2103_11962_gb300 import rmg
    return rmg.Context(0)


def _hc(seed=13, grid=(3, 2, 2), choices=(10, 19)):
    return W.highcontrast3d_7pt(region_grid=grid, choices=choices, seed=seed)


def _setup(ctx, p, levels=3, smoother="chebyshev"):
    from paper_2103_11962_gb300 import learned, rmg, upload
    dp = upload(p)
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
    h = rmg.Hierarchy(lay, learned._options(levels, smoother))
    return dp, lay, h


def _opts(smoother):
    from oracle import cycle
    if smoother == "jacobi":
        return cycle.Options(smoother="jacobi", nu1=2, nu2=2, omega=0.67)
    return cycle.Options(smoother="chebyshev", nu1=1, nu2=1, degree=3)


def test_opdep_weights_match_oracle(ctx):
    from oracle.learned import opdep_weights
    for p in (_hc(), W.diffusion3d_7pt(region_grid=(2, 2, 2), choices=(10, 19, 28), seed=5)):
        dp, lay, h = _setup(ctx, p)
        n_r = lay.sizes()["n_regional"]
        wr = torch.empty(3 * n_r, dtype=torch.float32, device="cuda")
        h.opdep_weights(0, wr)
        got = wr.view(3, n_r).cpu().numpy().astype(np.float64)
        expect = opdep_weights(p.A, p.global_dims)[:, p.region_gids]
        free = ~p.dirichlet.astype(bool)[p.region_gids]
        # FP64 weights rounded to FP32 (unit roundoff 6e-8 on values in [0, 1])
        assert np.abs(got[:, free] - expect[:, free]).max() <= 1.2e-7


def test_stored_weight_hierarchy_matches_oracle(ctx):
    """Operator-dependent weights on level 0: Galerkin operators, V-cycle and PCG agree with
    the oracle built on the same weights."""
    from oracle import cycle, hierarchy, krylov
    from oracle.learned import opdep_weights
    p = _hc()
    for smoother in ("jacobi", "chebyshev"):
        dp, lay, h = _setup(ctx, p, 3, smoother)
        n_r = lay.sizes()["n_regional"]
        wr = torch.empty(3 * n_r, dtype=torch.float32, device="cuda")
        h.opdep_weights(0, wr)
        h.set_transfer_weights(0, wr)
        h.setup_numeric()
        # the stored weights are an input of the transfer: hand the same FP32 values to the
        # oracle (composite id -> weights; co-located copies hold identical values)
        w0 = np.zeros((3, p.n_nodes), dtype=np.float32)
        w0[:, p.region_gids] = wr.view(3, n_r).cpu().numpy()
        levels = hierarchy.build(p, 3, weights=lambda l, lev: w0 if l == 0 else None)
        mg = cycle.RegionalMG(levels, _opts(smoother))
        for l, lev in enumerate(levels):
            n_l, _, kind = h.level_sizes(l)
            coef = torch.empty(kind * n_l, dtype=torch.float64, device="cuda")
            h.level_export(l, coeffs=coef)
            M = stencils_to_matrix(lev.layout.region_dims, coef.cpu().numpy(), kind)
            assert matrix_rel_diff(M, lev.Ar) <= 1e-12, (smoother, l)
        L0 = levels[0].layout
        z = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
        h.vcycle(dp.b, z)
        expect = L0.average_to_composite(mg.precondition(L0.to_regional(p.b)))
        assert rel_max(z.cpu().numpy(), expect) <= 1e-10
        x_or, it_or, _ = krylov.pcg(p.A, p.b, krylov.regional_preconditioner(mg), rtol=1e-10)
        x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
        res = h.pcg(dp.b, x, rtol=1e-10, maxit=200)
        assert res["iterations"] == it_or
        # restoring linear interpolation gives back the plain hierarchy
        h.set_transfer_weights(0, None)
        h.setup_numeric()
        plain = cycle.RegionalMG(hierarchy.build(p, 3), _opts(smoother))
        h.vcycle(dp.b, z)
        expect = L0.average_to_composite(plain.precondition(L0.to_regional(p.b)))
        assert rel_max(z.cpu().numpy(), expect) <= 1e-10


def test_convergence_factor_matches_oracle(ctx):
    from oracle import cycle, hierarchy
    from oracle.rng import uniform_pm1
    p = _hc()
    dp, lay, h = _setup(ctx, p, 3, "chebyshev")
    fac = h.convergence_factor(5, 11)
    levels = hierarchy.build(p, 3)
    mg = cycle.RegionalMG(levels, _opts("chebyshev"))
    L0 = levels[0].layout
    e = uniform_pm1(11, np.arange(p.n_nodes))
    e[p.dirichlet.astype(bool)] = 0.0
    er = L0.to_regional(e)
    A = lambda v: L0.interface_sum(levels[0].Ar @ v)
    e0 = L0.dot(er, A(er))
    for _ in range(5):
        er = er - mg.precondition(A(er))
    e5 = L0.dot(er, A(er))
    assert fac == pytest.approx((e5 / e0) ** (0.5 / 5), rel=1e-8)


def test_features_identical_on_copies(ctx):
    p = _hc()
    dp, lay, h = _setup(ctx, p)
    n_r = lay.sizes()["n_regional"]
    feats = torch.empty((n_r, 32), dtype=torch.float32, device="cuda")
    h.mlp_features(0, feats)
    f = feats.cpu().numpy()
    g = p.region_gids
    order = np.argsort(g, kind="stable")
    gs = g[order]
    same = gs[1:] == gs[:-1]
    assert same.any()
    assert np.array_equal(f[order][1:][same], f[order][:-1][same])
    assert np.isfinite(f).all()


def test_mlp_forward_and_gradient_match_oracle(ctx):
    """The forward outputs and every gradient entry against the oracle network with the same
    BF16 roundings. The GPU accumulates in FP32 where the oracle uses FP64, so a hidden
    activation can round to the neighbouring BF16 value (a relative step of 2^-8); such rare
    flips bound the per-entry tolerances."""
    from oracle import learned as Lo
    from paper_2103_11962_gb300 import learned, rmg
    p = _hc()
    dp, lay, h = _setup(ctx, p)
    n_r = lay.sizes()["n_regional"]
    feats = torch.empty((n_r, 32), dtype=torch.float32, device="cuda")
    h.mlp_features(0, feats)
    rng = np.random.default_rng(5)
    sel = rng.choice(n_r, 1000, replace=False)
    X = feats[torch.from_numpy(sel).cuda()].contiguous()
    Y = torch.from_numpy(rng.uniform(0, 1, (1000, 3)).astype(np.float32)).cuda()
    M = torch.from_numpy((rng.uniform(0, 1, (1000, 3)) > 0.25).astype(np.float32)).cuda()
    params = learned.init_params(3)
    net = rmg.MLP(ctx, params)
    out = torch.empty((1000, 3), dtype=torch.float32, device="cuda")
    net.forward(X, out)
    Xh = X.cpu().numpy().astype(np.float64)
    O_or, _ = Lo.forward(params.astype(np.float64), Xh)
    d = np.abs(out.cpu().numpy() - O_or)
    print(f"forward: max |O - O_or| = {d.max():.3e}, 99.9th pct {np.quantile(d, 0.999):.3e}")
    assert d.max() <= 1e-3                         # every entry
    assert np.quantile(d, 0.999) <= 1e-5           # all but BF16 rounding flips
    loss, g = net.gradient(X, Y, M)
    L_or, g_or = Lo.loss_and_grad(params.astype(np.float64), Xh,
                                  Y.cpu().numpy().astype(np.float64),
                                  M.cpu().numpy().astype(np.float64))
    assert loss == pytest.approx(L_or, rel=1e-4)
    err = np.abs(g - g_or)
    scale = np.abs(g_or).max()
    print(f"gradient: max |g - g_or| / max |g_or| = {err.max() / scale:.3e}")
    # every entry: 1e-3 of itself plus 1e-4 of the largest entry
    assert np.all(err <= 1e-3 * np.abs(g_or) + 1e-4 * scale)


def test_features_match_oracle(ctx):
    """Network inputs of every regional node against the oracle's features of its composite
    node (FP64 ratios, FP32 logarithms on the GPU)."""
    from oracle import learned as Lo
    for p in (_hc(), W.diffusion3d_7pt(region_grid=(2, 2, 2), choices=(10, 19, 28), seed=5)):
        dp, lay, h = _setup(ctx, p)
        n_r = lay.sizes()["n_regional"]
        feats = torch.empty((n_r, 32), dtype=torch.float32, device="cuda")
        h.mlp_features(0, feats)
        expect = Lo.features(p.A, p.global_dims)[p.region_gids]
        got = feats.cpu().numpy().astype(np.float64)
        assert np.abs(got - expect).max() <= 4e-6


def test_predicted_weights_match_oracle(ctx):
    """rmg_hier_mlp_weights against the oracle pipeline from the same parameters: oracle
    features of the composite operator, the oracle network with the GPU's BF16 roundings,
    zero weights along inactive axes. The features enter the network rounded to BF16, so a
    feature that differs in its last FP32 bits can round the other way; the tolerance covers
    such rare flips, and nearly every weight must agree to FP32-accumulation level."""
    from oracle import learned as Lo
    from paper_2103_11962_gb300 import learned, rmg
    p = _hc()
    dp, lay, h = _setup(ctx, p)
    n_r = lay.sizes()["n_regional"]
    params = learned.init_params(9)
    net = rmg.MLP(ctx, params)
    wr = torch.empty(3 * n_r, dtype=torch.float32, device="cuda")
    h.mlp_weights(0, net, wr)
    Fo = Lo.features(p.A, p.global_dims)
    Oo, _ = Lo.forward(params.astype(np.float64), Fo)
    expect = Lo.weights_from_outputs(Fo, Oo)[:, p.region_gids]
    got = wr.view(3, n_r).cpu().numpy().astype(np.float64)
    d = np.abs(got - expect)
    print(f"weights: max diff {d.max():.3e}, 99.9th pct {np.quantile(d, 0.999):.3e}")
    assert np.all((got == 0) == (expect == 0))
    assert d.max() <= 2e-3
    assert np.quantile(d, 0.999) <= 1e-5
    net.close()


def test_trained_network_against_plain_method(ctx):
    """Train on small log-normal-coefficient operators labelled by the plain method, then
    compare on held-out operators: a C2-shaped one (the network must not lose against linear
    interpolation and its gain is reported) and a high-contrast one whose jumps sit on coarse
    grid planes (linear interpolation is already the operator-dependent one there; the
    accept rule must keep the plain prolongator or an equivalent one)."""
    from paper_2103_11962_gb300 import learned
    mk = lambda s: W.diffusion3d_7pt(region_grid=(2, 2, 2), choices=(10, 19, 28), seed=2000 + s)
    F, Y, M, factors = learned.training_set(ctx, range(16), mk)
    assert F.shape[0] == Y.shape[0] == M.shape[0]
    assert np.mean(factors[:, 1] < factors[:, 0]) > 0.5       # the teacher usually wins
    net, hist = learned.train(ctx, F, Y, M, steps=600, batch=8192, lr=2e-3)
    assert np.isfinite(hist).all()
    assert hist[-50:].mean() < 0.5 * hist[:10].mean()
    for p in (W.diffusion3d_7pt(region_grid=(3, 3, 2), choices=(10, 19, 28), seed=77),
              W.highcontrast3d_7pt(region_grid=(3, 3, 2), choices=(10, 19), seed=77)):
        dp, lay, h = _setup(ctx, p, 3)
        x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
        plain = h.pcg(dp.b, x, rtol=1e-10, maxit=300)
        res = learned.apply_learned(h, net, lay.sizes()["n_regional"])
        x.zero_()
        after = h.pcg(dp.b, x, rtol=1e-10, maxit=300)
        print(f"{p.name}: plain {plain['iterations']} its (factor {res['factor_plain']:.4f}); "
              f"learned factor {res['factor_learned']:.4f}, accepted {res['accepted']}; "
              f"after: {after['iterations']} its")
        assert after["converged"] and after["true_relres"] <= 1.5e-10
        assert res["factor"] <= res["factor_plain"]
        if res["accepted"]:
            assert after["iterations"] <= plain["iterations"] + 1
        else:
            assert after["iterations"] == plain["iterations"]
        if p.name == "diffusion3d_7pt":
            assert res["factor"] < res["factor_plain"] * 1.01


def test_region_energies_match_oracle(ctx):
    """e_k^T A^(k) e_k of every region, before and after cycles of e <- e - M^-1 A e from the
    same SplitMix64 error, against the oracle's split region matrices; their sum is e^T A e."""
    from oracle import cycle, hierarchy
    from oracle.rng import uniform_pm1
    p = _hc()
    dp, lay, h = _setup(ctx, p, 3, "chebyshev")
    e0, eK = h.region_energies(4, 11)
    levels = hierarchy.build(p, 3)
    mg = cycle.RegionalMG(levels, _opts("chebyshev"))
    L0 = levels[0].layout
    e = uniform_pm1(11, np.arange(p.n_nodes))
    e[p.dirichlet.astype(bool)] = 0.0
    er = L0.to_regional(e)
    A = lambda v: L0.interface_sum(levels[0].Ar @ v)
    sizes = np.prod(np.asarray(p.region_dims).reshape(-1, 3), axis=1)
    reg = np.repeat(np.arange(len(sizes)), sizes)
    energy = lambda v: np.bincount(reg, weights=v * (levels[0].Ar @ v), minlength=len(sizes))
    o0 = energy(er)
    assert np.abs(e0 - o0).max() <= 1e-12 * np.abs(o0).max()
    assert np.all(o0 >= 0)
    assert e0.sum() == pytest.approx(L0.dot(er, A(er)), rel=1e-12)
    for _ in range(4):
        er = er - mg.precondition(A(er))
    oK = energy(er)
    assert np.abs(eK - oK).max() <= 1e-9 * np.abs(oK).max()


def test_blend_weights_match_oracle(ctx):
    """Learned weights at nodes whose regions all accept, linear ones elsewhere (interface
    nodes shared with a rejecting region included), against the oracle's restatement."""
    from oracle import learned as Lo
    p = _hc()
    dp, lay, h = _setup(ctx, p)
    n_r = lay.sizes()["n_regional"]
    rng = np.random.default_rng(4)
    # candidate weights identical on co-located copies (drawn per composite node)
    wc = rng.uniform(0.05, 0.95, (3, p.n_nodes)).astype(np.float32)
    learned = torch.from_numpy(np.ascontiguousarray(wc[:, p.region_gids]).reshape(-1)).cuda()
    accept = (rng.uniform(size=p.nregions) > 0.5).astype(np.uint8)
    out = torch.empty(3 * n_r, dtype=torch.float32, device="cuda")
    h.blend_weights(0, accept, learned, out)
    expect = Lo.blend_weights(p.region_dims, p.region_gids, accept,
                              learned.view(3, n_r).cpu().numpy().astype(np.float64), p.dim)
    got = out.view(3, n_r).cpu().numpy().astype(np.float64)
    assert np.array_equal(got, expect)
    # copies of every composite node carry identical weights
    g = p.region_gids
    order = np.argsort(g, kind="stable")
    same = g[order][1:] == g[order][:-1]
    for a in range(3):
        w = got[a][order]
        assert np.array_equal(w[1:][same], w[:-1][same])


def test_batched_labels_match_single_operators(ctx):
    """Operators labelled side by side (disconnected components of one system) get the two-grid
    factors they get alone, up to the shared Chebyshev interval (lambda_max of the union)."""
    from paper_2103_11962_gb300 import learned
    mk = lambda s: W.highcontrast3d_7pt(region_grid=(2, 2, 2), choices=(10,), seed=1000 + s)
    ps = [mk(s) for s in range(4)]
    F, Y, M, fac = learned.label_batch(ctx, ps)
    assert fac.shape == (4, 2)
    n = 0
    for k, p in enumerate(ps):
        f1, y1, m1, (fl, fo) = learned.label_operator(ctx, p)
        assert fac[k, 0] == pytest.approx(fl, rel=0.05) and fac[k, 1] == pytest.approx(fo, rel=0.05)
        rows = slice(n, n + f1.shape[0])
        assert torch.equal(F[rows], f1)
        n += f1.shape[0]
    assert n == F.shape[0]


def test_per_region_acceptance_keeps_helpful_regions(ctx):
    """A candidate transfer that helps in some regions (operator-dependent weights on a
    high-contrast operator whose jumps lie off the coarse planes) and hurts in others (weights
    0.02, far from interpolating linears) is kept region by region: the harmful regions are
    rejected, some helpful ones kept, and the blend converges no worse than linear
    interpolation."""
    from paper_2103_11962_gb300 import learned
    p = W.highcontrast3d_offset(region_grid=(3, 2, 2), choices=(19,), seed=3)
    dp, lay, h = _setup(ctx, p, 2)
    n_r = lay.sizes()["n_regional"]
    good = torch.empty(3 * n_r, dtype=torch.float32, device="cuda")
    h.opdep_weights(0, good)
    bad = torch.where(good > 0, torch.full_like(good, 0.02), good)   # far from linear
    # the harmful weights go to every node of the odd regions, copies included (a composite
    # node in any odd region), so the candidate keeps identical copies
    reg = np.repeat(np.arange(p.nregions), np.prod(np.asarray(p.region_dims), axis=1))
    odd_comp = np.zeros(p.n_nodes, dtype=bool)
    np.logical_or.at(odd_comp, p.region_gids, reg % 2 == 1)
    hurt = torch.from_numpy(np.tile(odd_comp[p.region_gids], 3)).cuda()
    cand = torch.where(hurt, bad, good)
    res = learned.accept_per_region(h, cand, n_r)
    print({k: v for k, v in res.items() if k != "weights"})
    assert res["factor"] <= res["factor_plain"]
    assert 0 < res["regions_accepted"] < p.nregions
    assert res["factor_candidate"] > res["factor_blended"]
    assert not res["accept"][np.arange(p.nregions) % 2 == 1].any()   # harmful ones rejected
