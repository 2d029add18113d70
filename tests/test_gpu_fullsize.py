"""Parity at full size, in the launch configuration the bench times: the 3D 7-point diffusion
workload with 256 regions of 28^3-82^3 nodes (29.4M unknowns) and the high-contrast workload
with 343 regions (33.5M unknowns); 4 levels, Chebyshev degree 3 with nu1 = nu2 = 1, the V-cycle
replayed as one CUDA graph, persistent grids over all regions.

The oracle cannot run the whole hierarchy at this size, so it checks what it can compute unit by
unit, on the same inputs:

* composite A x on the whole grid (the regional apply, Lemma 1: Psi^T Psi [[A]] Psi^T x = Psi^T A x),
* the split and the whole regional Galerkin chain of sampled regions (each region's chain
  [[Abar]]^(k) = P^(k)T A^(k) P^(k) depends on that region alone, Sec. 3.2 and Theorem 1),
* D~ on level 0 (the split rows sum back to the composite diagonal),
* the level-0 power method (Sec. 3.4) in composite form,

and the rest through properties that hold at any size: the V-cycle is symmetric and positive
(equal pre- and post-smoothing, R = P^T, exact coarse solve), and the PCG solutions of the FP64,
FP32 and BF16-coefficient cycles reach 1e-10 in the FP64 residual that the oracle recomputes from
the composite CSR.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from tests.gpu_common import stencils_to_matrix

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")]

OP_TOL = 1e-12
LEVELS = 4


def _options(rmg, precision):
    o = rmg.default_options(levels=LEVELS, precision=precision, use_graph=1)
    o.smoother, o.nu1, o.nu2, o.cheb_degree = rmg.CHEBYSHEV, 1, 1, 3
    return o


class Full:
    pass


@pytest.fixture(scope="module", params=["c2_diffusion3d", "c4_highcontrast3d"])
def full(request):
    from paper_2103_11962_gb300 import rmg, upload
    f = Full()
    f.name = request.param
    f.p = W.config(request.param)
    f.ctx = rmg.Context(0)
    f.dp = upload(f.p)
    p = f.p
    f.lay = rmg.Layout(f.ctx, p.dim, p.region_dims, f.dp.gids, p.n_nodes, f.dp.dirichlet)
    f.lay.operator_from_csr(p.stencil, f.dp.rowptr, f.dp.col, f.dp.val)
    f.h = rmg.Hierarchy(f.lay, _options(rmg, rmg.FP64))
    f.offsets = np.zeros(len(p.region_dims) + 1, dtype=np.int64)
    f.offsets[1:] = np.cumsum(np.prod(np.asarray(p.region_dims, dtype=np.int64), axis=1))
    f.mult = np.bincount(p.region_gids, minlength=p.n_nodes).astype(np.float64)
    yield f
    f.h.close()
    f.lay.close()
    del f.dp
    torch.cuda.empty_cache()


def _sample_regions(p):
    """A corner region (three Dirichlet faces), an interior one and the largest one."""
    rg = np.asarray([len(s) for s in p.slabs])
    interior = int(rg[0] // 2 + rg[0] * (rg[1] // 2 + rg[1] * (rg[2] // 2)))
    sizes = np.prod(np.asarray(p.region_dims, dtype=np.int64), axis=1)
    return sorted({0, interior, int(np.argmax(sizes))})


def _level_dims(dims, l):
    d = np.asarray(dims, dtype=np.int64)
    for _ in range(l):
        d = (d - 1) // 3 + 1
    return d


def test_fullsize_regional_apply(full):
    from oracle.rng import uniform_pm1
    p = full.p
    x = uniform_pm1(21, np.arange(p.n_nodes))
    xr = torch.from_numpy(x[p.region_gids]).cuda()
    y = torch.empty_like(xr)
    full.lay.regional_apply(xr, y)
    expect = (p.A @ x)[p.region_gids]
    err = np.abs(y.cpu().numpy() - expect).max() / np.abs(expect).max()
    assert err <= OP_TOL, err


def test_fullsize_split_and_galerkin_chain_of_sampled_regions(full):
    """Every level's regional operator of sampled regions against the oracle's chain for that
    region: split block (Sec. 4), then P^(k)T [[A]]^(k) P^(k) per level, masked coarse rows
    carrying 1/mult on the diagonal."""
    from types import SimpleNamespace
    from oracle import hierarchy
    from oracle.split import split_region_block
    p, h = full.p, full.h
    coefs = []
    for l in range(LEVELS):
        n_l, _, kind = h.level_sizes(l)
        c = torch.empty(kind * n_l, dtype=torch.float64, device="cuda")
        h.level_export(l, coeffs=c)
        coefs.append((c.view(kind, n_l), kind))
    for k in _sample_regions(p):
        dims0 = np.asarray(p.region_dims[k], dtype=np.int64)
        gk = p.region_gids[full.offsets[k]:full.offsets[k + 1]]
        Bk = split_region_block(p.A, p.region_gids, full.offsets, k)
        sub = SimpleNamespace(global_dims=tuple(int(v) for v in dims0), region_dims=[dims0],
                              region_gids=np.arange(gk.shape[0]),
                              dirichlet=p.dirichlet[gk], A=Bk)
        levels = hierarchy.build(sub, LEVELS)
        g3 = gk.reshape(int(dims0[2]), int(dims0[1]), int(dims0[0]))
        for l in range(LEVELS):
            dl = _level_dims(p.region_dims, l)
            off = np.zeros(len(dl) + 1, dtype=np.int64)
            off[1:] = np.cumsum(np.prod(dl, axis=1))
            c, kind = coefs[l]
            local = c[:, int(off[k]):int(off[k + 1])].cpu().numpy()
            G = stencils_to_matrix([dl[k]], local.reshape(-1), kind)
            E = levels[l].Ar.tocsr()
            if l > 0:
                # the single-region chain puts 1 on masked coarse diagonals; the regional
                # hierarchy puts 1/mult there (mult of the co-located fine node)
                s = 3 ** l
                m = full.mult[g3[::s, ::s, ::s].reshape(-1)]
                mask = levels[l].layout.mask.astype(float)
                E = (E + sp.diags(mask * (1.0 / m - 1.0))).tocsr()
            D = (G - E).tocsr()
            err = (abs(D).max() if D.nnz else 0.0) / abs(E).max()
            assert err <= OP_TOL, (k, l, err)


def test_fullsize_dinv_level0(full):
    """D~ = Psi^T Psi diag([[A]]) is the composite diagonal: the split rows sum back to A."""
    p, h = full.p, full.h
    n_r = full.lay.sizes()["n_regional"]
    d = torch.empty(n_r, dtype=torch.float64, device="cuda")
    h.level_export(0, dinv=d)
    expect = 1.0 / p.A.diagonal()[p.region_gids]
    err = np.abs(d.cpu().numpy() - expect).max() / np.abs(expect).max()
    assert err <= OP_TOL, err


def test_fullsize_power_method_level0(full):
    from oracle.rng import uniform_pm1
    from oracle.smoothers import power_method
    p, h = full.p, full.h
    free = ~p.dirichlet.astype(bool)
    x0 = uniform_pm1(10, np.arange(p.n_nodes))          # stream seed_base + level 0
    x0[~free] = 0.0
    dinv = 1.0 / p.A.diagonal()
    lam = power_method(lambda v: p.A @ v, dinv, np.dot, x0, iters=10)
    assert h.lam(0) == pytest.approx(lam, rel=OP_TOL)


def test_fullsize_vcycle_symmetric_positive(full):
    from oracle.rng import uniform_pm1
    p, h = full.p, full.h
    free = ~p.dirichlet.astype(bool)
    xs = []
    for s in (31, 32):
        v = uniform_pm1(s, np.arange(p.n_nodes))
        v[~free] = 0.0
        xs.append(v)
    z = []
    for v in xs:
        out = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
        h.vcycle(torch.from_numpy(v).cuda(), out)
        z.append(out.cpu().numpy())
    a, b = xs[1] @ z[0], xs[0] @ z[1]
    assert abs(a - b) <= 1e-9 * np.sqrt((xs[0] @ z[0]) * (xs[1] @ z[1]))
    assert xs[0] @ z[0] > 0 and xs[1] @ z[1] > 0
    assert np.all(z[0][~free] == 0.0)


def test_fullsize_pcg_reaches_tolerance_in_each_precision(full):
    """FP64, FP32 and BF16-coefficient cycles inside FP64 CG: the residual the oracle recomputes
    from the composite CSR is at the 1e-10 target; the mixed solutions' distance from the FP64
    one is reported."""
    from paper_2103_11962_gb300 import rmg
    p = full.p
    bn = np.linalg.norm(p.b)
    sols = {}
    for name, prec in (("fp64", rmg.FP64), ("fp32", rmg.FP32), ("bf16", rmg.FP32_BF16COEF)):
        h = full.h if prec == rmg.FP64 else rmg.Hierarchy(full.lay, _options(rmg, prec))
        x = torch.zeros(p.n_nodes, dtype=torch.float64, device="cuda")
        res = h.pcg(full.dp.b, x, rtol=1e-10, maxit=300)
        xs = x.cpu().numpy()
        rel = np.linalg.norm(p.b - p.A @ xs) / bn
        sols[name] = xs
        print(f"{full.name} {name}: {res['iterations']} its, recurrence {res['relres']:.3e}, "
              f"oracle residual {rel:.3e}")
        assert res["converged"]
        # the FP64 residual of a 1e-10 solution carries rounding noise of the same order
        # (eps ||A|| ||x|| / ||b||), so its two evaluations agree to a few per cent only
        assert rel <= 2e-10
        assert res["true_relres"] == pytest.approx(rel, rel=0.05)
        if h is not full.h:
            h.close()
    for name in ("fp32", "bf16"):
        d = np.linalg.norm(sols[name] - sols["fp64"]) / np.linalg.norm(sols["fp64"])
        print(f"{full.name} {name}: ||x - x_fp64|| / ||x_fp64|| = {d:.3e}")
