"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published test vectors,
closed forms, the lemmas and the theorem of Sec. 3.1, brute-force dense formulas, or an
independently coded algorithm. A plausible mistake in the oracle (a dropped term, a wrong
sign or index, a transposed operand) fails at least one of them.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import cycle, hierarchy, krylov, smoothers
from oracle.regions import make_layout
from oracle.rng import splitmix64, uniform_pm1
from oracle.split import (split_blocks, split_composite_pieces, split_region_block,
                          split_regional)
from oracle.transfer import composite_p, linear_p_1d

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.fixture(scope="module")
def p2d():
    return W.poisson2d_5pt(region_grid=(2, 3), n=28, seed=4)


@pytest.fixture(scope="module")
def p3d():
    return W.diffusion3d_7pt(region_grid=(2, 2, 2), choices=(10, 19), seed=5)


@pytest.fixture(scope="module")
def q3d():
    return W.q1_laplace3d(region_grid=(2, 2, 2), n=10, seed=6)


# ---------------------------------------------------------------------------- RNG
def test_splitmix64_published_vectors():
    for seed, idx, hexv in _golden("splitmix64.txt"):
        assert int(splitmix64(int(seed), [int(idx)])[0]) == int(hexv, 16)


def test_uniform_range_and_mean():
    v = uniform_pm1(3, np.arange(200000))
    assert v.min() >= -1.0 and v.max() < 1.0
    assert abs(v.mean()) < 0.01 and abs(v.var() - 1.0 / 3.0) < 0.01


# ---------------------------------------------------------------------------- workloads
def test_q1_element_closed_form():
    K = W.q1_element_laplacian(1.0)
    table = {int(d): float(v) for d, v in _golden("q1_element.txt")}
    for a in range(8):
        for c in range(8):
            ndiff = bin(a ^ c).count("1")
            assert K[a, c] == pytest.approx(table[ndiff], abs=1e-15)


def test_composite_operators_are_spd_like(p3d, q3d):
    for p in (p3d, q3d):
        A = p.A
        assert abs(A - A.T).max() < 1e-15
        free = ~p.dirichlet.astype(bool)
        assert np.all(A.diagonal()[free] > 0)
        # masked rows are identity rows without coupling
        Am = A[np.flatnonzero(~free)]
        assert np.allclose(Am.toarray()[:, free], 0.0)


# ---------------------------------------------------------------------------- layout / Psi
def test_psi_properties(p3d):
    lay = make_layout(p3d.region_dims, p3d.region_gids, p3d.n_nodes, p3d.dirichlet)
    # multiplicities are 1, 2, 4, 8 and count the copies of every composite node
    counts = np.bincount(p3d.region_gids, minlength=p3d.n_nodes)
    assert np.array_equal(lay.mult, counts)
    assert set(np.unique(lay.mult)) <= {1.0, 2.0, 4.0, 8.0}
    v = np.random.default_rng(0).standard_normal(p3d.n_nodes)
    vr = lay.to_regional(v)
    assert np.allclose(lay.average_to_composite(vr), v)
    assert np.allclose(lay.sum_to_composite(vr), v * counts)
    assert np.allclose(lay.interface_sum(vr), vr * lay.regional_mult())


# ---------------------------------------------------------------------------- splitting (Sec. 4)
@pytest.mark.parametrize("name", ["p2d", "p3d", "q3d"])
def test_lemma1_split_sums_to_composite(name, request):
    p = request.getfixturevalue(name)
    lay = make_layout(p.region_dims, p.region_gids, p.n_nodes, p.dirichlet)
    pieces = split_composite_pieces(lay, p.A)
    S = pieces[0]
    for Ak in pieces[1:]:
        S = S + Ak
    assert abs(S - p.A).max() <= 1e-15 * abs(p.A).max() * 4
    # Lemma 1 in the paper's notation: Psi [[A]] Psi^T = A
    Ar = split_regional(lay, p.A)
    assert abs(lay.Psi @ Ar @ lay.Psi.T - p.A).max() <= 1e-15 * abs(p.A).max() * 4


@pytest.mark.parametrize("name", ["p2d", "p3d", "q3d"])
def test_split_of_a_symmetric_matrix_is_symmetric(name, request):
    """Sec. 4 divides A_ij and A_ji by the same count q_ij = q_ji (the regions holding both
    nodes), so a symmetric A gives region matrices that are symmetric bit for bit. This is
    what lets the FP32 cycle store half of a region stencil. A single moved entry breaks
    exactly the mirrored pairs that hold it."""
    p = request.getfixturevalue(name)
    A = p.A.tocsr()
    assert (A - A.T).count_nonzero() == 0
    lay = make_layout(p.region_dims, p.region_gids, p.n_nodes, p.dirichlet)
    Ar = split_regional(lay, A).tocsr()
    assert (Ar - Ar.T).count_nonzero() == 0
    # the same after rounding to FP32, where the half form compares the pairs
    A32 = Ar.astype(np.float32)
    assert (A32 - A32.T).count_nonzero() == 0
    # move one off-diagonal entry between two free nodes: every copy of that edge in the
    # regional matrix loses its mirror
    free = ~p.dirichlet.astype(bool)
    rows, cols = A.nonzero()
    k = next(t for t in range(len(rows))
             if rows[t] < cols[t] and free[rows[t]] and free[cols[t]])
    i, j = int(rows[k]), int(cols[k])
    B = A.copy()
    B[i, j] = B[i, j] * (1.0 + 2.0 ** -10)
    Br = split_regional(lay, B).tocsr()
    D = (Br - Br.T).tocsr()
    D.eliminate_zeros()
    # q_ij copies of the edge, each a pair (a, b) and (b, a) in the difference
    q = sum(1 for r in range(lay.m)
            if {i, j} <= set(int(g) for g in lay.region_gids[lay.offsets[r]:lay.offsets[r + 1]]))
    assert q >= 1 and D.nnz == 2 * q


def test_split_entries_follow_rule(p3d):
    """Off-diagonals are A_ij / q_ij; interior region rows (away from masks) sum to zero."""
    lay = make_layout(p3d.region_dims, p3d.region_gids, p3d.n_nodes, p3d.dirichlet)
    blocks = split_blocks(lay, p3d.A)
    A = p3d.A.tocsr()
    mask = p3d.dirichlet.astype(bool)
    # region membership sets for brute-force q_ij
    members = {}
    for k in range(lay.m):
        for g in lay.region_gids[lay.offsets[k]:lay.offsets[k + 1]]:
            members.setdefault(int(g), set()).add(k)
    rng = np.random.default_rng(1)
    for k in rng.choice(lay.m, 3, replace=False):
        gk = lay.region_gids[lay.offsets[k]:lay.offsets[k + 1]]
        B = blocks[k].tocsr()
        for li in rng.choice(len(gk), 60, replace=False):
            gi = int(gk[li])
            row = B.getrow(li)
            for lj, v in zip(row.indices, row.data):
                gj = int(gk[lj])
                if gj != gi:
                    q = len(members[gi] & members[gj])
                    assert v == pytest.approx(A[gi, gj] / q, rel=1e-15)
            nb = A.getrow(gi).indices
            if not mask[gi] and not mask[nb].any() and not mask[gi]:
                # interior row w.r.t. Dirichlet: composite row sum is 0, so region row sum is 0
                if abs(A.getrow(gi).sum()) < 1e-14:
                    assert abs(row.sum()) < 1e-14


@pytest.mark.parametrize("name", ["p2d", "p3d", "q3d"])
def test_single_copy_rows_split_to_the_matrix_row(name, request):
    """A node held by one region only has every coupling inside that region with q_ij = 1, so
    the nullspace rule returns its matrix row unchanged: diagonal A_ii (to rounding of the two
    sums the oracle forms), off-diagonals A_ij exactly."""
    p = request.getfixturevalue(name)
    lay = make_layout(p.region_dims, p.region_gids, p.n_nodes, p.dirichlet)
    blocks = split_blocks(lay, p.A)
    A = p.A.tocsr()
    mult = np.bincount(p.region_gids, minlength=p.n_nodes)
    for k in range(lay.m):
        gk = np.asarray(p.region_gids[lay.offsets[k]:lay.offsets[k + 1]])
        B = blocks[k].tocsr()
        for li in np.flatnonzero(mult[gk] == 1)[::7]:
            gi = int(gk[li])
            row = B.getrow(li)
            scale = abs(A.getrow(gi).data).max()
            for lj, v in zip(row.indices, row.data):
                if lj == li:
                    assert abs(v - A[gi, gi]) <= 1e-14 * scale
                else:
                    assert v == A[gi, int(gk[lj])]
            # and nothing of the row is lost: same number of couplings
            assert row.nnz == A.getrow(gi).nnz


@pytest.mark.parametrize("name", ["p2d", "p3d", "q3d"])
def test_single_region_split_equals_whole_problem_split(name, request):
    """The per-region split (used where the whole-problem form is too large) gives exactly the
    blocks of the whole-problem split, which Lemma 1 pins."""
    p = request.getfixturevalue(name)
    lay = make_layout(p.region_dims, p.region_gids, p.n_nodes, p.dirichlet)
    blocks = split_blocks(lay, p.A)
    for k in range(lay.m):
        Bk = split_region_block(p.A, p.region_gids, lay.offsets, k)
        assert Bk.shape == blocks[k].shape
        assert abs(Bk - blocks[k]).max() <= 1e-15 * abs(blocks[k]).max()


def test_constant_coefficient_q1_split_equals_element_split():
    """For constant-coefficient Q1, the /q splitting gives exactly the matrix a region would
    assemble from its own elements (the paper's motivation for the splitting rule)."""
    p = W.q1_laplace3d(region_grid=(2, 2, 1), n=10, seed=0)
    lay = make_layout(p.region_dims, p.region_gids, p.n_nodes, p.dirichlet)
    blocks = split_blocks(lay, p.A)
    Nx, Ny, Nz = p.global_dims
    Ke = W.q1_element_laplacian(1.0 / (Nx - 1))
    mask = p.dirichlet.astype(bool)
    for k in range(lay.m):
        nx, ny, nz = (int(v) for v in p.region_dims[k])
        gk = lay.region_gids[lay.offsets[k]:lay.offsets[k + 1]]
        E = np.zeros((len(gk), len(gk)))
        for ez in range(nz - 1):
            for ey in range(ny - 1):
                for ex in range(nx - 1):
                    loc = [(ex + (a & 1)) + nx * ((ey + ((a >> 1) & 1)) + ny * (ez + (a >> 2)))
                           for a in range(8)]
                    for a in range(8):
                        for c in range(8):
                            E[loc[a], loc[c]] += Ke[a, c]
        # compare on rows/cols that are unmasked (masked rows are identity by convention)
        free = ~mask[gk]
        B = blocks[k].toarray()
        assert np.allclose(B[np.ix_(free, free)], E[np.ix_(free, free)], atol=1e-15)


# ---------------------------------------------------------------------------- regional matvec
@pytest.mark.parametrize("name", ["p2d", "p3d", "q3d"])
def test_regional_residual_equals_composite(name, request):
    """Psi^T Psi [[A]] Psi^T x = Psi^T (A x)  (eq. "regional residual")."""
    p = request.getfixturevalue(name)
    lay = make_layout(p.region_dims, p.region_gids, p.n_nodes, p.dirichlet)
    Ar = split_regional(lay, p.A)
    x = np.random.default_rng(2).standard_normal(p.n_nodes)
    lhs = lay.interface_sum(Ar @ lay.to_regional(x))
    rhs = lay.to_regional(p.A @ x)
    assert np.abs(lhs - rhs).max() <= 1e-14 * np.abs(rhs).max()


# ---------------------------------------------------------------------------- transfers
def _hat_p_1d(n):
    """Independent construction: evaluate coarse piecewise-linear hats at fine coordinates."""
    if n == 1:
        return np.ones((1, 1))
    nc = (n - 1) // 3 + 1
    xf = np.arange(n) / (n - 1)
    xc = np.arange(nc) / (nc - 1)
    H = xc[1] - xc[0]
    return np.maximum(0.0, 1.0 - np.abs(xf[:, None] - xc[None, :]) / H)


def test_linear_p_equals_hat_functions():
    for n in (4, 10, 28, 82):
        assert np.allclose(linear_p_1d(n).toarray(), _hat_p_1d(n), rtol=0, atol=1e-13)


def test_p_reproduces_linear_functions():
    dims = (19, 10, 7)
    P = composite_p(dims, np.zeros(np.prod(dims), bool), np.zeros(7 * 4 * 3, bool))
    cz, cy, cx = np.meshgrid(np.arange(3) * 3.0, np.arange(4) * 3.0, np.arange(7) * 3.0,
                             indexing="ij")
    fz, fy, fx = np.meshgrid(np.arange(7.0), np.arange(10.0), np.arange(19.0), indexing="ij")
    coarse = (2 * cx - cy + 0.5 * cz + 1).reshape(-1)
    fine = (2 * fx - fy + 0.5 * fz + 1).reshape(-1)
    assert np.allclose(P @ coarse, fine)


@pytest.mark.parametrize("name", ["p2d", "p3d"])
def test_lemma2_and_rap_theorem(name, request):
    p = request.getfixturevalue(name)
    levels = hierarchy.build(p, 2)
    f, c = levels
    Psi, Psib = f.layout.Psi, c.layout.Psi
    # Lemma 2: [[P]] Psibar^T = Psi^T P
    assert abs(f.Pr @ Psib.T - Psi.T @ f.P).max() < 1e-15
    # Lemma 3: Psibar [[R]] = R Psi
    assert abs(Psib @ f.Pr.T - f.P.T @ Psi).max() < 1e-15
    # Theorem 1: Psibar [[R]] [[A]] [[P]] Psibar^T = R A P (before the masked-row reset)
    lhs = Psib @ (f.Pr.T @ f.Ar @ f.Pr) @ Psib.T
    rhs = f.P.T @ f.A @ f.P
    assert abs(lhs - rhs).max() <= 1e-13 * abs(rhs).max()
    # and with the masked identity reset on both sides
    assert abs(hierarchy.coarse_composite_from_regional(c) - c.A).max() <= 1e-13 * abs(c.A).max()


def test_rap_closed_form_1d():
    n = 28
    h = 1.0 / (n - 1)
    A = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) / h
    P = linear_p_1d(n)
    Ac = (P.T @ A @ P).toarray()
    factor = {r[0]: float(r[1]) for r in _golden("coarse_stencils.txt")}["1d_p1_laplacian"]
    for i in range(1, Ac.shape[0] - 1):
        assert Ac[i, i - 1:i + 2] == pytest.approx(factor * np.array([-1, 2, -1]) / h, rel=1e-13)


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_rap_closed_form_q1(case):
    """Galerkin coarse Q1 stencil equals the re-assembled Q1 stencil on the 3h mesh."""
    factor = {r[0]: float(r[1]) for r in _golden("coarse_stencils.txt")}[f"{case}_q1_laplacian"]
    if case == "2d":
        p = W.q1_laplace2d(region_grid=(2, 2), n=28)
        S = 9
    else:
        p = W.q1_laplace3d(region_grid=(2, 2, 2), n=19)
        S = 27
    levels = hierarchy.build(p, 2)
    f, c = levels
    Nx, Ny, Nz = f.dims
    cNx, cNy, cNz = c.dims
    # a fine and a coarse interior node far from the boundary, both at the grid centre
    def stencil(A, dims, x, y, z):
        nx, ny, _ = dims
        g = x + nx * (y + ny * z)
        row = A.getrow(g)
        out = {}
        for j, v in zip(row.indices, row.data):
            out[(j % nx - x, (j // nx) % ny - y, j // (nx * ny) - z)] = v
        return out
    if case == "2d":
        fs = stencil(f.A, f.dims, Nx // 2, Ny // 2, 0)
        cs = stencil(c.A, c.dims, cNx // 2, cNy // 2, 0)
    else:
        fs = stencil(f.A, f.dims, Nx // 2, Ny // 2, Nz // 2)
        cs = stencil(c.A, c.dims, cNx // 2, cNy // 2, cNz // 2)
    assert len(fs) in (S, 21 if S == 27 else S)
    for key, v in fs.items():
        assert cs.get(key, 0.0) == pytest.approx(factor * v, rel=1e-12, abs=1e-14)


def test_splitting_independence_of_vcycle(p3d):
    """Another valid split (off-diagonals of shared edges given to one region only) changes
    the region matrices but not the V-cycle: with geometric transfers and Jacobi the cycle
    only sees composite quantities (Sec. 4: no numerical impact)."""
    opts = cycle.Options(smoother="jacobi", nu1=2, nu2=2, omega=0.67)
    lev_a = hierarchy.build(p3d, 3)
    lev_b = hierarchy.build(p3d, 3)
    lay = lev_b[0].layout
    # alternative split: element-free "owner takes all" for every shared off-diagonal
    A = p3d.A.tocsr()
    blocks = []
    owner = {}
    for k in range(lay.m):
        gk = lay.region_gids[lay.offsets[k]:lay.offsets[k + 1]]
        B = (lay.Psi_k[k].T @ A @ lay.Psi_k[k]).tocoo()
        keep = []
        for i, j, v in zip(B.row, B.col, B.data):
            if i == j:
                continue
            key = (int(gk[i]), int(gk[j]))
            if owner.setdefault(key, k) == k:
                keep.append((i, j, v))
        n_k = len(gk)
        off = sp.csr_matrix(([v for _, _, v in keep], ([i for i, _, _ in keep],
                                                       [j for _, j, _ in keep])),
                            shape=(n_k, n_k))
        z = lay.Psi_k[k].T @ (A @ np.ones(A.shape[0]))
        mk = lay.Psi_k[k].T @ lay.mult
        diag = z / mk - np.asarray(off.sum(axis=1)).ravel()
        blocks.append((off + sp.diags(diag)).tocsr())
    Ar_alt = sp.block_diag(blocks, format="csr")
    assert abs(lay.Psi @ Ar_alt @ lay.Psi.T - A).max() < 1e-13
    # rebuild hierarchy b's regional part from the alternative split
    lev_b[0].Ar = Ar_alt
    for l in range(len(lev_b) - 1):
        f, c = lev_b[l], lev_b[l + 1]
        Arc = (f.Pr.T @ f.Ar @ f.Pr).tocsr()
        rm = c.layout.regional_mask()
        c.Ar = (Arc + sp.diags(np.where(rm, 1.0 / c.layout.regional_mult(), 0.0))).tocsr()
    for lev in lev_b:
        lev.Dinv_r = 1.0 / lev.layout.interface_sum(lev.Ar.diagonal())
    ma, mb = cycle.RegionalMG(lev_a, opts), cycle.RegionalMG(lev_b, opts)
    b = lay.to_regional(p3d.b)
    ua = ma.cycle(np.zeros_like(b), b)
    ub = mb.cycle(np.zeros_like(b), b)
    assert np.abs(ua - ub).max() <= 1e-12 * np.abs(ua).max()
    assert abs(lev_a[0].Ar - Ar_alt).max() > 1e-3   # the splits really differ


# ---------------------------------------------------------------------------- smoothers
def _laplace2d_eig(N, i, j):
    x = np.arange(N) / (N - 1)
    v = np.outer(np.sin(j * np.pi * x), np.sin(i * np.pi * x)).reshape(-1)   # (y, x)
    mu = 1.0 - 0.5 * (np.cos(i * np.pi / (N - 1)) + np.cos(j * np.pi / (N - 1)))
    return v, mu


def test_regional_jacobi_closed_form(p2d):
    """On the 5-point Laplacian with Dirichlet boundary, sin(i pi x) sin(j pi y) is an
    eigenvector of D^-1 A with eigenvalue mu = 1 - (cos(i pi h) + cos(j pi h))/2, so nu damped
    Jacobi sweeps multiply it by (1 - omega mu)^nu. The regional smoother must agree because
    D~ is the composite diagonal."""
    p = W.poisson2d_5pt(region_grid=(2, 2), n=28, seed=0)
    lev = hierarchy.build(p, 1)[0]
    lay = lev.layout
    N = p.global_dims[0]
    for (i, j) in [(1, 1), (3, 7), (20, 30), (N - 2, N - 2)]:
        v, mu = _laplace2d_eig(N, i, j)
        res = lambda u, b: b - lay.interface_sum(lev.Ar @ u)
        ur = smoothers.jacobi(lay.to_regional(v), np.zeros(lay.n_r), res, lev.Dinv_r, 0.67, 3)
        expect = lay.to_regional(v) * (1 - 0.67 * mu) ** 3
        assert np.abs(ur - expect).max() < 1e-13


def _cheb_T(K, x):
    return np.cosh(K * np.arccosh(x)) if abs(x) >= 1 else np.cos(K * np.arccos(x))


@pytest.mark.parametrize("degree", [1, 2, 3, 4])
def test_regional_chebyshev_closed_form(degree):
    """With fixed [alpha, beta], an eigenvector of D^-1 A with eigenvalue mu is multiplied by
    T_K((theta - mu)/d) / T_K(theta/d), theta = (alpha+beta)/2, d = (beta-alpha)/2
    (Chebyshev acceleration; Saad, Iterative Methods, Sec. 12.3)."""
    p = W.poisson2d_5pt(region_grid=(2, 2), n=28, seed=0)
    lev = hierarchy.build(p, 1)[0]
    lay = lev.layout
    N = p.global_dims[0]
    alpha, beta = 0.1, 2.05
    theta, d = 0.5 * (alpha + beta), 0.5 * (beta - alpha)
    res = lambda u, b: b - lay.interface_sum(lev.Ar @ u)
    for (i, j) in [(1, 2), (5, 9), (30, 40), (N - 2, N - 3)]:
        v, mu = _laplace2d_eig(N, i, j)
        ur = smoothers.chebyshev(lay.to_regional(v), np.zeros(lay.n_r), res, lev.Dinv_r,
                                 alpha, beta, degree)
        factor = _cheb_T(degree, (theta - mu) / d) / _cheb_T(degree, theta / d)
        assert np.abs(ur - factor * lay.to_regional(v)).max() < 1e-12


def test_power_method_bounds():
    p = W.poisson2d_5pt(region_grid=(2, 2), n=28, seed=0)
    levels = hierarchy.build(p, 2)
    opts = cycle.Options(smoother="chebyshev")
    mg = cycle.RegionalMG(levels, opts)
    N = p.global_dims[0]
    lam_true = 1.0 + np.cos(np.pi / (N - 1))
    lam = levels[0].lam_r
    assert 0.85 * lam_true < lam <= lam_true * (1 + 1e-12)
    cm = cycle.CompositeMG(hierarchy.build(p, 2), opts)
    assert cm.levels[0].lam == pytest.approx(lam, rel=1e-12)


@pytest.mark.parametrize("k", [1, 3, 10])
def test_power_method_equals_its_spectral_closed_form(k):
    """k normalised power steps on M = D^-1 A, then x^T M x / x^T x, written out through the
    eigenpairs of the symmetric S = D^-1/2 A D^-1/2 = Q L Q^T (M = D^-1/2 S D^1/2). With
    c = Q^T D^1/2 x0, M^k x0 = D^-1/2 Q L^k c, so the estimate is
    (L^k c)^T Q^T D^-1 Q (L^(k+1) c) / (L^k c)^T Q^T D^-1 Q (L^k c), with no iteration.
    A dropped D^-1, a step too many or too few, or another quotient fails."""
    p = W.diffusion3d_7pt(region_grid=(1, 1, 1), choices=(10,), seed=3)
    A = p.A.toarray()
    d = np.diag(A).copy()
    x0 = uniform_pm1(10, np.arange(p.n_nodes))
    x0[p.dirichlet.astype(bool)] = 0.0
    lam = smoothers.power_method(lambda v: p.A @ v, 1.0 / d, np.dot, x0, iters=k)
    L, Q = np.linalg.eigh(A / np.sqrt(np.outer(d, d)))
    c = Q.T @ (np.sqrt(d) * x0)
    G = Q.T @ (Q / d[:, None])                  # Q^T D^-1 Q
    a, b = L ** k * c, L ** (k + 1) * c
    assert lam == pytest.approx((a @ G @ b) / (a @ G @ a), rel=1e-12)


# ---------------------------------------------------------------------------- cycles
@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
@pytest.mark.parametrize("name", ["p2d", "p3d"])
def test_regional_vcycle_equals_composite(name, smoother, request):
    """Sec. 6.1 / Table 1: with identical coarsening the region cycle reproduces the composite
    cycle (Jacobi columns identical in every printed digit)."""
    p = request.getfixturevalue(name)
    nlev = 3
    levels = hierarchy.build(p, nlev)
    opts = cycle.Options(smoother=smoother, nu1=2 if smoother == "jacobi" else 1,
                         nu2=2 if smoother == "jacobi" else 1)
    cm, rm = cycle.CompositeMG(levels, opts), cycle.RegionalMG(levels, opts)
    lay = levels[0].layout
    u = np.zeros(p.n)
    ur = np.zeros(lay.n_r)
    for _ in range(3):
        u = cm.cycle(u, p.b)
        ur = rm.cycle(ur, lay.to_regional(p.b))
        assert np.abs(lay.to_regional(u) - ur).max() <= 1e-12 * np.abs(u).max()


def test_two_grid_equals_dense_projection(p2d):
    """Two-grid cycle with exact coarse solve: e <- S2 (I - P Abar^-1 P^T A) S1 e."""
    levels = hierarchy.build(p2d, 2)
    opts = cycle.Options(smoother="jacobi", nu1=1, nu2=2, omega=0.6)
    rm = cycle.RegionalMG(levels, opts)
    f, c = levels
    free = ~f.layout.mask
    cfree = ~c.layout.mask
    A = f.A.toarray()[np.ix_(free, free)]
    P = f.P.toarray()[np.ix_(free, cfree)]
    D = np.diag(A)
    S = np.eye(A.shape[0]) - 0.6 * A / D[:, None]
    Ac = P.T @ A @ P
    CG = np.eye(A.shape[0]) - P @ np.linalg.solve(Ac, P.T @ A)
    E = np.linalg.matrix_power(S, 2) @ CG @ S
    rng = np.random.default_rng(7)
    xs = np.zeros(p2d.n); xs[free] = rng.standard_normal(free.sum())
    u0 = np.zeros(p2d.n); u0[free] = rng.standard_normal(free.sum())
    b = f.A @ xs
    lay = f.layout
    u1 = lay.average_to_composite(rm.cycle(lay.to_regional(u0), lay.to_regional(b)))
    e1 = (xs - u1)[free]
    e_expect = E @ (xs - u0)[free]
    assert np.abs(e1 - e_expect).max() <= 1e-11 * np.abs(e_expect).max()


def _gepp_solve(M, rhs):
    """Gaussian elimination with partial pivoting, written out (independent of Cholesky)."""
    M = M.astype(float).copy()
    x = rhs.astype(float).copy()
    n = M.shape[0]
    for k in range(n):
        piv = k + int(np.argmax(np.abs(M[k:, k])))
        if piv != k:
            M[[k, piv]] = M[[piv, k]]
            x[[k, piv]] = x[[piv, k]]
        f = M[k + 1:, k] / M[k, k]
        M[k + 1:, k:] -= np.outer(f, M[k, k:])
        x[k + 1:] -= f * x[k]
    for k in range(n - 1, -1, -1):
        x[k] = (x[k] - M[k, k + 1:] @ x[k + 1:]) / M[k, k]
    return x


def test_coarse_cholesky_vs_gepp():
    p = W.diffusion3d_7pt(region_grid=(2, 2, 2), choices=(19,), seed=8)
    levels = hierarchy.build(p, 2)
    rm = cycle.RegionalMG(levels, cycle.Options())
    last = levels[-1]
    rhs = np.random.default_rng(3).standard_normal(last.layout.n)
    rhs[last.layout.mask] = 0
    x = rm.coarse.solve(rhs)
    free = ~last.layout.mask
    xg = _gepp_solve(rm.Abar.toarray()[np.ix_(free, free)], rhs[free])
    assert np.abs(x[free] - xg).max() <= 1e-12 * np.abs(xg).max()
    assert np.all(x[~free] == 0)


@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
def test_pcg_matches_direct(p3d, smoother):
    levels = hierarchy.build(p3d, 3)
    opts = cycle.Options(smoother=smoother, nu1=2 if smoother == "jacobi" else 1,
                         nu2=2 if smoother == "jacobi" else 1)
    rm = cycle.RegionalMG(levels, opts)
    x, it, hist = krylov.pcg(p3d.A, p3d.b, krylov.regional_preconditioner(rm), rtol=1e-13)
    xd = sp.linalg.spsolve(p3d.A.tocsc(), p3d.b)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert 3 <= it <= 40
    # the regional and the composite preconditioner give the same iteration count
    cm = cycle.CompositeMG(levels, opts)
    _, it2, _ = krylov.pcg(p3d.A, p3d.b, cm.precondition, rtol=1e-10)
    _, it1, _ = krylov.pcg(p3d.A, p3d.b, krylov.regional_preconditioner(rm), rtol=1e-10)
    assert it1 == it2


def test_jacobi_mg_contraction_band():
    """Sanity band, not a parity target: the 2D Laplace region MG with Jacobi contracts the
    residual by a factor well below 1 per cycle (Table 1 shows about 0.2 with a 7-point
    stencil and nu = 1/1); with the 5-point stencil, omega = 0.67 and nu = 2/2 the factor
    must stay below 0.5."""
    p = W.poisson2d_5pt(region_grid=(2, 2), n=82, seed=0)
    levels = hierarchy.build(p, 4)
    rm = cycle.RegionalMG(levels, cycle.Options(smoother="jacobi", nu1=2, nu2=2, omega=0.67))
    lay = levels[0].layout
    b = lay.to_regional(p.b)
    u = np.zeros_like(b)
    res = [np.linalg.norm(p.b)]
    for _ in range(8):
        u = rm.cycle(u, b)
        res.append(np.linalg.norm(p.b - p.A @ lay.average_to_composite(u)))
    rates = np.array(res[1:]) / np.array(res[:-1])
    assert np.all(rates[2:] < 0.5)


# ---------------------------------------------------------------------------- learned prolongator
def test_stored_p_with_linear_weights_is_linear_p():
    from oracle.transfer import stored_p
    dims = (19, 10, 7)
    n = int(np.prod(dims))
    g = np.arange(n)
    coord = [g % 19, (g // 19) % 10, g // 190]
    wr = np.stack([(c % 3) / 3.0 for c in coord])
    fm = np.zeros(n, bool); fm[::7] = True
    cm = np.zeros(7 * 4 * 3, bool); cm[::5] = True
    A = stored_p(dims, wr, fm, cm)
    B = composite_p(dims, fm, cm)
    # same sparsity; entries equal up to the FP32 rounding of the stored weights
    assert (A != 0).sum() == (B != 0).sum()
    assert abs(A - B).max() <= 2e-7


def test_opdep_weights_constant_coefficient_is_linear():
    from oracle.learned import opdep_weights
    p = W.q1_laplace3d(region_grid=(1, 1, 1), n=10)     # not an M-matrix: linear fallback
    p7 = W.diffusion3d_7pt(region_grid=(2, 1, 1), choices=(10,), seed=0, sigma=0.0)
    for prob in (p, p7):
        wr = opdep_weights(prob.A, prob.global_dims)
        Nx, Ny, Nz = prob.global_dims
        g = np.arange(prob.n_nodes)
        coord = [g % Nx, (g // Nx) % Ny, g // (Nx * Ny)]
        free = ~prob.dirichlet.astype(bool)
        # away from the Dirichlet boundary every conductance on a line is equal
        inner = free.copy()
        for c, N in zip(coord, (Nx, Ny, Nz)):
            inner &= (c >= 3) & (c <= N - 4)
        for a in range(3):
            r = coord[a] % 3
            sel = inner & (r != 0)
            assert np.allclose(wr[a][sel], r[sel] / 3.0, atol=1e-14)


def test_opdep_weights_make_flux_continuous():
    """With the series-resistance weights the interpolated values on a line between two
    coarse nodes carry the same flux k_e (v_e+1 - v_e) across all three edges: the discrete
    1D A-harmonic extension."""
    from oracle.learned import opdep_weights
    p = W.highcontrast3d_7pt(region_grid=(3, 2, 2), choices=(10,), seed=13)
    wr = opdep_weights(p.A, p.global_dims)
    Nx, Ny, Nz = p.global_dims
    A = p.A.tocsr()
    rng = np.random.default_rng(2)
    checked = 0
    for _ in range(400):
        x, y, z = rng.integers(1, Nx - 1), rng.integers(1, Ny - 1), rng.integers(1, Nz - 1)
        rem = x % 3
        if rem == 0 or x - rem + 3 >= Nx:
            continue
        x0 = x - rem
        nodes = [x0 + e + Nx * (y + Ny * z) for e in range(4)]
        k = np.array([-A[nodes[e], nodes[e + 1]] for e in range(3)])
        if np.any(k <= 0):
            continue
        v0, v3 = 0.3, 1.7
        w1, w2 = wr[0][nodes[1]], wr[0][nodes[2]]
        v = [v0, v0 + w1 * (v3 - v0), v0 + w2 * (v3 - v0), v3]
        flux = [k[e] * (v[e + 1] - v[e]) for e in range(3)]
        assert np.allclose(flux, flux[0], rtol=1e-12)
        checked += 1
    assert checked > 50


def test_mlp_oracle_gradient_matches_finite_differences():
    from oracle import learned as Lm
    rng = np.random.default_rng(0)
    params = rng.standard_normal(Lm.NPARAMS) * 0.3
    X = rng.standard_normal((40, Lm.NFEAT))
    Y = rng.uniform(0, 1, (40, 3))
    M = (rng.uniform(0, 1, (40, 3)) > 0.3).astype(float)
    L0, g = Lm.loss_and_grad(params, X, Y, M, rounding=False)
    idx = rng.choice(Lm.NPARAMS, 60, replace=False)
    for i in idx:
        e = np.zeros(Lm.NPARAMS); e[i] = 1e-6
        lp, _ = Lm.loss_and_grad(params + e, X, Y, M, rounding=False)
        lm, _ = Lm.loss_and_grad(params - e, X, Y, M, rounding=False)
        fd = (lp - lm) / 2e-6
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9)


def test_bf16_rounding_matches_definition():
    from oracle.learned import bf16_round
    # bfloat16 keeps 8 significand bits; ties go to even
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5, 3.0e-39])
    out = bf16_round(vals)
    assert out[0] == 1.0
    assert out[1] == 1.0                     # tie between 1 and 1 + 2^-7: even (1.0)
    assert out[2] == 1.0 + 2 ** -6          # tie between 1+2^-7 and 1+2^-6: even mantissa
    assert out[3] == 1.0
    assert out[4] == -2.5


# ---------------------------------------------------------------------------- elasticity (3 dofs)
def test_elasticity_element_rigid_body_modes():
    """The Q1 elasticity element annihilates the six rigid-body motions and is symmetric."""
    K = W.q1_element_elasticity(0.1, 2.0, 0.3)
    assert abs(K - K.T).max() < 1e-15
    corners = np.array([[(a >> 0) & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float) * 0.1
    modes = []
    for c in range(3):
        t = np.zeros(24); t[c::3] = 1.0; modes.append(t)
    for (i, j) in [(0, 1), (1, 2), (0, 2)]:
        r = np.zeros(24); r[i::3] = -corners[:, j]; r[j::3] = corners[:, i]; modes.append(r)
    for m in modes:
        assert abs(K @ m).max() < 1e-14
    w = np.linalg.eigvalsh(K)
    assert np.sum(w < 1e-12 * w.max()) == 6          # exactly the rigid-body modes


@pytest.fixture(scope="module")
def el3d():
    return W.elasticity3d(region_grid=(2, 2, 1), choices=(10,), seed=4)


def test_elasticity_block_split_and_apply(el3d):
    p = el3d
    levels = hierarchy.build_block(p, 2)
    L0 = levels[0].layout
    assert abs(L0.Psi @ levels[0].Ar @ L0.Psi.T - levels[0].A).max() <= 1e-15 * abs(levels[0].A).max() * 4
    x = np.random.default_rng(1).standard_normal(3 * p.n_nodes)
    lhs = L0.interface_sum(levels[0].Ar @ L0.to_regional(x))
    rhs = L0.to_regional(levels[0].A @ x)
    assert np.abs(lhs - rhs).max() <= 1e-14 * np.abs(rhs).max()
    # the Galerkin theorem with I (x) P
    f, c = levels
    Psib = c.layout.Psi
    lhs = Psib @ (f.Pr.T @ f.Ar @ f.Pr) @ Psib.T
    rhs = f.P.T @ f.A @ f.P
    assert abs(lhs - rhs).max() <= 1e-13 * abs(rhs).max()


def test_elasticity_regional_cycle_equals_composite(el3d):
    p = el3d
    levels = hierarchy.build_block(p, 2)
    o = cycle.Options(smoother="chebyshev", nu1=1, nu2=1, degree=3)
    cm, rm = cycle.CompositeMG(levels, o), cycle.RegionalMG(levels, o)
    perm = hierarchy.node_major_to_component_major(p.n_nodes, 3)
    b = p.b[perm]
    L0 = levels[0].layout
    uc = cm.precondition(b)
    ur = L0.average_to_composite(rm.precondition(L0.to_regional(b)))
    assert np.abs(uc - ur).max() <= 1e-12 * np.abs(uc).max()
    x, it, _ = krylov.pcg(levels[0].A, b, krylov.regional_preconditioner(rm), rtol=1e-12)
    xd = sp.linalg.spsolve(levels[0].A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def test_piecewise_constant_galerkin_closed_form():
    """3:1 piecewise-constant transfers aggregate 3x3 fine nodes; the Galerkin product of the
    5-point Laplacian is then 3 times the 5-point Laplacian on the coarse grid (three fine
    edges cross every side of an aggregate; Table 4 'Const')."""
    from oracle.transfer import stored_p
    p = W.poisson2d_5pt(region_grid=(2, 2), n=28, seed=0)
    Nx, Ny, _ = p.global_dims
    g = np.arange(p.n_nodes)
    coord = [g % Nx, g // Nx, np.zeros_like(g)]
    wr = np.stack([(c % 3 == 2).astype(np.float32) for c in coord])
    levels = hierarchy.build(p, 2, weights=lambda l, lev: wr)
    P = levels[0].P
    free = ~p.dirichlet.astype(bool)
    rows = P[np.flatnonzero(free)]
    assert np.all(np.diff(rows.indptr) <= 1)             # at most one coarse node per fine node
    assert np.all(rows.data == 1.0)
    c = levels[1]
    cNx, cNy, _ = c.dims
    x, y = cNx // 2, cNy // 2
    row = c.A.getrow(x + cNx * y)
    st = {(j % cNx - x, j // cNx - y): v for j, v in zip(row.indices, row.data) if v != 0}
    assert st == pytest.approx({(0, 0): 12.0, (1, 0): -3.0, (-1, 0): -3.0, (0, 1): -3.0,
                                (0, -1): -3.0})


# ------------------------------------------------------------- region Gauss-Seidel (Algorithm 1)
@pytest.mark.parametrize("make", [
    lambda: W.poisson2d_5pt(region_grid=(1, 1), n=19, seed=3),
    lambda: W.diffusion3d_7pt(region_grid=(1, 1, 1), choices=(10,), seed=3),
    lambda: W.q1_laplace3d(region_grid=(1, 1, 1), n=10, seed=3),
])
@pytest.mark.parametrize("omega", [1.0, 0.8])
def test_gauss_seidel_sweep_is_the_triangular_solve(make, omega):
    """On a single region, one sweep of the multicolour region Gauss-Seidel is the textbook
    SOR step u + (D/omega + L)^-1 (b - A u), with L the strictly lower part of A in the colour
    order (nodes of one colour are uncoupled, so their order inside a colour is free)."""
    import scipy.sparse.linalg as spla
    from oracle import cycle, hierarchy, smoothers
    p = make()
    lev = hierarchy.build(p, 1)[0]
    A = lev.Ar.tocsr()
    colours, ncol = cycle.gs_colours(lev)
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal(A.shape[0])
    b = rng.standard_normal(A.shape[0])
    got = smoothers.gauss_seidel_colored(u0, b, lambda u, bb: bb - A @ u, lambda d: A @ d,
                                         lev.Dinv_r, omega, 1, colours, list(range(ncol)))
    perm = np.argsort(colours, kind="stable")
    Ap = A[perm][:, perm].tocsr()
    M = (sp.tril(Ap, k=-1) + sp.diags(Ap.diagonal() / omega)).tocsr()
    r = (b - A @ u0)[perm]
    delta = spla.spsolve_triangular(M, r, lower=True)
    expect = u0.copy()
    expect[perm] += delta
    assert np.abs(got - expect).max() <= 1e-12 * np.abs(expect).max()
    # the colouring leaves no coupling inside a colour
    C = A.tocoo()
    off = C.row != C.col
    assert not np.any(colours[C.row[off]] == colours[C.col[off]])


def test_flexible_pcg_equals_pcg_for_a_symmetric_preconditioner():
    """With a symmetric fixed preconditioner r.z_old vanishes in exact arithmetic, so the
    flexible (Polak-Ribiere) beta gives the same iterates as the classical one."""
    from oracle import cycle, hierarchy, krylov
    p = W.diffusion3d_7pt(region_grid=(2, 2, 1), choices=(10, 19), seed=8)
    mg = cycle.RegionalMG(hierarchy.build(p, 2), cycle.Options(smoother="jacobi", nu1=2, nu2=2,
                                                               omega=0.67))
    pre = krylov.regional_preconditioner(mg)
    x1, it1, h1 = krylov.pcg(p.A, p.b, pre, rtol=1e-10)
    x2, it2, h2 = krylov.pcg(p.A, p.b, pre, rtol=1e-10, flexible=True)
    assert it1 == it2
    assert np.allclose(h1, h2, rtol=1e-6, atol=0)


# ---------------------------------------------------------------------------- MLP forward pins
# A hand-set network whose value is traced by hand. Layer-1 unit h reads feature (h + 1) mod 32
# (units 32..63 have zero weights and bias -1, so ReLU keeps them at 0), layer-2 unit m reads
# layer-1 unit (m + 7) mod 64, output j reads layer-2 unit 5 j + 2. So output j depends on the
# single feature k(j) through units m = 5 j + 2, h = m + 7: j = 0 -> m 2, h 9, k 10;
# j = 1 -> m 7, h 14, k 15; j = 2 -> m 12, h 19, k 20. All parameters and inputs are exact in
# BF16 and every intermediate below stays exact in BF16, so the rounded and the exact network
# give the same value.
_HS_A = {9: 2.0, 14: 0.5, 19: -1.0}           # layer-1 weights of the used units
_HS_B1 = {9: -0.25, 14: 0.75, 19: 0.5}
_HS_C = {2: 1.5, 7: -2.0, 12: 0.25}           # layer-2 weights of the used units
_HS_B2 = {2: 0.125, 7: 1.0, 12: -0.5}
_HS_E = [-0.75, 3.0, 0.5]                     # output weights
_HS_B3 = [0.5, -1.0, 0.25]


def _handset_params():
    from oracle import learned as Lm
    W1 = np.zeros((64, 32)); b1 = np.full(64, -1.0)
    for h in range(32):
        W1[h, (h + 1) % 32] = _HS_A.get(h, 1.0)
        b1[h] = _HS_B1.get(h, 0.0)
    W2 = np.zeros((64, 64)); b2 = np.zeros(64)
    for m in range(64):
        W2[m, (m + 7) % 64] = _HS_C.get(m, 1.0)
        b2[m] = _HS_B2.get(m, 0.0)
    W3 = np.zeros((3, 64))
    for j in range(3):
        W3[j, 5 * j + 2] = _HS_E[j]
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), np.asarray(_HS_B3)])
    assert p.size == Lm.NPARAMS
    return p


# Inputs: sample 0 keeps every used unit active; sample 1 drives layer-1 unit 9 negative (ReLU
# zero); sample 2 drives layer-2 unit 7 negative.
_HS_X = np.zeros((3, 32))
_HS_X[0, [10, 15, 20]] = [0.375, 2.0, -1.5]
_HS_X[1, [10, 15, 20]] = [-1.0, 0.5, 0.25]
_HS_X[2, [10, 15, 20]] = [1.0, 6.0, 0.0]
# Traced by hand, z3 of every (sample, output):
#  s0 j0: h1 = relu(2*0.375 - 0.25) = 0.5,  h2 = relu(1.5*0.5 + 0.125) = 0.875, z3 = -0.75*0.875 + 0.5
#  s0 j1: h1 = relu(0.5*2 + 0.75) = 1.75,   h2 = relu(-2*1.75 + 1) = 0,         z3 = -1
#  s0 j2: h1 = relu(-1*-1.5 + 0.5) = 2,     h2 = relu(0.25*2 - 0.5) = 0,        z3 = 0.25
#  s1 j0: h1 = relu(-2 - 0.25) = 0,         h2 = relu(0.125) = 0.125,           z3 = -0.75*0.125 + 0.5
#  s1 j1: h1 = relu(0.25 + 0.75) = 1,       h2 = relu(-2 + 1) = 0,              z3 = -1
#  s1 j2: h1 = relu(-0.25 + 0.5) = 0.25,    h2 = relu(0.0625 - 0.5) = 0,        z3 = 0.25
#  s2 j0: h1 = relu(2 - 0.25) = 1.75,       h2 = relu(2.625 + 0.125) = 2.75,    z3 = -0.75*2.75 + 0.5
#  s2 j1: h1 = relu(3 + 0.75) = 3.75,       h2 = relu(-7.5 + 1) = 0,            z3 = -1
#  s2 j2: h1 = relu(0 + 0.5) = 0.5,         h2 = relu(0.125 - 0.5) = 0,         z3 = 0.25
_HS_Z3 = np.array([[-0.15625, -1.0, 0.25],
                   [0.40625, -1.0, 0.25],
                   [-1.5625, -1.0, 0.25]])


def _check_handset(forward):
    p = _handset_params()
    expect = 1.0 / (1.0 + np.exp(-_HS_Z3))
    for rounding in (False, True):
        O, _ = forward(p, _HS_X, rounding=rounding)
        assert O.shape == (3, 3)
        assert np.abs(O - expect).max() <= 1e-15, rounding


def test_mlp_forward_handset_network():
    from oracle import learned as Lm
    _check_handset(Lm.forward)


def _loop_forward(params, x):
    """One sample through the network by explicit sums over the flat parameter layout of the
    C header: W1[64][32] at 0, b1[64] at 2048, W2[64][64] at 2112, b2[64] at 6208, W3[3][64]
    at 6272, b3[3] at 6464 (row = output unit, column = input unit)."""
    import math
    h1 = []
    for h in range(64):
        z = params[2048 + h]
        for k in range(32):
            z += params[h * 32 + k] * x[k]
        h1.append(z if z > 0 else 0.0)
    h2 = []
    for m in range(64):
        z = params[6208 + m]
        for h in range(64):
            z += params[2112 + m * 64 + h] * h1[h]
        h2.append(z if z > 0 else 0.0)
    out = []
    for j in range(3):
        z = params[6464 + j]
        for m in range(64):
            z += params[6272 + j * 64 + m] * h2[m]
        out.append(1.0 / (1.0 + math.exp(-z)))
    return out


def test_mlp_forward_matches_per_sample_loop():
    from oracle import learned as Lm
    rng = np.random.default_rng(3)
    params = rng.standard_normal(Lm.NPARAMS) * 0.4
    X = rng.standard_normal((6, 32))
    O, _ = Lm.forward(params, X, rounding=False)
    for s in range(6):
        assert np.abs(O[s] - np.asarray(_loop_forward(params, X[s]))).max() <= 1e-13


@pytest.mark.parametrize("plant", ["transpose_w2", "swap_biases", "flip_w3", "transpose_w1"])
def test_mlp_pins_catch_planted_mistakes(plant, monkeypatch):
    """Each plausible slip in the oracle network makes the hand-set pin fail."""
    from oracle import learned as Lm
    real = Lm.unpack

    def planted(params):
        W1, b1, W2, b2, W3, b3 = real(params)
        if plant == "transpose_w2":
            W2 = W2.T
        elif plant == "swap_biases":
            b1, b2 = b2, b1
        elif plant == "flip_w3":
            W3 = -W3
        else:
            W1 = W1.T
        return W1, b1, W2, b2, W3, b3

    monkeypatch.setattr(Lm, "unpack", planted)
    with pytest.raises((AssertionError, ValueError)):
        _check_handset(Lm.forward)
    with pytest.raises((AssertionError, ValueError)):
        rng = np.random.default_rng(3)
        params = rng.standard_normal(Lm.NPARAMS) * 0.4
        x = rng.standard_normal((1, 32))
        O, _ = Lm.forward(params, x, rounding=False)
        assert np.abs(O[0] - np.asarray(_loop_forward(params, x[0]))).max() <= 1e-13


def test_mlp_features_constant_laplacian_closed_form():
    """Features of the constant-coefficient 7-point operator (couplings -h, diagonal 6h; masked
    rows identity): a line of unmasked nodes gives log10(h / 6h) for every conductance and 0 for
    every diagonal ratio; a line starting at the masked face x = 0 gives -12 for its first
    conductance (a masked row has no coupling) and log10(1 / 6h) for its first diagonal."""
    from oracle.learned import features
    p = W.diffusion3d_7pt(region_grid=(2, 2, 1), choices=(10,), seed=0, sigma=0.0, rhs=False)
    Nx, Ny, Nz = p.global_dims
    h = 1.0 / (Nx - 1)
    F = features(p.A, p.global_dims)
    assert np.allclose(features(3.5 * p.A, p.global_dims), F, atol=1e-14)    # scale free
    g = lambda x, y, z: x + Nx * (y + Ny * z)
    inner = [np.log10(1 / 6)] * 3 + [0.0] * 4
    # (4, 5, 4): x rem 1, y rem 2, z rem 1, every line inside the unmasked nodes
    f = F[g(4, 5, 4)]
    assert np.allclose(f[0:9], inner + [1 / 3, 1.0], atol=1e-14)
    assert np.allclose(f[9:18], inner + [2 / 3, 1.0], atol=1e-14)
    assert np.allclose(f[18:27], inner + [1 / 3, 1.0], atol=1e-14)
    assert np.all(f[27:] == 0.0)
    # (4, 5, 7): the z line ends at the masked face z = Nz - 1 = 9: its last conductance is
    # -12 and its last diagonal ratio log10(1 / 6h)
    f = F[g(4, 5, 7)]
    expect_z = [np.log10(1 / 6), np.log10(1 / 6), -12.0, 0.0, 0.0, 0.0,
                np.log10(1.0 / (6 * h)), 1 / 3, 1.0]
    assert np.allclose(f[18:27], expect_z, atol=1e-13)
    # (2, 6, 4): x line from the masked node x = 0; y on a coarse index (rem 0)
    f = F[g(2, 6, 4)]
    expect_x = [-12.0, np.log10(1 / 6), np.log10(1 / 6),
                np.log10(1.0 / (6 * h)), 0.0, 0.0, 0.0, 2 / 3, 1.0]
    assert np.allclose(f[0:9], expect_x, atol=1e-13)
    assert np.all(f[9:18] == 0.0)
    assert np.allclose(f[18:27], inner + [1 / 3, 1.0], atol=1e-14)
