"""Seeded synthetic workloads for region multigrid: region maps and composite operators.

This module is the application side of the problem: it lays a structured global node grid,
tiles it with box-shaped regions that share their interface node layers, assembles the
fully assembled ("composite") matrix of a PDE on that grid, and draws a right-hand side.
It holds none of the multigrid method's arithmetic (no splitting, interpolation, Galerkin
products, smoothing or Krylov steps); both the CPU oracle and the GPU library consume its
output.

What an application hands to the method (Sec. 4 of the paper): a composite matrix, the
number of grid points per axis of every region, and a map from every regional node to its
composite node (global id). Interface nodes appear in every region that contains them.

Conventions used everywhere in this repository:

* Composite nodes are numbered lexicographically, x fastest: g = x + Nx*(y + Ny*z).
  Two-dimensional problems use Nz = 1.
* Regions are boxes of the global grid. Region (a, b, c) of a region grid covers global
  node indices [ox_a, ox_a + nx_a - 1] x [oy_b, ...] x [oz_c, ...] with o_{a+1} = o_a + n_a - 1,
  so neighbouring regions share one node layer. Regions are ordered x-fastest over the region
  grid; nodes inside a region are ordered x-fastest too.
* Dirichlet nodes stay in the grid but are masked: their row of the composite matrix is the
  identity, no unmasked row couples to them, and the right-hand side is zero there.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Problem:
    """A composite linear system A u = b on a structured grid tiled by box regions."""

    name: str
    dim: int                      # 2 or 3
    dofs_per_node: int            # 1 (scalar) or 3 (elasticity)
    global_dims: tuple            # (Nx, Ny, Nz) composite nodes per axis
    slabs: tuple                  # per axis, the node counts of the region slabs
    region_dims: np.ndarray       # (nregions, 3) int32, nodes per axis of every region
    region_gids: np.ndarray       # (n_r,) int64, composite node id of every regional node
    dirichlet: np.ndarray         # (n_nodes,) uint8, 1 where the node is masked
    A: sp.csr_matrix              # (n, n) float64 composite matrix, n = n_nodes * dofs_per_node
    b: np.ndarray                 # (n,) float64
    stencil: int                  # nominal stencil points per row (5, 7, 9, 27 or 81)
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.global_dims))

    @property
    def n(self) -> int:
        return self.n_nodes * self.dofs_per_node

    @property
    def n_regional_nodes(self) -> int:
        return int(self.region_gids.shape[0])

    @property
    def n_unknowns(self) -> int:
        """Unmasked degrees of freedom (the DOF count used for throughput)."""
        return int((self.dirichlet == 0).sum()) * self.dofs_per_node

    @property
    def nregions(self) -> int:
        return int(self.region_dims.shape[0])


# ----------------------------------------------------------------------------------------
# region maps

def slab_origins(sizes):
    """Global index of the first node of every slab; neighbours share one node layer."""
    o = [0]
    for s in sizes[:-1]:
        o.append(o[-1] + s - 1)
    return o


def region_map(slabs):
    """Region dims and the concatenated regional -> composite id map for a box tiling.

    ``slabs`` holds, per axis (x, y, z), the node counts of the slabs along that axis.
    """
    sx, sy, sz = (list(s) for s in slabs)
    Nx = sum(sx) - len(sx) + 1
    Ny = sum(sy) - len(sy) + 1
    Nz = sum(sz) - len(sz) + 1
    ox, oy, oz = slab_origins(sx), slab_origins(sy), slab_origins(sz)
    dims, gids = [], []
    for c, nz in enumerate(sz):
        for b, ny in enumerate(sy):
            for a, nx in enumerate(sx):
                dims.append((nx, ny, nz))
                x = ox[a] + np.arange(nx, dtype=np.int64)
                y = oy[b] + np.arange(ny, dtype=np.int64)
                z = oz[c] + np.arange(nz, dtype=np.int64)
                g = x[None, None, :] + Nx * (y[None, :, None] + Ny * z[:, None, None])
                gids.append(g.reshape(-1))
    return (Nx, Ny, Nz), np.asarray(dims, dtype=np.int32), np.concatenate(gids)


def boundary_mask(global_dims, faces=("x0", "x1", "y0", "y1", "z0", "z1")):
    """uint8 mask of nodes on the named faces of the global box (x0 = the x == 0 face)."""
    Nx, Ny, Nz = global_dims
    m = np.zeros((Nz, Ny, Nx), dtype=np.uint8)
    if "x0" in faces:
        m[:, :, 0] = 1
    if "x1" in faces:
        m[:, :, -1] = 1
    if "y0" in faces:
        m[:, 0, :] = 1
    if "y1" in faces:
        m[:, -1, :] = 1
    if Nz > 1:
        if "z0" in faces:
            m[0, :, :] = 1
        if "z1" in faces:
            m[-1, :, :] = 1
    return m.reshape(-1)


# ----------------------------------------------------------------------------------------
# composite assembly helpers

def _csr_from_stencil(global_dims, offsets, values, mask):
    """Assemble CSR from per-node stencil values.

    ``offsets`` is a list of (dx, dy, dz) in increasing order of the column index they
    produce; ``values`` is (len(offsets), Nz, Ny, Nx) with the coupling of node p to node
    p + offset. Entries that leave the grid or are exactly zero are dropped. Masked rows
    become identity rows and columns of masked nodes are removed from unmasked rows.
    """
    Nx, Ny, Nz = global_dims
    n = Nx * Ny * Nz
    S = len(offsets)
    z, y, x = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    maskg = mask.reshape(Nz, Ny, Nx).astype(bool)
    cols = np.empty((n, S), dtype=np.int64)
    vals = np.empty((n, S), dtype=np.float64)
    keep = np.empty((n, S), dtype=bool)
    for s, (dx, dy, dz) in enumerate(offsets):
        xx, yy, zz = x + dx, y + dy, z + dz
        inside = (xx >= 0) & (xx < Nx) & (yy >= 0) & (yy < Ny) & (zz >= 0) & (zz < Nz)
        g = np.where(inside, xx + Nx * (yy + Ny * zz), 0)
        centre = (dx, dy, dz) == (0, 0, 0)
        v = np.where(inside, values[s], 0.0)
        nb_masked = np.zeros_like(inside)
        nb_masked[inside] = maskg.reshape(-1)[g[inside]]
        if centre:
            v = np.where(maskg, 1.0, v)
            k = np.ones_like(inside)
        else:
            k = inside & ~maskg & ~nb_masked & (v != 0.0)
        cols[:, s] = g.reshape(-1)
        vals[:, s] = v.reshape(-1)
        keep[:, s] = k.reshape(-1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(keep.sum(axis=1), out=rowptr[1:])
    A = sp.csr_matrix((vals[keep], cols[keep], rowptr), shape=(n, n))
    A.sort_indices()
    return A


def _rhs(rng, n, mask, dofs_per_node=1):
    b = rng.uniform(-1.0, 1.0, size=n)
    if dofs_per_node == 1:
        b[mask.astype(bool)] = 0.0
    else:
        b.reshape(-1, dofs_per_node)[mask.astype(bool)] = 0.0
    return b


OFFS5 = [(0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
OFFS7 = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
OFFS27 = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
OFFS9 = [(dx, dy, 0) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


# ----------------------------------------------------------------------------------------
# workload families

def poisson2d_5pt(region_grid=(2, 2), n=82, seed=0, rhs=True):
    """2D Poisson, 5-point stencil [-1, 4], Dirichlet on the whole boundary."""
    slabs = ([n] * region_grid[0], [n] * region_grid[1], [1])
    gdims, rdims, gids = region_map(slabs)
    mask = boundary_mask(gdims)
    Nx, Ny, Nz = gdims
    vals = np.zeros((5, Nz, Ny, Nx))
    for s, off in enumerate(OFFS5):
        vals[s] = 4.0 if off == (0, 0, 0) else -1.0
    A = _csr_from_stencil(gdims, OFFS5, vals, mask)
    rng = np.random.default_rng(seed)
    b = _rhs(rng, A.shape[0], mask) if rhs else np.zeros(A.shape[0])
    return Problem("poisson2d_5pt", 2, 1, gdims, slabs, rdims, gids, mask, A, b, 5,
                   dict(seed=seed, region_grid=tuple(region_grid), n=n))


def _edge_kappa_3d(kappa):
    """Per axis, the mean element coefficient of the (up to 4) elements around each edge.

    ``kappa`` is (Ez, Ey, Ex) per element. Returns three arrays shaped (Nz, Ny, Nx) holding,
    for the edge from node p to p + e_axis, that mean (0 where the edge leaves the grid).
    """
    Ez, Ey, Ex = kappa.shape
    Nz, Ny, Nx = Ez + 1, Ey + 1, Ex + 1
    pad = np.full((Ez + 2, Ey + 2, Ex + 2), np.nan)
    pad[1:-1, 1:-1, 1:-1] = kappa
    out = []
    # x-edges: (x..x+1, y, z): elements with ex = x, ey in {y-1, y}, ez in {z-1, z}
    ex = np.zeros((Nz, Ny, Nx))
    blk = np.stack([pad[z0:z0 + Nz, y0:y0 + Ny, 1:Ex + 1]
                    for z0 in (0, 1) for y0 in (0, 1)])
    ex[:, :, :Ex] = np.nanmean(blk, axis=0)
    out.append(ex)
    ey = np.zeros((Nz, Ny, Nx))
    blk = np.stack([pad[z0:z0 + Nz, 1:Ey + 1, x0:x0 + Nx]
                    for z0 in (0, 1) for x0 in (0, 1)])
    ey[:, :Ey, :] = np.nanmean(blk, axis=0)
    out.append(ey)
    ez = np.zeros((Nz, Ny, Nx))
    blk = np.stack([pad[1:Ez + 1, y0:y0 + Ny, x0:x0 + Nx]
                    for y0 in (0, 1) for x0 in (0, 1)])
    ez[:Ez, :, :] = np.nanmean(blk, axis=0)
    out.append(ez)
    return out


def diffusion3d_7pt_from_kappa(gdims, kappa, mask):
    """Vertex-centred 7-point finite differences for -div(kappa grad u).

    The coupling across the edge (p, p + e) is -h * (mean kappa of the elements around that
    edge); the diagonal is minus the sum of all couplings of the node, including those to
    masked neighbours (which are then removed from the row). h = 1/(Nx - 1).
    """
    Nx, Ny, Nz = gdims
    h = 1.0 / (Nx - 1)
    ekx, eky, ekz = _edge_kappa_3d(kappa)
    vals = np.zeros((7, Nz, Ny, Nx))
    cx, cy, cz = -h * ekx, -h * eky, -h * ekz
    # offsets order: -z, -y, -x, 0, +x, +y, +z
    vals[6] = cz
    vals[5] = cy
    vals[4] = cx
    vals[2][:, :, 1:] = cx[:, :, :-1]
    vals[1][:, 1:, :] = cy[:, :-1, :]
    vals[0][1:, :, :] = cz[:-1, :, :]
    vals[3] = -(vals[0] + vals[1] + vals[2] + vals[4] + vals[5] + vals[6])
    return _csr_from_stencil(gdims, OFFS7, vals, mask)


def draw_slabs(rng, region_grid, choices):
    return tuple(list(rng.choice(np.asarray(choices), size=k)) for k in region_grid)


def diffusion3d_7pt(region_grid=(8, 8, 4), choices=(28, 55, 82), seed=1, sigma=1.0,
                    rhs=True):
    """3D variable-coefficient diffusion, 7-point stencil, log-normal per-element kappa.

    Slab node counts per axis and then the per-element kappa = exp(N(0, sigma^2)) and the
    right-hand side U[-1, 1] all come from one numpy Generator seeded with ``seed``.
    Homogeneous Dirichlet on all six faces.
    """
    rng = np.random.default_rng(seed)
    slabs = tuple(int(v) for v in rng.choice(np.asarray(choices), size=region_grid[0])), \
        tuple(int(v) for v in rng.choice(np.asarray(choices), size=region_grid[1])), \
        tuple(int(v) for v in rng.choice(np.asarray(choices), size=region_grid[2]))
    gdims, rdims, gids = region_map(slabs)
    Nx, Ny, Nz = gdims
    kappa = np.exp(sigma * rng.standard_normal(size=(Nz - 1, Ny - 1, Nx - 1)))
    mask = boundary_mask(gdims)
    A = diffusion3d_7pt_from_kappa(gdims, kappa, mask)
    b = _rhs(rng, A.shape[0], mask) if rhs else np.zeros(A.shape[0])
    return Problem("diffusion3d_7pt", 3, 1, gdims, slabs, rdims, gids, mask, A, b, 7,
                   dict(seed=seed, region_grid=tuple(region_grid), choices=tuple(choices),
                        sigma=sigma))


def highcontrast3d_7pt(region_grid=(7, 7, 7), choices=(28, 55, 82), seed=3, rhs=True,
                       log10_range=(-3.0, 3.0)):
    """3D 7-point diffusion with kappa constant per region, log-uniform in 10^range."""
    rng = np.random.default_rng(seed)
    slabs = tuple(tuple(int(v) for v in rng.choice(np.asarray(choices), size=k))
                  for k in region_grid)
    gdims, rdims, gids = region_map(slabs)
    Nx, Ny, Nz = gdims
    kreg = 10.0 ** rng.uniform(log10_range[0], log10_range[1], size=tuple(region_grid)[::-1])
    kappa = np.empty((Nz - 1, Ny - 1, Nx - 1))
    ox, oy, oz = (slab_origins(s) for s in slabs)
    for c, nz in enumerate(slabs[2]):
        for bb, ny in enumerate(slabs[1]):
            for a, nx in enumerate(slabs[0]):
                kappa[oz[c]:oz[c] + nz - 1, oy[bb]:oy[bb] + ny - 1, ox[a]:ox[a] + nx - 1] = \
                    kreg[c, bb, a]
    mask = boundary_mask(gdims)
    A = diffusion3d_7pt_from_kappa(gdims, kappa, mask)
    b = _rhs(rng, A.shape[0], mask) if rhs else np.zeros(A.shape[0])
    return Problem("highcontrast3d_7pt", 3, 1, gdims, slabs, rdims, gids, mask, A, b, 7,
                   dict(seed=seed, region_grid=tuple(region_grid), choices=tuple(choices),
                        kappa_region=kreg))


def q1_element_laplacian(h=1.0):
    """8x8 stiffness matrix of the trilinear hexahedron [0,h]^3 by 2x2x2 Gauss quadrature.

    Local node a has corner offsets (a & 1, (a >> 1) & 1, (a >> 2) & 1).
    """
    g = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    corners = np.array([[(a >> 0) & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float)
    K = np.zeros((8, 8))
    for qz in g:
        for qy in g:
            for qx in g:
                xi = (np.array([qx, qy, qz]) + 1.0) / 2.0  # in [0,1]^3
                grads = np.zeros((8, 3))
                for a in range(8):
                    c = corners[a]
                    f = [xi[d] if c[d] else 1.0 - xi[d] for d in range(3)]
                    df = [1.0 if c[d] else -1.0 for d in range(3)]
                    grads[a] = [df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]]
                # reference [0,1]^3 -> [0,h]^3: grad scales 1/h, volume h^3, weights 1/8 each
                K += (grads @ grads.T) * (1.0 / 8.0)
    return K * h  # h^3 * (1/h)^2


def q1_laplace3d(region_grid=(8, 8, 8), n=55, seed=2, rhs=True):
    """3D Q1 (trilinear) Laplacian, 27-point stencil, constant coefficient."""
    slabs = tuple([n] * k for k in region_grid)
    gdims, rdims, gids = region_map(slabs)
    Nx, Ny, Nz = gdims
    h = 1.0 / (Nx - 1)
    Ke = q1_element_laplacian(h)
    corners = [((a >> 0) & 1, (a >> 1) & 1, (a >> 2) & 1) for a in range(8)]
    vals = np.zeros((27, Nz, Ny, Nx))
    # every element adds Ke[a, c] to the coupling node(a) -> node(c)
    for a, (ax, ay, az) in enumerate(corners):
        for c, (cx, cy, cz) in enumerate(corners):
            dx, dy, dz = cx - ax, cy - ay, cz - az
            s = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
            # node p = element origin + corner a, for element origins e in [0, N-2]
            vals[s, az:az + Nz - 1, ay:ay + Ny - 1, ax:ax + Nx - 1] += Ke[a, c]
    mask = boundary_mask(gdims)
    A = _csr_from_stencil(gdims, OFFS27, vals, mask)
    rng = np.random.default_rng(seed)
    b = _rhs(rng, A.shape[0], mask) if rhs else np.zeros(A.shape[0])
    return Problem("q1_laplace3d", 3, 1, gdims, slabs, rdims, gids, mask, A, b, 27,
                   dict(seed=seed, region_grid=tuple(region_grid), n=n))


def q1_laplace2d(region_grid=(2, 2), n=28, seed=0, rhs=True):
    """2D Q1 (bilinear) Laplacian, 9-point stencil [-1/3 ... 8/3]."""
    slabs = ([n] * region_grid[0], [n] * region_grid[1], [1])
    gdims, rdims, gids = region_map(slabs)
    Nx, Ny, Nz = gdims
    vals = np.zeros((9, Nz, Ny, Nx))
    # bilinear element stiffness on a square: diag 2/3, edge -1/6, diagonal -1/3
    Ke = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    corners = [(0, 0), (1, 0), (0, 1), (1, 1)]
    for a, (ax, ay) in enumerate(corners):
        for c, (cx, cy) in enumerate(corners):
            s = (cx - ax + 1) + 3 * (cy - ay + 1)
            vals[s, 0, ay:ay + Ny - 1, ax:ax + Nx - 1] += Ke[a, c]
    mask = boundary_mask(gdims)
    A = _csr_from_stencil(gdims, OFFS9, vals, mask)
    rng = np.random.default_rng(seed)
    b = _rhs(rng, A.shape[0], mask) if rhs else np.zeros(A.shape[0])
    return Problem("q1_laplace2d", 2, 1, gdims, slabs, rdims, gids, mask, A, b, 9,
                   dict(seed=seed, region_grid=tuple(region_grid), n=n))


# ----------------------------------------------------------------------------------------
# named configurations

def q1_laplace2d_box(nx, ny, seed=0, rhs=True):
    """2D Q1 Laplacian (9-point) on one region of nx x ny nodes (the single-region meshes of
    the triple-product timings, Table 4)."""
    slabs = ([nx], [ny], [1])
    gdims, rdims, gids = region_map(slabs)
    Nx, Ny, Nz = gdims
    vals = np.zeros((9, Nz, Ny, Nx))
    Ke = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    corners = [(0, 0), (1, 0), (0, 1), (1, 1)]
    for a, (ax, ay) in enumerate(corners):
        for c, (cx, cy) in enumerate(corners):
            s = (cx - ax + 1) + 3 * (cy - ay + 1)
            vals[s, 0, ay:ay + Ny - 1, ax:ax + Nx - 1] += Ke[a, c]
    mask = boundary_mask(gdims)
    A = _csr_from_stencil(gdims, OFFS9, vals, mask)
    rng = np.random.default_rng(seed)
    b = _rhs(rng, A.shape[0], mask) if rhs else np.zeros(A.shape[0])
    return Problem("q1_laplace2d_box", 2, 1, gdims, slabs, rdims, gids, mask, A, b, 9,
                   dict(seed=seed, nx=nx, ny=ny))


def config(name: str, **kw) -> Problem:
    """The five paper-shaped workloads by name, with optional size overrides."""
    if name == "c1_poisson2d":
        return poisson2d_5pt(**{"region_grid": (2, 2), "n": 82, "seed": 0, **kw})
    if name == "c2_diffusion3d":
        return diffusion3d_7pt(**{"region_grid": (8, 8, 4), "choices": (28, 55, 82),
                                  "seed": 1, **kw})
    if name == "c3_q1laplace3d":
        return q1_laplace3d(**{"region_grid": (8, 8, 8), "n": 55, "seed": 2, **kw})
    if name == "c4_highcontrast3d":
        return highcontrast3d_7pt(**{"region_grid": (7, 7, 7), "choices": (28, 55, 82),
                                     "seed": 3, **kw})
    raise KeyError(name)


# ----------------------------------------------------------------------------------------
# linear elasticity (3 dofs per node)

def q1_element_elasticity(h=1.0, E=1.0, nu=0.3):
    """24x24 stiffness of the trilinear hexahedron [0,h]^3 for isotropic linear elasticity
    (2x2x2 Gauss quadrature). Dofs are node-major: 3 a + c for local node a, component c;
    local node a has corner offsets (a & 1, (a >> 1) & 1, (a >> 2) & 1)."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    g = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    corners = np.array([[(a >> 0) & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float)
    K = np.zeros((24, 24))
    for qz in g:
        for qy in g:
            for qx in g:
                xi = (np.array([qx, qy, qz]) + 1.0) / 2.0
                Bm = np.zeros((6, 24))
                for a in range(8):
                    c = corners[a]
                    f = [xi[d] if c[d] else 1.0 - xi[d] for d in range(3)]
                    df = [1.0 if c[d] else -1.0 for d in range(3)]
                    dx, dy, dz = (np.array([df[0] * f[1] * f[2], f[0] * df[1] * f[2],
                                            f[0] * f[1] * df[2]]) / h)
                    Bm[0, 3 * a] = dx
                    Bm[1, 3 * a + 1] = dy
                    Bm[2, 3 * a + 2] = dz
                    Bm[3, 3 * a], Bm[3, 3 * a + 1] = dy, dx
                    Bm[4, 3 * a + 1], Bm[4, 3 * a + 2] = dz, dy
                    Bm[5, 3 * a], Bm[5, 3 * a + 2] = dz, dx
                K += Bm.T @ D @ Bm * (h ** 3 / 8.0)
    return K


def _csr_from_block_stencil(global_dims, offsets, values, mask, B):
    """CSR (dofs node-major, g * B + c) from per-node B x B block stencils values[s, c, c']."""
    Nx, Ny, Nz = global_dims
    n = Nx * Ny * Nz
    S = len(offsets)
    z, y, x = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    maskg = mask.reshape(Nz, Ny, Nx).astype(bool)
    cols = np.empty((n, B, S, B), dtype=np.int64)
    vals = np.empty((n, B, S, B), dtype=np.float64)
    keep = np.empty((n, B, S, B), dtype=bool)
    for s, (dx, dy, dz) in enumerate(offsets):
        xx, yy, zz = x + dx, y + dy, z + dz
        inside = (xx >= 0) & (xx < Nx) & (yy >= 0) & (yy < Ny) & (zz >= 0) & (zz < Nz)
        g = np.where(inside, xx + Nx * (yy + Ny * zz), 0)
        centre = (dx, dy, dz) == (0, 0, 0)
        nb_masked = np.zeros_like(inside)
        nb_masked[inside] = maskg.reshape(-1)[g[inside]]
        for c in range(B):
            for c2 in range(B):
                v = np.where(inside, values[s, c, c2], 0.0)
                if centre:
                    v = np.where(maskg, 1.0 if c == c2 else 0.0, v)
                    k = (~maskg) | (c == c2)
                    k = k & ((v != 0.0) | (c == c2))
                else:
                    k = inside & ~maskg & ~nb_masked & (v != 0.0)
                cols[:, c, s, c2] = (g * B + c2).reshape(-1)
                vals[:, c, s, c2] = v.reshape(-1)
                keep[:, c, s, c2] = k.reshape(-1)
    cols = cols.reshape(n * B, S * B)
    vals = vals.reshape(n * B, S * B)
    keep = keep.reshape(n * B, S * B)
    rowptr = np.zeros(n * B + 1, dtype=np.int64)
    np.cumsum(keep.sum(axis=1), out=rowptr[1:])
    A = sp.csr_matrix((vals[keep], cols[keep], rowptr), shape=(n * B, n * B))
    A.sort_indices()
    return A


def elasticity3d(region_grid=(3, 3, 3), choices=(28,), seed=4, sigma=0.5, nu=0.3, rhs=True,
                 load=(0.0, 0.0, -1.0)):
    """3D linear elasticity, trilinear hexahedra, 3 dofs per node, Young's modulus
    E = exp(N(0, sigma^2)) per element, Poisson ratio nu, the x = 0 face clamped, uniform body
    load lumped to the nodes (h^3 per node)."""
    rng = np.random.default_rng(seed)
    slabs = tuple(tuple(int(v) for v in rng.choice(np.asarray(choices), size=k))
                  for k in region_grid)
    gdims, rdims, gids = region_map(slabs)
    Nx, Ny, Nz = gdims
    h = 1.0 / (Nx - 1)
    E = np.exp(sigma * rng.standard_normal(size=(Nz - 1, Ny - 1, Nx - 1)))
    Ke = q1_element_elasticity(h, 1.0, nu)
    corners = [((a >> 0) & 1, (a >> 1) & 1, (a >> 2) & 1) for a in range(8)]
    vals = np.zeros((27, 3, 3, Nz, Ny, Nx))
    for a, (ax, ay, az) in enumerate(corners):
        for c, (cx, cy, cz) in enumerate(corners):
            s = (cx - ax + 1) + 3 * (cy - ay + 1) + 9 * (cz - az + 1)
            blk = Ke[3 * a:3 * a + 3, 3 * c:3 * c + 3]
            for i in range(3):
                for j in range(3):
                    vals[s, i, j, az:az + Nz - 1, ay:ay + Ny - 1, ax:ax + Nx - 1] += blk[i, j] * E
    mask = boundary_mask(gdims, faces=("x0",))
    A = _csr_from_block_stencil(gdims, OFFS27, vals, mask, 3)
    n = Nx * Ny * Nz
    b = np.zeros(3 * n)
    if rhs:
        b.reshape(n, 3)[:] = np.asarray(load) * h ** 3
        b.reshape(n, 3)[mask.astype(bool)] = 0.0
    return Problem("elasticity3d", 3, 3, gdims, slabs, rdims, gids, mask, A, b, 27,
                   dict(seed=seed, region_grid=tuple(region_grid), choices=tuple(choices),
                        sigma=sigma, nu=nu))


# ----------------------------------------------------------------------------------------
# batches of independent problems

@dataclass
class Batch:
    """Independent problems side by side as one system: the composite ids and regions of
    problem k follow those of problems 0 .. k-1, A is block diagonal, and b, the mask and the
    region maps are concatenated. The method sees K disconnected components, so one hierarchy
    (and one V-cycle) treats all of them at once, and quantities summed over the regions of a
    component belong to that problem alone."""

    name: str
    dim: int
    dofs_per_node: int
    stencil: int
    region_dims: np.ndarray       # (nregions, 3) int32
    region_gids: np.ndarray       # (n_r,) int64
    dirichlet: np.ndarray         # (n_nodes,) uint8
    A: sp.csr_matrix
    b: np.ndarray
    region_component: np.ndarray  # (nregions,) int32: the problem every region belongs to
    node_offsets: np.ndarray      # (K + 1,) int64: composite id range of every problem
    members: list = field(default_factory=list)

    @property
    def n_nodes(self) -> int:
        return int(self.dirichlet.shape[0])

    @property
    def n(self) -> int:
        return self.n_nodes * self.dofs_per_node

    @property
    def n_regional_nodes(self) -> int:
        return int(self.region_gids.shape[0])

    @property
    def n_unknowns(self) -> int:
        return int((self.dirichlet == 0).sum()) * self.dofs_per_node

    @property
    def nregions(self) -> int:
        return int(self.region_dims.shape[0])


def batch(problems) -> Batch:
    """Concatenate scalar problems of one dimension and stencil into a Batch."""
    p0 = problems[0]
    assert all(p.dim == p0.dim and p.stencil == p0.stencil and p.dofs_per_node == 1
               for p in problems)
    offs = np.concatenate([[0], np.cumsum([p.n_nodes for p in problems])]).astype(np.int64)
    gids = np.concatenate([p.region_gids + o for p, o in zip(problems, offs[:-1])])
    comp = np.concatenate([np.full(p.nregions, k, dtype=np.int32)
                           for k, p in enumerate(problems)])
    return Batch(name=f"batch_{p0.name}", dim=p0.dim, dofs_per_node=1, stencil=p0.stencil,
                 region_dims=np.concatenate([p.region_dims for p in problems]).astype(np.int32),
                 region_gids=gids.astype(np.int64),
                 dirichlet=np.concatenate([p.dirichlet for p in problems]).astype(np.uint8),
                 A=sp.block_diag([p.A for p in problems], format="csr"),
                 b=np.concatenate([p.b for p in problems]),
                 region_component=comp, node_offsets=offs, members=list(problems))


def highcontrast3d_offset(region_grid=(2, 2, 2), choices=(10,), seed=0, rhs=True,
                          log10_range=(-3.0, 3.0), blocks=4):
    """3D 7-point diffusion whose coefficient jumps lie off the coarse-grid planes: kappa is
    log-uniform in 10^range on a `blocks`^3 grid of boxes whose faces sit at element layers
    1 or 2 modulo 3 (never on a layer of coarse nodes), so a fine node between two coarse nodes
    can see a jump inside its interpolation line."""
    rng = np.random.default_rng(seed)
    slabs = tuple(tuple(int(v) for v in rng.choice(np.asarray(choices), size=k))
                  for k in region_grid)
    gdims, rdims, gids = region_map(slabs)
    Nx, Ny, Nz = gdims
    cuts = []
    for N in (Nx, Ny, Nz):
        inner = [e for e in range(1, N - 2) if e % 3 != 0]
        pick = np.sort(rng.choice(np.asarray(inner), size=min(blocks - 1, len(inner)),
                                  replace=False))
        cuts.append(np.concatenate([[0], pick, [N - 1]]))
    kb = 10.0 ** rng.uniform(log10_range[0], log10_range[1],
                             size=(len(cuts[2]) - 1, len(cuts[1]) - 1, len(cuts[0]) - 1))
    kappa = np.empty((Nz - 1, Ny - 1, Nx - 1))
    for c in range(len(cuts[2]) - 1):
        for bb in range(len(cuts[1]) - 1):
            for a in range(len(cuts[0]) - 1):
                kappa[cuts[2][c]:cuts[2][c + 1], cuts[1][bb]:cuts[1][bb + 1],
                      cuts[0][a]:cuts[0][a + 1]] = kb[c, bb, a]
    mask = boundary_mask(gdims)
    A = diffusion3d_7pt_from_kappa(gdims, kappa, mask)
    b = _rhs(rng, A.shape[0], mask) if rhs else np.zeros(A.shape[0])
    return Problem("highcontrast3d_offset", 3, 1, gdims, slabs, rdims, gids, mask, A, b, 7,
                   dict(seed=seed, region_grid=tuple(region_grid), choices=tuple(choices),
                        cuts=[c.tolist() for c in cuts], kappa_block=kb))
