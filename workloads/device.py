"""Device-side generation of the large structured workloads.

The 3D Q1 Laplacian on 8x8x8 regions of 55^3 nodes (81M unknowns, 2.2 billion nonzeros) and
3D linear elasticity on 8x8x8 regions (54M unknowns, 4.4 billion nonzeros) would need tens of
GB of host memory and minutes of single-threaded numpy to assemble on the host. This module
assembles the same composite CSR with torch on the device: the same recipe, the same values
(bit for bit, as the CPU tests check against the numpy generators on small grids), the same
random numbers (drawn on the host with numpy from the same seeds). It holds none of the
method's arithmetic.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import (OFFS27, boundary_mask, q1_element_elasticity, q1_element_laplacian, region_map)


class DeviceWorkload:
    """A problem whose composite CSR (rowptr, col, val) and right-hand side b live on the
    device; region map, mask and sizes on the host (the fields of workloads.Problem)."""

    def __init__(self, name, dim, dofs_per_node, global_dims, slabs, region_dims, region_gids,
                 dirichlet, rowptr, col, val, b, stencil, meta):
        self.name, self.dim, self.dofs_per_node = name, dim, dofs_per_node
        self.global_dims, self.slabs = tuple(global_dims), slabs
        self.region_dims = np.asarray(region_dims, dtype=np.int32)
        self.region_gids = np.asarray(region_gids, dtype=np.int64)
        self.dirichlet = np.asarray(dirichlet, dtype=np.uint8)
        self.rowptr, self.col, self.val, self.b = rowptr, col, val, b
        self.stencil, self.meta = stencil, meta

    @property
    def n_nodes(self):
        return int(np.prod(self.global_dims))

    @property
    def n(self):
        return self.n_nodes * self.dofs_per_node

    @property
    def n_regional_nodes(self):
        return int(self.region_gids.shape[0])

    @property
    def n_unknowns(self):
        return int(np.count_nonzero(self.dirichlet == 0)) * self.dofs_per_node

    @property
    def nregions(self):
        return int(self.region_dims.shape[0])

    @property
    def nnz(self):
        return int(self.col.numel())

    def rows(self, idx):
        """Host scipy CSR of shape (n, n) holding the given rows of A (others empty)."""
        import torch
        idx = np.asarray(idx, dtype=np.int64)
        rp = self.rowptr.cpu().numpy() if self.rowptr.numel() < (1 << 27) else None
        if rp is None:
            t = torch.from_numpy(idx).to(self.rowptr.device)
            starts, ends = self.rowptr[t].cpu().numpy(), self.rowptr[t + 1].cpu().numpy()
        else:
            starts, ends = rp[idx], rp[idx + 1]
        lens = ends - starts
        pos = np.repeat(starts - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens) + \
            np.arange(int(lens.sum()))
        tp = torch.from_numpy(pos).to(self.col.device)
        cols = self.col[tp].cpu().numpy()
        vals = self.val[tp].cpu().numpy()
        rows = np.repeat(idx, lens)
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n, self.n))


def _grid(gdims, device):
    import torch
    Nx, Ny, Nz = gdims
    z = torch.arange(Nz, device=device, dtype=torch.int64).view(Nz, 1, 1)
    y = torch.arange(Ny, device=device, dtype=torch.int64).view(1, Ny, 1)
    x = torch.arange(Nx, device=device, dtype=torch.int64).view(1, 1, Nx)
    return x, y, z


def _slot_terms(gdims, off, x, y, z, maskg, vals_s, centre, c_is_c2=True):
    """Per-node column, value and keep flag of stencil slot `off` (the rules of the numpy
    assembly: entries leaving the grid or exactly zero dropped, masked rows identity rows,
    columns of masked nodes removed)."""
    import torch
    Nx, Ny, Nz = gdims
    dx, dy, dz = off
    xx, yy, zz = x + dx, y + dy, z + dz
    inside = (xx >= 0) & (xx < Nx) & (yy >= 0) & (yy < Ny) & (zz >= 0) & (zz < Nz)
    g = torch.where(inside, xx + Nx * (yy + Ny * zz), torch.zeros((), dtype=torch.int64,
                                                                   device=x.device))
    nb_masked = maskg.reshape(-1)[g.reshape(-1)].view_as(inside) & inside
    v = torch.where(inside, vals_s, torch.zeros((), dtype=vals_s.dtype, device=x.device))
    if centre:
        one = torch.ones((), dtype=v.dtype, device=x.device)
        zero = torch.zeros((), dtype=v.dtype, device=x.device)
        v = torch.where(maskg, one if c_is_c2 else zero, v)
        if c_is_c2:
            k = torch.ones_like(inside)
        else:
            k = (~maskg) & (v != 0.0)
    else:
        k = inside & ~maskg & ~nb_masked & (v != 0.0)
    return g.reshape(-1), v.reshape(-1), k.reshape(-1)


def _csr_scalar(gdims, offsets, values, mask, device):
    import torch
    x, y, z = _grid(gdims, device)
    Nx, Ny, Nz = gdims
    n = Nx * Ny * Nz
    maskg = mask.view(Nz, Ny, Nx)
    count = torch.zeros(n, dtype=torch.int64, device=device)
    for s, off in enumerate(offsets):
        _, _, k = _slot_terms(gdims, off, x, y, z, maskg, values[s], off == (0, 0, 0))
        count += k
    rowptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(count, 0, out=rowptr[1:])
    nnz = int(rowptr[-1].item())
    col = torch.empty(nnz, dtype=torch.int64, device=device)
    val = torch.empty(nnz, dtype=torch.float64, device=device)
    running = rowptr[:-1].clone()
    for s, off in enumerate(offsets):
        g, v, k = _slot_terms(gdims, off, x, y, z, maskg, values[s], off == (0, 0, 0))
        pos = running[k]
        col[pos] = g[k]
        val[pos] = v[k]
        running += k
        del g, v, k, pos
    return rowptr, col, val


def _csr_block(gdims, offsets, values, mask, B, device):
    """Node-major dofs (g * B + c); columns of a row in (slot, c') order, as the numpy one."""
    import torch
    x, y, z = _grid(gdims, device)
    Nx, Ny, Nz = gdims
    n = Nx * Ny * Nz
    maskg = mask.view(Nz, Ny, Nx)
    count = torch.zeros((n, B), dtype=torch.int64, device=device)
    for s, off in enumerate(offsets):
        for c in range(B):
            for c2 in range(B):
                _, _, k = _slot_terms(gdims, off, x, y, z, maskg, values[s, c, c2],
                                      off == (0, 0, 0), c == c2)
                count[:, c] += k
    rowptr = torch.zeros(n * B + 1, dtype=torch.int64, device=device)
    torch.cumsum(count.reshape(-1), 0, out=rowptr[1:])
    del count
    nnz = int(rowptr[-1].item())
    col = torch.empty(nnz, dtype=torch.int64, device=device)
    val = torch.empty(nnz, dtype=torch.float64, device=device)
    running = rowptr[:-1].view(n, B).clone()
    for s, off in enumerate(offsets):
        for c in range(B):
            for c2 in range(B):
                g, v, k = _slot_terms(gdims, off, x, y, z, maskg, values[s, c, c2],
                                      off == (0, 0, 0), c == c2)
                pos = running[:, c][k]
                col[pos] = g[k] * B + c2
                val[pos] = v[k]
                running[:, c] += k
                del g, v, k, pos
    return rowptr, col, val


def q1_laplace3d(region_grid=(8, 8, 8), n=55, seed=2, device="cuda:0"):
    """The 3D Q1 Laplacian of workloads.q1_laplace3d, assembled on the device."""
    import torch
    slabs = tuple([n] * k for k in region_grid)
    gdims, rdims, gids = region_map(slabs)
    Nx, Ny, Nz = gdims
    h = 1.0 / (Nx - 1)
    Ke = q1_element_laplacian(h)
    corners = [((a >> 0) & 1, (a >> 1) & 1, (a >> 2) & 1) for a in range(8)]
    vals = torch.zeros((27, Nz, Ny, Nx), dtype=torch.float64, device=device)
    for a, (ax, ay, az) in enumerate(corners):
        for c, (cx, cy, cz) in enumerate(corners):
            s = (cx - ax + 1) + 3 * (cy - ay + 1) + 9 * (cz - az + 1)
            vals[s, az:az + Nz - 1, ay:ay + Ny - 1, ax:ax + Nx - 1] += float(Ke[a, c])
    mask = boundary_mask(gdims)
    maskt = torch.from_numpy(mask.astype(bool)).to(device)
    rowptr, col, val = _csr_scalar(gdims, OFFS27, vals, maskt, device)
    del vals
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1.0, 1.0, size=Nx * Ny * Nz)
    b[mask.astype(bool)] = 0.0
    return DeviceWorkload("q1_laplace3d", 3, 1, gdims, slabs, rdims, gids, mask, rowptr, col,
                          val, torch.from_numpy(b).to(device), 27,
                          dict(seed=seed, region_grid=tuple(region_grid), n=n))


def elasticity3d(region_grid=(8, 8, 8), choices=(28, 55), seed=95, sigma=0.5, nu=0.3,
                 load=(0.0, 0.0, -1.0), device="cuda:0"):
    """The 3D linear elasticity of workloads.elasticity3d, assembled on the device."""
    import torch
    rng = np.random.default_rng(seed)
    slabs = tuple(tuple(int(v) for v in rng.choice(np.asarray(choices), size=k))
                  for k in region_grid)
    gdims, rdims, gids = region_map(slabs)
    Nx, Ny, Nz = gdims
    h = 1.0 / (Nx - 1)
    E = torch.from_numpy(np.exp(sigma * rng.standard_normal(size=(Nz - 1, Ny - 1, Nx - 1)))
                         ).to(device)
    Ke = q1_element_elasticity(h, 1.0, nu)
    corners = [((a >> 0) & 1, (a >> 1) & 1, (a >> 2) & 1) for a in range(8)]
    vals = torch.zeros((27, 3, 3, Nz, Ny, Nx), dtype=torch.float64, device=device)
    for a, (ax, ay, az) in enumerate(corners):
        for c, (cx, cy, cz) in enumerate(corners):
            s = (cx - ax + 1) + 3 * (cy - ay + 1) + 9 * (cz - az + 1)
            for i in range(3):
                for j in range(3):
                    vals[s, i, j, az:az + Nz - 1, ay:ay + Ny - 1, ax:ax + Nx - 1] += \
                        float(Ke[3 * a + i, 3 * c + j]) * E
    del E
    mask = boundary_mask(gdims, faces=("x0",))
    maskt = torch.from_numpy(mask.astype(bool)).to(device)
    rowptr, col, val = _csr_block(gdims, OFFS27, vals, maskt, 3, device)
    del vals
    n = Nx * Ny * Nz
    b = np.zeros(3 * n)
    b.reshape(n, 3)[:] = np.asarray(load) * h ** 3
    b.reshape(n, 3)[mask.astype(bool)] = 0.0
    return DeviceWorkload("elasticity3d", 3, 3, gdims, slabs, rdims, gids, mask, rowptr, col,
                          val, torch.from_numpy(b).to(device), 27,
                          dict(seed=seed, region_grid=tuple(region_grid), choices=tuple(choices),
                               sigma=sigma, nu=nu))


def _edge_kappa_3d(kappa):
    """Torch form of workloads._edge_kappa_3d: per axis, the mean coefficient of the (up to 4)
    elements around each edge, added in the numpy order (slice 0, 1, 2, 3) and divided by the
    count of elements present."""
    import torch
    Ez, Ey, Ex = kappa.shape
    Nz, Ny, Nx = Ez + 1, Ey + 1, Ex + 1
    dev = kappa.device
    pad = torch.full((Ez + 2, Ey + 2, Ex + 2), float("nan"), dtype=torch.float64, device=dev)
    pad[1:-1, 1:-1, 1:-1] = kappa

    def nanmean(slices):
        tot = torch.zeros_like(slices[0])
        cnt = torch.zeros_like(slices[0])
        for v in slices:
            ok = ~torch.isnan(v)
            tot = tot + torch.where(ok, v, torch.zeros((), dtype=v.dtype, device=dev))
            cnt = cnt + ok.to(v.dtype)
        return tot / cnt

    ex = torch.zeros((Nz, Ny, Nx), dtype=torch.float64, device=dev)
    ex[:, :, :Ex] = nanmean([pad[z0:z0 + Nz, y0:y0 + Ny, 1:Ex + 1]
                             for z0 in (0, 1) for y0 in (0, 1)])
    ey = torch.zeros((Nz, Ny, Nx), dtype=torch.float64, device=dev)
    ey[:, :Ey, :] = nanmean([pad[z0:z0 + Nz, 1:Ey + 1, x0:x0 + Nx]
                             for z0 in (0, 1) for x0 in (0, 1)])
    ez = torch.zeros((Nz, Ny, Nx), dtype=torch.float64, device=dev)
    ez[:Ez, :, :] = nanmean([pad[1:Ez + 1, y0:y0 + Ny, x0:x0 + Nx]
                             for y0 in (0, 1) for x0 in (0, 1)])
    return ex, ey, ez


def _diffusion_csr(gdims, kappa, mask, device):
    """Vertex-centred 7-point coefficients of workloads.diffusion3d_7pt_from_kappa, assembled
    into CSR on the device."""
    import torch
    from . import OFFS7
    Nx, Ny, Nz = gdims
    h = 1.0 / (Nx - 1)
    ekx, eky, ekz = _edge_kappa_3d(kappa)
    vals = torch.zeros((7, Nz, Ny, Nx), dtype=torch.float64, device=device)
    cx, cy, cz = -h * ekx, -h * eky, -h * ekz
    del ekx, eky, ekz
    vals[6] = cz
    vals[5] = cy
    vals[4] = cx
    vals[2][:, :, 1:] = cx[:, :, :-1]
    vals[1][:, 1:, :] = cy[:, :-1, :]
    vals[0][1:, :, :] = cz[:-1, :, :]
    del cx, cy, cz
    vals[3] = -(vals[0] + vals[1] + vals[2] + vals[4] + vals[5] + vals[6])
    maskt = torch.from_numpy(mask.astype(bool)).to(device)
    return _csr_scalar(gdims, OFFS7, vals, maskt, device)


def _rhs_device(rng, n, mask, device):
    import torch
    b = rng.uniform(-1.0, 1.0, size=n)
    b[mask.astype(bool)] = 0.0
    return torch.from_numpy(b).to(device)


def diffusion3d_7pt(region_grid=(8, 8, 4), choices=(28, 55, 82), seed=1, sigma=1.0,
                    device="cuda:0"):
    """The 3D variable-coefficient diffusion of workloads.diffusion3d_7pt, assembled on the
    device (slab sizes, kappa and b drawn on the host from the same Generator, in the same
    order)."""
    import torch
    rng = np.random.default_rng(seed)
    slabs = tuple(tuple(int(v) for v in rng.choice(np.asarray(choices), size=k))
                  for k in region_grid)
    gdims, rdims, gids = region_map(slabs)
    Nx, Ny, Nz = gdims
    kappa = torch.from_numpy(np.exp(sigma * rng.standard_normal(size=(Nz - 1, Ny - 1, Nx - 1)))
                             ).to(device)
    mask = boundary_mask(gdims)
    rowptr, col, val = _diffusion_csr(gdims, kappa, mask, device)
    del kappa
    b = _rhs_device(rng, Nx * Ny * Nz, mask, device)
    return DeviceWorkload("diffusion3d_7pt", 3, 1, gdims, slabs, rdims, gids, mask, rowptr,
                          col, val, b, 7, dict(seed=seed, region_grid=tuple(region_grid),
                                               choices=tuple(choices), sigma=sigma))


def highcontrast3d_7pt(region_grid=(7, 7, 7), choices=(28, 55, 82), seed=3,
                       log10_range=(-3.0, 3.0), device="cuda:0"):
    """The high-contrast diffusion of workloads.highcontrast3d_7pt (kappa constant per region,
    log-uniform), assembled on the device."""
    import torch
    from . import slab_origins
    rng = np.random.default_rng(seed)
    slabs = tuple(tuple(int(v) for v in rng.choice(np.asarray(choices), size=k))
                  for k in region_grid)
    gdims, rdims, gids = region_map(slabs)
    Nx, Ny, Nz = gdims
    kreg = 10.0 ** rng.uniform(log10_range[0], log10_range[1], size=tuple(region_grid)[::-1])
    kappa = torch.empty((Nz - 1, Ny - 1, Nx - 1), dtype=torch.float64, device=device)
    ox, oy, oz = (slab_origins(s) for s in slabs)
    for c, nz in enumerate(slabs[2]):
        for bb, ny in enumerate(slabs[1]):
            for a, nx in enumerate(slabs[0]):
                kappa[oz[c]:oz[c] + nz - 1, oy[bb]:oy[bb] + ny - 1, ox[a]:ox[a] + nx - 1] = \
                    float(kreg[c, bb, a])
    mask = boundary_mask(gdims)
    rowptr, col, val = _diffusion_csr(gdims, kappa, mask, device)
    del kappa
    b = _rhs_device(rng, Nx * Ny * Nz, mask, device)
    return DeviceWorkload("highcontrast3d_7pt", 3, 1, gdims, slabs, rdims, gids, mask, rowptr,
                          col, val, b, 7, dict(seed=seed, region_grid=tuple(region_grid),
                                               choices=tuple(choices), kappa_region=kreg))
