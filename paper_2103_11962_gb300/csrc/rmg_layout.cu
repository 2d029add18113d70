// Region layout (Psi), non-invasive operator splitting and composite <-> regional maps.
#include <algorithm>
#include <climits>

#include "rmg_kernels.cuh"
#include "rmg_launch.cuh"
#include "rmg_layout.cuh"

namespace rmg {

unsigned long long g_launches = 0;
bool g_capturing = false;

int persistent_grid(const Ctx& c, int work_items, int per_sm) {
  const long cap = (long)c.nsm * per_sm;
  return (int)std::max(1L, std::min<long>(cap, std::max(1, work_items)));
}

void Ctx::check_device_error(const char* where) {
  int h = 0;
  RMG_CUDA(cudaMemcpyAsync(&h, d_err.get(), sizeof(int), cudaMemcpyDeviceToHost, stream));
  RMG_CUDA(cudaStreamSynchronize(stream));
  if (h == 0) return;
  RMG_CUDA(cudaMemsetAsync(d_err.get(), 0, sizeof(int), stream));
  const char* what = "unknown device error";
  rmg_status st = RMG_ERR_LAYOUT;
  switch (h) {
    case DERR_GID_RANGE: what = "a region gid is outside [0, n_composite)"; break;
    case DERR_UNCOVERED: what = "a composite node belongs to no region"; break;
    case DERR_MULT: what = "a composite node has more than 255 regional copies"; break;
    case DERR_STENCIL: what = "a matrix entry couples nodes that are not stencil neighbours "
                              "inside a common region"; break;
    case DERR_COARSE_MISMATCH: what = "co-located nodes disagree on being coarse points "
                                      "(regions do not coarsen conformingly)"; break;
    case DERR_NOT_SPD: what = "coarsest composite operator is not positive definite";
      st = RMG_ERR_SINGULAR; break;
  }
  throw Error(st, std::string(where) + ": " + what);
}

// ------------------------------------------------------------------ scan
namespace {
constexpr int kScanBS = 512;
constexpr int kScanPer = 4;
constexpr int kScanChunk = kScanBS * kScanPer;

__global__ void k_scan_blocks(const int* __restrict__ in, int* __restrict__ out, int n,
                              int* __restrict__ block_sums) {
  __shared__ int sh[kScanBS];
  const int base = blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
  int v[kScanPer];
  int tsum = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    tsum += v[k];
  }
  sh[threadIdx.x] = tsum;
  __syncthreads();
  for (int o = 1; o < kScanBS; o <<= 1) {
    const int t = (threadIdx.x >= o) ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  int run = sh[threadIdx.x] - tsum;   // exclusive prefix of this thread
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanBS - 1) block_sums[blockIdx.x] = sh[kScanBS - 1];
}

__global__ void k_scan_add(int* __restrict__ out, int n, const int* __restrict__ offs) {
  const int base = blockIdx.x * kScanChunk;
  const int add = offs[blockIdx.x];
  for (int k = threadIdx.x; k < kScanChunk; k += blockDim.x)
    if (base + k < n) out[base + k] += add;
}
}  // namespace

static void scan_rec(Ctx& c, const int* in, int* out, int n, int* total_dev) {
  const int nb = (n + kScanChunk - 1) / kScanChunk;
  DBuf<int> bs(nb + 1), bso(nb + 1);
  k_scan_blocks<<<nb, kScanBS, 0, c.stream>>>(in, out, n, bs.get());
  RMG_LAUNCHED();
  if (nb == 1) {
    RMG_CUDA(cudaMemcpyAsync(total_dev, bs.get(), sizeof(int), cudaMemcpyDeviceToDevice,
                             c.stream));
  } else {
    scan_rec(c, bs.get(), bso.get(), nb, total_dev);
    k_scan_add<<<nb, kScanBS, 0, c.stream>>>(out, n, bso.get());
    RMG_LAUNCHED();
  }
  // the temporaries are freed when the stream work that uses them has finished
  RMG_CUDA(cudaStreamSynchronize(c.stream));
}

int exclusive_scan(Ctx& c, const int* in, int* out, int n) {
  if (n == 0) return 0;
  DBuf<int> tot(1);
  scan_rec(c, in, out, n, tot.get());
  int h = 0;
  RMG_CUDA(cudaMemcpy(&h, tot.get(), sizeof(int), cudaMemcpyDeviceToHost));
  return h;
}

// ------------------------------------------------------------------ layout kernels
namespace {
__global__ void k_gids_in(int n_r, const int64_t* __restrict__ g64, int64_t ncomp,
                          int* __restrict__ gid, int* __restrict__ count, int* err) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_r; k += gridDim.x * blockDim.x) {
    const int64_t g = g64[k];
    if (g < 0 || g >= ncomp) { set_err(err, DERR_GID_RANGE); gid[k] = 0; continue; }
    gid[k] = (int)g;
    atomicAdd(&count[g], 1);
  }
}

__global__ void k_node_attrs(int n_r, const int* __restrict__ gid, const int* __restrict__ count,
                             const uint8_t* __restrict__ dir, uint8_t* __restrict__ mult,
                             uint8_t* __restrict__ mask, int* __restrict__ c2r, int* err) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_r; k += gridDim.x * blockDim.x) {
    const int g = gid[k];
    const int m = count[g];
    if (m > 255) set_err(err, DERR_MULT);
    mult[k] = (uint8_t)min(m, 255);
    mask[k] = dir ? (dir[g] ? 1 : 0) : 0;
    atomicMin(&c2r[g], k);
  }
}

__global__ void k_group_flags(int ncomp, const int* __restrict__ count, int* __restrict__ flag,
                              int* __restrict__ scount, int* err) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ncomp; g += gridDim.x * blockDim.x) {
    const int m = count[g];
    if (m == 0) set_err(err, DERR_UNCOVERED);
    flag[g] = m >= 2 ? 1 : 0;
    scount[g] = m >= 2 ? m : 0;
  }
}

__global__ void k_group_index(int ncomp, const int* __restrict__ count,
                              const int* __restrict__ gidx, const int* __restrict__ sstart,
                              int* __restrict__ cgrp, int* __restrict__ gptr, int nslots,
                              int ngroups) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ncomp; g += gridDim.x * blockDim.x) {
    if (count[g] >= 2) {
      cgrp[g] = gidx[g];
      gptr[gidx[g]] = sstart[g];
    } else {
      cgrp[g] = -1;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) gptr[ngroups] = nslots;
}

__global__ void k_group_fill(int n_r, const int* __restrict__ gid, const int* __restrict__ cgrp,
                             const int* __restrict__ gptr, int* __restrict__ fill,
                             int* __restrict__ gslot) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_r; k += gridDim.x * blockDim.x) {
    const int grp = cgrp[gid[k]];
    if (grp < 0) continue;
    const int pos = atomicAdd(&fill[grp], 1);
    gslot[gptr[grp] + pos] = k;
  }
}

// Group of every group slot (the inverse of gptr), for the slot-parallel phase B.
__global__ void k_slot_groups(int ngroups, const int* __restrict__ gptr, int* __restrict__ sgrp) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += gridDim.x * blockDim.x)
    for (int q = gptr[g]; q < gptr[g + 1]; ++q) sgrp[q] = g;
}

__global__ void k_group_sort(int ngroups, const int* __restrict__ gptr, int* __restrict__ gslot) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += gridDim.x * blockDim.x) {
    const int a = gptr[g], e = gptr[g + 1];
    for (int p = a + 1; p < e; ++p) {
      const int v = gslot[p];
      int q = p - 1;
      while (q >= a && gslot[q] > v) { gslot[q + 1] = gslot[q]; --q; }
      gslot[q + 1] = v;
    }
  }
}

__global__ void k_fill_int(int n, int* p, int v) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) p[k] = v;
}

// Candidate affine gid map of every region, gid(i, j, l) = g0 + i + gy j + gz l, read off the
// nodes (1,0,0), (0,1,0) and (0,0,1). It is kept (w = 1) only when the split can invert it by
// comparisons: gy >= 3 and, in 3D, gz >= 2 gy + 3 (see box_offset_affine); 2D regions take
// gz = 2^30, which no column offset reaches.
__global__ void k_affine_init(int nreg, int dim, const RegionDev* __restrict__ regions,
                              const int* __restrict__ gid, int4* __restrict__ aff) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreg; r += gridDim.x * blockDim.x) {
    const RegionDev R = regions[r];
    int4 a = make_int4(0, 0, 0, 0);
    bool ok = R.nx >= 2 && R.ny >= 2 && (dim == 2 ? R.nz == 1 : R.nz >= 2);
    if (ok) {
      a.x = gid[R.off];
      ok = gid[R.off + 1] - a.x == 1;
      a.y = gid[R.off + R.nx] - a.x;
      a.z = dim == 2 ? (1 << 30) : gid[R.off + R.nx * R.ny] - a.x;
      ok = ok && a.y >= 3 && (dim == 2 || (a.z >= 2 * a.y + 3 && a.z < (1 << 29)));
    }
    a.w = ok ? 1 : 0;
    aff[r] = a;
  }
}

// Clears the flag of a region with any node off its candidate map.
__global__ void k_affine_check(Grid G, const int* __restrict__ gid, int4* __restrict__ aff) {
  RMG_FOR_NODES(G)
    const int4 a = aff[tile_.region];
    if (!a.w) continue;
    int i, j, l;
    decode(li, R, i, j, l);
    const long long want = (long long)a.x + i + (long long)a.y * j + (long long)a.z * l;
    if (want != (long long)gid[n]) aff[tile_.region].w = 0;   // every writer stores 0
  RMG_END_FOR_NODES
}
}  // namespace

// Affine gid maps of the regions of a level (Level::affine), for the split's shortcut.
void build_affine(Ctx& c, Level& L) {
  L.affine.alloc(L.nreg);
  k_affine_init<<<persistent_grid(c, (L.nreg + 255) / 256), 256, 0, c.stream>>>(
      L.nreg, L.dim, L.regions.get(), L.gid.get(), L.affine.get());
  RMG_LAUNCHED();
  k_affine_check<<<persistent_grid(c, (int)L.htiles.size()), kTile, 0, c.stream>>>(
      L.grid(), L.gid.get(), L.affine.get());
  RMG_LAUNCHED();
}

void build_tiles(Level& L) {
  L.htiles.clear();
  for (int r = 0; r < L.nreg; ++r) {
    const int sz = L.hdims[3 * r] * L.hdims[3 * r + 1] * L.hdims[3 * r + 2];
    for (int s = 0; s < sz; s += kTile) L.htiles.push_back(Tile{r, s, 0, 0, 0, 0});
  }
  L.tiles.alloc(L.htiles.size());
  RMG_CUDA(cudaMemcpy(L.tiles.get(), L.htiles.data(), L.htiles.size() * sizeof(Tile),
                      cudaMemcpyHostToDevice));
  std::vector<RegionDev> hr(L.nreg);
  for (int r = 0; r < L.nreg; ++r)
    hr[r] = make_region(L.hdims[3 * r], L.hdims[3 * r + 1], L.hdims[3 * r + 2], L.hoff[r]);
  L.regions.alloc(L.nreg);
  RMG_CUDA(cudaMemcpy(L.regions.get(), hr.data(), hr.size() * sizeof(RegionDev),
                      cudaMemcpyHostToDevice));
}

void set_geometry(Level& L, int dim, int nreg, const int* dims) {
  L.dim = dim;
  L.nreg = nreg;
  L.hdims.assign(dims, dims + 3 * nreg);
  L.hoff.assign(nreg + 1, 0);
  long long tot = 0;
  for (int r = 0; r < nreg; ++r) {
    const long long sz = (long long)dims[3 * r] * dims[3 * r + 1] * dims[3 * r + 2];
    L.hoff[r] = (int)tot;
    tot += sz;
    RMG_REQUIRE(tot < INT_MAX, RMG_ERR_ARG, "more than 2^31-1 regional nodes");
  }
  L.hoff[nreg] = (int)tot;
  L.n_r = (int)tot;
  build_tiles(L);
}

// Multiplicities, masks, composite -> regional maps and interface groups of a level whose
// gid array (int) is already on the device. `dir` is a composite-indexed mask or NULL;
// `rmask` (regional) may be given instead.
void build_groups(Ctx& c, Level& L, const uint8_t* dir_comp, const uint8_t* rmask,
                  DBuf<int>& count) {
  const int n_r = L.n_r, nc = L.ncomp;
  const int gb = persistent_grid(c, (n_r + 255) / 256), gc = persistent_grid(c, (nc + 255) / 256);
  L.mult.alloc(n_r);
  L.mask.alloc(n_r);
  L.c2r.alloc(nc);
  k_fill_int<<<gc, 256, 0, c.stream>>>(nc, L.c2r.get(), INT_MAX);
  RMG_LAUNCHED();
  k_node_attrs<<<gb, 256, 0, c.stream>>>(n_r, L.gid.get(), count.get(), dir_comp, L.mult.get(),
                                         L.mask.get(), L.c2r.get(), c.d_err.get());
  RMG_LAUNCHED();
  if (rmask)
    RMG_CUDA(cudaMemcpyAsync(L.mask.get(), rmask, n_r, cudaMemcpyDeviceToDevice, c.stream));
  DBuf<int> flag(nc), scount(nc), gidx(nc), sstart(nc);
  k_group_flags<<<gc, 256, 0, c.stream>>>(nc, count.get(), flag.get(), scount.get(),
                                          c.d_err.get());
  RMG_LAUNCHED();
  L.ngroups = exclusive_scan(c, flag.get(), gidx.get(), nc);
  L.nslots = exclusive_scan(c, scount.get(), sstart.get(), nc);
  L.cgrp.alloc(nc);
  L.gptr.alloc(L.ngroups + 1);
  L.gslot.alloc(std::max(1, L.nslots));
  k_group_index<<<gc, 256, 0, c.stream>>>(nc, count.get(), gidx.get(), sstart.get(),
                                          L.cgrp.get(), L.gptr.get(), L.nslots, L.ngroups);
  RMG_LAUNCHED();
  DBuf<int> fill(std::max(1, L.ngroups));
  RMG_CUDA(cudaMemsetAsync(fill.get(), 0, fill.bytes(), c.stream));
  k_group_fill<<<gb, 256, 0, c.stream>>>(n_r, L.gid.get(), L.cgrp.get(), L.gptr.get(),
                                         fill.get(), L.gslot.get());
  RMG_LAUNCHED();
  if (L.ngroups) {
    k_group_sort<<<persistent_grid(c, (L.ngroups + 255) / 256), 256, 0, c.stream>>>(
        L.ngroups, L.gptr.get(), L.gslot.get());
    RMG_LAUNCHED();
  }
  L.sgrp.alloc(std::max(1, L.nslots));
  if (L.ngroups) {
    k_slot_groups<<<persistent_grid(c, (L.ngroups + 255) / 256), 256, 0, c.stream>>>(
        L.ngroups, L.gptr.get(), L.sgrp.get());
    RMG_LAUNCHED();
  }
  RMG_CUDA(cudaStreamSynchronize(c.stream));
}

void layout_create(Ctx& c, Level& L, int dim, int nreg, const int* dims, const int64_t* g64,
                   int64_t ncomp, const uint8_t* dir) {
  RMG_REQUIRE(dim == 2 || dim == 3, RMG_ERR_ARG, "dim must be 2 or 3");
  RMG_REQUIRE(nreg > 0 && dims && g64, RMG_ERR_ARG, "regions, dims and gids are required");
  RMG_REQUIRE(ncomp > 0 && ncomp < INT_MAX, RMG_ERR_ARG, "n_composite out of range");
  for (int r = 0; r < nreg; ++r) {
    RMG_REQUIRE(dims[3 * r] >= 1 && dims[3 * r + 1] >= 1 && dims[3 * r + 2] >= 1, RMG_ERR_ARG,
                "region dims must be positive");
    if (dim == 2) RMG_REQUIRE(dims[3 * r + 2] == 1, RMG_ERR_ARG, "2D regions need nz = 1");
  }
  set_geometry(L, dim, nreg, dims);
  L.ncomp = (int)ncomp;
  L.gid.alloc(L.n_r);
  DBuf<int> count(L.ncomp);
  RMG_CUDA(cudaMemsetAsync(count.get(), 0, count.bytes(), c.stream));
  k_gids_in<<<persistent_grid(c, (L.n_r + 255) / 256), 256, 0, c.stream>>>(
      L.n_r, g64, ncomp, L.gid.get(), count.get(), c.d_err.get());
  RMG_LAUNCHED();
  build_groups(c, L, dir, nullptr, count);
  build_affine(c, L);
  c.check_device_error("rmg_layout_create");
}

// ------------------------------------------------------------------ splitting (Sec. 4)
namespace {
// Number of regions holding both composite nodes a and b. Group slots are ascending and
// regions occupy ascending slot ranges, so the region ids of a group are ascending too and the
// regions common to the two groups are found by one merge of the two lists.
__device__ __forceinline__ int share_count(int a, int b, const int* __restrict__ rid,
                                           const int* __restrict__ cgrp,
                                           const int* __restrict__ gptr,
                                           const int* __restrict__ gslot) {
  const int ga = cgrp[a], gb = cgrp[b];
  if (ga < 0 || gb < 0) return 1;
  int p = gptr[ga], s = gptr[gb];
  const int pe = gptr[ga + 1], se = gptr[gb + 1];
  int q = 0;
  int ra = rid[gslot[p]], rb = rid[gslot[s]];
  for (;;) {
    if (ra == rb) {
      ++q;
      if (++p == pe || ++s == se) break;
      ra = rid[gslot[p]];
      rb = rid[gslot[s]];
    } else if (ra < rb) {
      if (++p == pe) break;
      ra = rid[gslot[p]];
    } else {
      if (++s == se) break;
      rb = rid[gslot[s]];
    }
  }
  return q;
}

__global__ void k_region_ids(Grid G, int* __restrict__ rid) {
  RMG_FOR_NODES(G)
    rid[n] = tile_.region;
  RMG_END_FOR_NODES
}

// Offset (dx, dy, dz) of regional node n + d from node n of a region with row stride sy and
// plane stride sz, for a neighbour inside the 3x3x3 box: peel the plane and row offsets off d
// by comparison (exact when sy >= 3, since |dx| <= 1 < sy / 2 and |dx + sy dy| < sz / 2).
__device__ __forceinline__ void box_offset(int d, int sy, int sz, int& dx, int& dy, int& dz) {
  dz = 0;
  if (2 * d > sz) { dz = 1; d -= sz; } else if (2 * d < -sz) { dz = -1; d += sz; }
  dy = 0;
  if (2 * d > sy) { dy = 1; d -= sy; } else if (2 * d < -sy) { dy = -1; d += sy; }
  dx = d;
}

// The same for a composite column offset d = c - g = dx + gy dy + gz dz of an affine region
// (gy >= 3, gz >= 2 gy + 3). d comes from an unchecked column, so the comparisons halve the
// strides instead of doubling d (2 d > s <=> d > floor(s / 2) for integers), and dx is clamped
// to [-2, 2]: an offset outside the 3x3x3 box comes out with |dx| > 1 or lands on the wrong
// node, which the caller rules out (affine_holds).
__device__ __forceinline__ void box_offset_affine(int d, int gy, int gz, int& dx, int& dy,
                                                  int& dz) {
  dz = 0;
  if (d > (gz >> 1)) { dz = 1; d -= gz; } else if (-d > (gz >> 1)) { dz = -1; d += gz; }
  dy = 0;
  if (d > (gy >> 1)) { dy = 1; d -= gy; } else if (-d > (gy >> 1)) { dy = -1; d += gy; }
  dx = d > 2 ? 2 : (d < -2 ? -2 : d);
}

// Whether composite node c (0 <= c < 2^31) is a node of affine region R (a: its map).
__device__ __forceinline__ bool affine_holds(int c, const int4& a, const RegionDev& R) {
  const int rel = c - a.x;                     // a.x >= 0: no overflow
  if (rel < 0) return false;
  const int l = rel / a.z, rem = rel - l * a.z, j = rem / a.y, i = rem - j * a.y;
  return l < R.nz && j < R.ny && i < R.nx;
}

// The split of one CSR row: regional node n of region R (local index li), row component c_row.
// Every entry is handled in the row's order and goes straight into its coefficient stream
// coef[((c * B + c') * S + slot) * n_r + n]. For the diagonal slot's nullspace rule a shared
// row collects the whole row (zsum = A 1 at the node) and the split off-diagonal values
// (offsum); a single-copy row, where the two sums would cancel in every in-region coupling,
// collects only its diagonal entry and its couplings to other regions. At the end a slot that
// received no entry is zeroed; a repeated column (not produced by a well-formed CSR) is
// accumulated.
template <int KIND, int B>
struct RowSplit {
  using S = Sten<KIND>;
  RegionDev R;
  int n, i, j, l, g, nodes, n_r;
  bool shared, affine_map, peel;
  int4 af;
  double zsum[B], offsum[B];
  unsigned seen[B];                            // slots already written (27 < 32 bits)
  double* cbase;

  __device__ __forceinline__ void begin(int n_, int li, int region, const RegionDev& R_,
                                        int c_row, int n_r_, const int* __restrict__ gid,
                                        const uint8_t* __restrict__ mult,
                                        const int4* __restrict__ affine, double* coef) {
    R = R_;
    n = n_;
    n_r = n_r_;
    decode(li, R, i, j, l);
    nodes = R.nx * R.ny * R.nz;
    peel = R.nx >= 3 && R.ny >= 3;             // box_offset is exact
    g = gid[n];
    shared = mult[n] > 1;
    // rows of a region whose gid map is affine (k_affine_*) find the slot of every entry from
    // c - g alone, without the composite-indexed gathers (a shared row still counts the regions
    // that hold both ends of each coupling, share_count)
    af = affine[region];
    affine_map = af.w != 0;
#pragma unroll
    for (int b = 0; b < B; ++b) { zsum[b] = 0.0; offsum[b] = 0.0; seen[b] = 0u; }
    cbase = coef + (size_t)c_row * B * S::S * n_r + n;
  }

  // Composite node of a column (its component in cp), or -1 for an id out of range (flagged).
  __device__ __forceinline__ int node_of(int64_t c64, int ncomp, int* err, int& cp) const {
    cp = 0;
    if (c64 < 0 || c64 >= (int64_t)ncomp * B) { set_err(err, DERR_GID_RANGE); return -1; }
    int c = (int)c64;
    if (B > 1) {                                 // compile-time divisor: multiply-shift
      c = (int)(c64 / B);
      cp = (int)(c64 - (int64_t)c * B);
    }
    return c;
  }

  // Whether entry c needs its interface group (the general path's first gather).
  __device__ __forceinline__ bool needs_group(int c) const { return c != g && !affine_map; }

  // One entry, in row order; grp = cgrp[c] when needs_group(c).
  __device__ __forceinline__ void apply(int c, int b, double v, int grp,
                                        const int* __restrict__ c2r,
                                        const int* __restrict__ cgrp,
                                        const int* __restrict__ gptr,
                                        const int* __restrict__ gslot,
                                        const int* __restrict__ rid, int* err) {
    // the row component b of the entry is a run-time index: select it with an unrolled loop
    // so that the per-component sums stay in registers. A shared row sums every entry (A 1);
    // a single-copy row only the entries that do not land off the diagonal of its region
    // (see end())
#pragma unroll
    for (int k = 0; k < B; ++k)
      if (k == b && (shared || c == g)) zsum[k] += v;
    if (c == g) return;
    int dx, dy, dz;
    if (affine_map) {
      // c = g + dx + gy dy + gz dz inside the 3x3x3 box: when that position lies in the
      // region, c is the node there (the map is affine over the region). Any other column is
      // a node of this region (outside the stencil: the error below, as on the general path)
      // or of other regions only (skipped, as there).
      box_offset_affine(c - g, af.y, af.z, dx, dy, dz);
      const bool in_region = dx >= -1 && dx <= 1 && i + dx >= 0 && i + dx < R.nx &&
                             j + dy >= 0 && j + dy < R.ny && l + dz >= 0 && l + dz < R.nz;
      if (!in_region) {
        if (affine_holds(c, af, R)) set_err(err, DERR_STENCIL);
        else add_outside(b, v);
        return;
      }
    } else {
      // regional slot of c inside this region
      int sc = -1;
      if (grp < 0) {
        const int s0 = c2r[c];
        sc = (s0 >= R.off && s0 < R.off + nodes) ? s0 : -1;
      } else {
        for (int q = gptr[grp]; q < gptr[grp + 1]; ++q) {
          const int s0 = gslot[q];
          if (s0 >= R.off && s0 < R.off + nodes) { sc = s0; break; }
        }
      }
      if (sc < 0) {                              // entry belongs to other regions only
        add_outside(b, v);
        return;
      }
      if (peel) {
        box_offset(sc - n, R.nx, R.nx * R.ny, dx, dy, dz);
      } else {
        int ic, jc, lc;
        decode(sc - R.off, R, ic, jc, lc);
        dx = ic - i; dy = jc - j; dz = lc - l;
      }
    }
    const bool inside = dx >= -1 && dx <= 1 && i + dx >= 0 && i + dx < R.nx &&
                        j + dy >= 0 && j + dy < R.ny && l + dz >= 0 && l + dz < R.nz;
    const int slot = inside ? sten_slot<KIND>(dx, dy, dz) : -1;
    if (slot < 0) { set_err(err, DERR_STENCIL); return; }
    const int q = shared ? share_count(g, c, rid, cgrp, gptr, gslot) : 1;
    const double vs = q == 1 ? v : v * inv_mult<double>(q);
    double* dst = cbase + ((size_t)b * S::S + slot) * n_r;
    const unsigned bit = 1u << slot;
    bool again = false;
#pragma unroll
    for (int k = 0; k < B; ++k)
      if (k == b) {
        if (shared) offsum[k] += vs;
        again = (seen[k] & bit) != 0;
        seen[k] |= bit;
      }
    if (again) *dst += vs; else *dst = vs;
  }

  // An entry of a single-copy row that couples to other regions only keeps its place in the
  // row sum of the nullspace rule.
  __device__ __forceinline__ void add_outside(int b, double v) {
#pragma unroll
    for (int k = 0; k < B; ++k)
      if (k == b && !shared) zsum[k] += v;
  }

  __device__ __forceinline__ void end(const uint8_t* __restrict__ mult) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      double* cb = cbase + (size_t)b * S::S * n_r;
#pragma unroll
      for (int s = 0; s < S::S; ++s)
        if (s != S::CENTER && !((seen[b] >> s) & 1u)) cb[(size_t)s * n_r] = 0.0;
      // the nullspace rule z_i / mult_i - (split off-diagonal sum); with a single copy every
      // off-diagonal entry in the region enters both terms whole, so the rule is the diagonal
      // entry plus the entries coupling to other regions, formed without that cancellation
      cb[(size_t)S::CENTER * n_r] =
          shared ? zsum[b] * inv_mult<double>(mult[n]) - offsum[b] : zsum[b];
    }
  }
};

#define RMG_SPLIT_PARAMS                                                                  \
  const int* __restrict__ gid, const uint8_t* __restrict__ mult,                          \
      const int* __restrict__ c2r, const int* __restrict__ cgrp,                          \
      const int* __restrict__ gptr, const int* __restrict__ gslot,                        \
      const int* __restrict__ rid, const int4* __restrict__ affine,                       \
      const int64_t* __restrict__ rowptr, const int64_t* __restrict__ col,                \
      const double* __restrict__ val, int ncomp, double* __restrict__ coef, int* err

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// Entries of a row staged per pass: 27 = 3 x 9 (a shared row stride of 9 words of 8 bytes
// keeps the lanes' reads of their own rows free of bank conflicts).
constexpr int kSplitChunk = 9;

// Single-copy rows (the rows of shared nodes are left to k_split_shared, so that a warp of
// single-copy rows does not wait on the longer path of the interface rows among them). A warp
// takes 32 consecutive nodes of a tile. Their CSR rows are staged through shared memory nine
// entries at a time, the lanes copying the 32 rows' entries together (the rows of consecutive
// nodes lie side by side in the CSR, so each pass reads whole sectors once); then every lane
// handles its own row's entries in order.
template <int KIND, int B>
__global__ void __launch_bounds__(kTile)
k_split_csr(Grid G, RMG_SPLIT_PARAMS) {
  constexpr int kWarps = kTile / 32;
  __shared__ __align__(16) int64_t s_col[kWarps][32 * kSplitChunk];
  __shared__ __align__(16) double s_val[kWarps][32 * kSplitChunk];
  __shared__ int64_t s_e0[kWarps][32];           // first entry and length of every lane's row
  __shared__ int s_len[kWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t* wc = s_col[warp];
  double* wv = s_val[warp];
  const int c_row = blockIdx.y;
  const int tasks = G.ntiles * kWarps;
  for (int task = blockIdx.x * kWarps + warp; task < tasks; task += gridDim.x * kWarps) {
    const Tile tile = G.tiles[task / kWarps];
    const RegionDev R = G.regions[tile.region];
    const int li = tile.start + (task % kWarps) * 32 + lane;
    const int n = R.off + li;
    const bool active = li < R.nx * R.ny * R.nz && mult[n] == 1;
    RowSplit<KIND, B> rs;
    int64_t e0 = 0;
    int len = 0;
    if (active) {
      rs.begin(n, li, tile.region, R, c_row, G.n_r, gid, mult, affine, coef);
      const int64_t row = (int64_t)rs.g * B + c_row;
      e0 = rowptr[row];
      len = (int)(rowptr[row + 1] - e0);
    }
    s_e0[warp][lane] = e0;
    s_len[warp][lane] = len;
    __syncwarp();
    const int passes = ((int)__reduce_max_sync(0xffffffffu, (unsigned)len) + kSplitChunk - 1) /
                       kSplitChunk;
    for (int h = 0; h < passes; ++h) {
      // entry h * 9 + k of the row of lane r goes to w*[r * 9 + k]
#pragma unroll 3
      for (int m = 0; m < kSplitChunk; ++m) {
        const int idx = lane + 32 * m;
        const int r = idx / kSplitChunk, k = idx - r * kSplitChunk;
        const int e = h * kSplitChunk + k;
        if (e < s_len[warp][r]) {
          const int64_t at = s_e0[warp][r] + e;
          cp_async8(wc + idx, col + at);
          cp_async8(wv + idx, val + at);
        }
      }
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      __syncwarp();
      if (active) {
        const int kn = min(kSplitChunk, len - h * kSplitChunk);
        for (int k = 0; k < kn; ++k) {
          int cp;
          const int c = rs.node_of(wc[lane * kSplitChunk + k], ncomp, err, cp);
          if (c < 0) continue;
          const int grp = rs.needs_group(c) ? cgrp[c] : -2;
          rs.apply(c, cp, wv[lane * kSplitChunk + k], grp, c2r, cgrp, gptr, gslot, rid, err);
        }
      }
      __syncwarp();                              // before the next pass overwrites the rows
    }
    if (active) rs.end(mult);
  }
}

// Rows of shared nodes, one thread per regional copy, in group-slot order (the copies of one
// composite node are neighbours, so their common CSR row is read once into L1). The entries
// go in batches: the column, value and group loads of a batch are issued together (they do not
// depend on each other), then the entries are applied in order.
#ifndef RMG_SPLIT_BATCH
#define RMG_SPLIT_BATCH 4
#endif
template <int KIND, int B>
__global__ void __launch_bounds__(kTile)
k_split_shared(int nslots, const RegionDev* __restrict__ regions, int n_r, RMG_SPLIT_PARAMS) {
  const int c_row = blockIdx.y;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nslots; q += gridDim.x * blockDim.x) {
    const int n = gslot[q];
    const int r = rid[n];
    const RegionDev R = regions[r];
    RowSplit<KIND, B> rs;
    rs.begin(n, n - R.off, r, R, c_row, n_r, gid, mult, affine, coef);
    const int64_t row = (int64_t)rs.g * B + c_row;
    const int64_t e0 = rowptr[row], e1 = rowptr[row + 1];
    constexpr int U = RMG_SPLIT_BATCH;
    for (int64_t eb = e0; eb < e1; eb += U) {
      int cn[U], cp[U], grp[U];
      double vv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool in = eb + u < e1;
        const int64_t c64 = in ? col[eb + u] : 0;
        vv[u] = in ? val[eb + u] : 0.0;
        cn[u] = in ? rs.node_of(c64, ncomp, err, cp[u]) : -1;
        if (!in) cp[u] = 0;
        grp[u] = (cn[u] >= 0 && rs.needs_group(cn[u])) ? cgrp[cn[u]] : -2;
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (cn[u] >= 0) rs.apply(cn[u], cp[u], vv[u], grp[u], c2r, cgrp, gptr, gslot, rid, err);
    }
    rs.end(mult);
  }
}
#undef RMG_SPLIT_PARAMS

// Composite vectors with B dofs per node are node-major (dof g*B + c); regional vectors are
// component-major (c * n_r + n).
__global__ void k_comp_to_reg(int n_r, int B, const int* __restrict__ gid,
                              const uint8_t* __restrict__ mask, const double* __restrict__ c,
                              double* __restrict__ r) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_r; k += gridDim.x * blockDim.x)
    for (int b = 0; b < B; ++b)
      r[(size_t)b * n_r + k] = (mask && mask[k]) ? 0.0 : c[(size_t)gid[k] * B + b];
}

__global__ void k_reg_to_comp(int ncomp, int n_r, int B, const int* __restrict__ c2r,
                              const int* __restrict__ cgrp, const int* __restrict__ gptr,
                              const int* __restrict__ gslot, const double* __restrict__ r,
                              double* __restrict__ c, int average) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ncomp; g += gridDim.x * blockDim.x) {
    const int grp = cgrp[g];
    for (int b = 0; b < B; ++b) {
      const double* rb = r + (size_t)b * n_r;
      if (grp < 0) { c[(size_t)g * B + b] = rb[c2r[g]]; continue; }
      double s = 0.0;
      const int a = gptr[grp], e = gptr[grp + 1];
      for (int q = a; q < e; ++q) s += rb[gslot[q]];
      c[(size_t)g * B + b] = average ? s / (double)(e - a) : s;
    }
  }
}
}  // namespace

void split_from_csr(Ctx& c, Level& L, int kind, int B, const int64_t* rowptr, const int64_t* col,
                    const double* val) {
  RMG_REQUIRE(rowptr && col && val, RMG_ERR_ARG, "CSR arrays are required");
  RMG_REQUIRE((L.dim == 2 && (kind == 5 || kind == 9)) || (L.dim == 3 && (kind == 7 || kind == 27)),
              RMG_ERR_ARG, "stencil must be 5/9 in 2D and 7/27 in 3D");
  RMG_REQUIRE(B == 1 || (B == 3 && (kind == 27 || kind == 9)), RMG_ERR_ARG,
              "block operators need 3 dofs per node and a 27- or 9-point stencil");
  L.kind = kind;
  L.B = B;
  L.coef.ensure((size_t)B * B * kind * L.n_r);
  const Grid G = L.grid();
  if (!L.rid.get()) {
    L.rid.alloc(L.n_r);
    k_region_ids<<<persistent_grid(c, G.ntiles), kTile, 0, c.stream>>>(G, L.rid.get());
    RMG_LAUNCHED();
  }
  if (L.affine.n < (size_t)L.nreg) build_affine(c, L);
  // single-copy rows over the tiles, then the rows of shared nodes over the group slots; both
  // grids are one resident wave
#define RMG_SPLIT_ARGS                                                                     \
  L.gid.get(), L.mult.get(), L.c2r.get(), L.cgrp.get(), L.gptr.get(), L.gslot.get(),        \
      L.rid.get(), L.affine.get(), rowptr, col, val, L.ncomp, L.coef.get(), c.d_err.get()
#define RMG_SPLIT(K, BB)                                                                    \
  do {                                                                                      \
    const dim3 gb(persistent_grid(c, G.ntiles, resident_per_sm((const void*)k_split_csr<K, BB>)), \
                  B);                                                                       \
    k_split_csr<K, BB><<<gb, kTile, 0, c.stream>>>(G, RMG_SPLIT_ARGS);                      \
    if (L.nslots) {                                                                         \
      const dim3 gs(persistent_grid(c, (L.nslots + kTile - 1) / kTile,                      \
                                    resident_per_sm((const void*)k_split_shared<K, BB>)),   \
                    B);                                                                     \
      k_split_shared<K, BB><<<gs, kTile, 0, c.stream>>>(L.nslots, L.regions.get(), L.n_r,   \
                                                        RMG_SPLIT_ARGS);                    \
    }                                                                                       \
  } while (0)
  switch (kind) {
    case 5: RMG_SPLIT(5, 1); break;
    case 7: RMG_SPLIT(7, 1); break;
    case 9: if (B == 3) RMG_SPLIT(9, 3); else RMG_SPLIT(9, 1); break;
    default: if (B == 3) RMG_SPLIT(27, 3); else RMG_SPLIT(27, 1); break;
  }
#undef RMG_SPLIT
#undef RMG_SPLIT_ARGS
  RMG_LAUNCHED();
  c.check_device_error("rmg_operator_from_csr");
}

void comp_to_reg(Ctx& c, const Level& L, const double* comp, double* reg, bool zero_masked) {
  const int gb = persistent_grid(c, (L.n_r + 255) / 256);
  k_comp_to_reg<<<gb, 256, 0, c.stream>>>(L.n_r, L.B, L.gid.get(),
                                          zero_masked ? L.mask.get() : nullptr, comp, reg);
  RMG_LAUNCHED();
}

void reg_to_comp(Ctx& c, const Level& L, const double* reg, double* comp, int average) {
  k_reg_to_comp<<<persistent_grid(c, (L.ncomp + 255) / 256), 256, 0, c.stream>>>(
      L.ncomp, L.n_r, L.B, L.c2r.get(), L.cgrp.get(), L.gptr.get(), L.gslot.get(), reg, comp,
      average);
  RMG_LAUNCHED();
}

// y = Psi^T Psi [[A]] u in FP64 with the level's FP64 coefficients.
void regional_apply(Ctx& c, const Level& L, const double* u, double* y, double* ypart) {
  launch_stencil(c, L, L.coef.get(), u, ypart, EpiStore<double>{y}, c.stream, nullptr);
}

}  // namespace rmg
