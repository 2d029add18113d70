// Device kernels of the regional V-cycle and its setup.
//
// Every node-parallel kernel is a persistent grid-stride loop over a tile list that covers
// all regions of a level (one launch batches all regions, whatever their sizes). A tile is a
// run of up to kTile consecutive nodes of one region, or, for the stencil sweeps, a box of
// kTile nodes whose shape the hierarchy picks by timing (autotuned); blockDim.x == kTile.
//
// The interface summation Psi^T Psi (Sec. 3.1) is split in two phases. Phase A applies the
// region stencil at every node; a node with a single copy finishes its update at once, a
// node shared by several regions stores its partial row result y[n]. Phase B runs over the
// interface groups (the copies of one shared composite node), sums the partial results in
// ascending slot order and applies the same epilogue to every copy, so the copies stay
// identical ("consistent").
#pragma once

#include "rmg_internal.cuh"

namespace rmg {

// a / d for 0 <= a < 2^22 from the float reciprocal rd of d: the truncated product is within
// one of the quotient (relative error below 2^-22 on a value below 2^22), and one correction
// step makes it exact.
__device__ __forceinline__ int div_rcp(int a, int d, float rd) {
  int q = __float2int_rz(__int2float_rn(a) * rd);
  const int r = a - q * d;
  q += (r >= d) - (r < 0);
  return q;
}

__device__ __forceinline__ void decode(int li, const RegionDev& R, int& i, int& j, int& l) {
  if (R.rnx != 0.0f) {
    const int rest = div_rcp(li, R.nx, R.rnx);
    i = li - rest * R.nx;
    l = div_rcp(rest, R.ny, R.rny);
    j = rest - l * R.ny;
  } else {
    i = li % R.nx;
    const int rest = li / R.nx;
    j = rest % R.ny;
    l = rest / R.ny;
  }
}

__device__ __forceinline__ void set_err(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// Region containing regional node n (binary search over region offsets).
__device__ __forceinline__ int region_of(const RegionDev* R, int nreg, int n) {
  int lo = 0, hi = nreg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (R[mid].off <= n) lo = mid; else hi = mid - 1;
  }
  return lo;
}

#define RMG_FOR_NODES(G)                                                       \
  for (int t_ = blockIdx.x; t_ < (G).ntiles; t_ += gridDim.x) {                \
    const Tile tile_ = (G).tiles[t_];                                          \
    const RegionDev R = (G).regions[tile_.region];                             \
    int li, bi_ = -1, bj_ = 0, bl_ = 0;                                        \
    if ((G).lx < 0) {                                                          \
      li = tile_.start + (int)threadIdx.x;                                     \
      if (li >= R.nx * R.ny * R.nz) continue;                                  \
    } else {                                                                   \
      bi_ = tile_.x0 + ((int)threadIdx.x & ((1 << (G).lx) - 1));               \
      bj_ = tile_.y0 + (((int)threadIdx.x >> (G).lx) & ((1 << (G).ly) - 1));   \
      bl_ = tile_.z0 + ((int)threadIdx.x >> ((G).lx + (G).ly));                \
      if (bi_ >= R.nx || bj_ >= R.ny || bl_ >= R.nz) continue;                 \
      li = bi_ + R.nx * (bj_ + R.ny * bl_);                                    \
    }                                                                          \
    const int n = R.off + li;

// (i, j, l) of the current node inside RMG_FOR_NODES: from the box in box mode, else decoded.
#define RMG_DECODE(i, j, l)                                                    \
  if (bi_ >= 0) { i = bi_; j = bj_; l = bl_; } else decode(li, R, i, j, l);

#define RMG_END_FOR_NODES }

// ------------------------------------------------------------------ stencil application
// au = sum_s coef[s][n] * u[n + off(s)] over the neighbours inside the region.
template <int KIND, typename CT, typename VT, typename AT>
__device__ __forceinline__ AT stencil_row(const CT* __restrict__ coef, const VT* __restrict__ u,
                                          int n, int n_r, int i, int j, int l,
                                          const RegionDev& R) {
  using S = Sten<KIND>;
  AT au = AT(0);
  const int sx = 1, sy = R.nx, sz = R.nx * R.ny;
#pragma unroll
  for (int s = 0; s < S::S; ++s) {
    const int dx = S::dx(s), dy = S::dy(s), dz = S::dz(s);
    bool ok = true;
    if (dx < 0) ok &= (i > 0);
    if (dx > 0) ok &= (i < R.nx - 1);
    if (dy < 0) ok &= (j > 0);
    if (dy > 0) ok &= (j < R.ny - 1);
    if (dz < 0) ok &= (l > 0);
    if (dz > 0) ok &= (l < R.nz - 1);
    if (ok) {
      const AT c = AT(coef[(size_t)s * (size_t)n_r + n]);
      const AT v = AT(u[n + dx * sx + dy * sy + dz * sz]);
      au = fma(c, v, au);
    }
  }
  return au;
}

template <typename T> __device__ __forceinline__ T to_acc(T v) { return v; }

// Phase A: stencil at every node; single-copy nodes finish through the epilogue.
template <int KIND, typename CT, typename VT, typename AT, class Epi>
__global__ void __launch_bounds__(kTile)
k_stencil(Grid G, const CT* __restrict__ coef, const VT* __restrict__ u,
          const uint8_t* __restrict__ mult, AT* __restrict__ y, Epi epi) {
  RMG_FOR_NODES(G)
    int i, j, l;
    RMG_DECODE(i, j, l);
    const AT au = stencil_row<KIND, CT, VT, AT>(coef, u, n, G.n_r, i, j, l, R);
    if (mult[n] > 1) y[n] = au; else epi(n, au, 1);
  RMG_END_FOR_NODES
}

// ---- half storage of a symmetric FP32 stencil ----------------------------------------------
// In every stencil kind slot S-1-s is the mirror offset of slot s and the centre is slot
// C = (S-1)/2. A symmetric regional operator has a(n, n+e) = a(n+e, n), so planes C..S-1 hold
// it all: half plane p is slot C+p at every node, and slot s < C of node n is half plane
// S-1-s-C at the neighbour n + off(s). stencil_row_half forms the same products in the same
// order as stencil_row, so its row is bit for bit the full form's whenever the mirrored pairs
// are bitwise equal.
template <int KIND>
__host__ __device__ constexpr bool mirrored_slots() {
  using S = Sten<KIND>;
  if (2 * S::CENTER + 1 != S::S) return false;
  for (int s = 0; s < S::S; ++s)
    if (S::dx(S::S - 1 - s) != -S::dx(s) || S::dy(S::S - 1 - s) != -S::dy(s) ||
        S::dz(S::S - 1 - s) != -S::dz(s))
      return false;
  return true;
}

template <int KIND>
__device__ __forceinline__ float stencil_row_half(const float* __restrict__ half,
                                                  const float* __restrict__ u, int n, int n_r,
                                                  int i, int j, int l, const RegionDev& R) {
  using S = Sten<KIND>;
  static_assert(mirrored_slots<KIND>(), "half storage needs mirrored stencil slots");
  constexpr int C = S::CENTER;
  const int sy = R.nx, sz = R.nx * R.ny;
  float au = 0.f;
#pragma unroll
  for (int s = 0; s < S::S; ++s) {
    const int dx = S::dx(s), dy = S::dy(s), dz = S::dz(s);
    bool ok = true;
    if (dx < 0) ok &= (i > 0);
    if (dx > 0) ok &= (i < R.nx - 1);
    if (dy < 0) ok &= (j > 0);
    if (dy > 0) ok &= (j < R.ny - 1);
    if (dz < 0) ok &= (l > 0);
    if (dz > 0) ok &= (l < R.nz - 1);
    if (ok) {
      const int nb = n + dx + dy * sy + dz * sz;
      const float c = s < C ? half[(size_t)(S::S - 1 - s - C) * (size_t)n_r + nb]
                            : half[(size_t)(s - C) * (size_t)n_r + n];
      au = fmaf(c, u[nb], au);
    }
  }
  return au;
}

// Phase A of the FP32 cycle on a level with half planes: the half form when the pack found the
// operator symmetric (*asym == 0), else the full planes as k_stencil.
template <bool HALF, int KIND, class Epi>
__device__ __forceinline__ void stencil_pass(const Grid& G, const float* __restrict__ coef,
                                             const float* __restrict__ u,
                                             const uint8_t* __restrict__ mult,
                                             float* __restrict__ y, const Epi& epi) {
  RMG_FOR_NODES(G)
    int i, j, l;
    RMG_DECODE(i, j, l);
    const float au = HALF ? stencil_row_half<KIND>(coef, u, n, G.n_r, i, j, l, R)
                          : stencil_row<KIND, float, float, float>(coef, u, n, G.n_r, i, j, l, R);
    if (mult[n] > 1) y[n] = au; else epi(n, au, 1);
  RMG_END_FOR_NODES
}

template <int KIND, class Epi>
__global__ void __launch_bounds__(kTile)
k_stencil_half(Grid G, const float* __restrict__ coef, const float* __restrict__ half,
               const int* __restrict__ asym, const float* __restrict__ u,
               const uint8_t* __restrict__ mult, float* __restrict__ y, Epi epi) {
  if (*asym) stencil_pass<false, KIND>(G, coef, u, mult, y, epi);
  else stencil_pass<true, KIND>(G, half, u, mult, y, epi);
}

// ---- staged 27-point half-plane sweep: region tiles in shared memory, pipelined ----------
// A block owns a kStX x kStY tile of the x-y planes of one region (tiles[t] = {region, -, x0,
// y0}) and steps through all z-planes of the region. For plane l it needs u of planes l-1..l+1
// and the 14 half planes of planes l-1 and l (the own coefficients of plane l; the mirrored
// coefficients of the in-plane neighbours, half planes 1..4, and of the neighbours below, half
// planes 5..13), each with a one-node ring around the tile. Every row of such a window (34
// nodes) is copied from global to shared memory with 16-byte cp.async, starting at the 16-byte
// boundary at or below the row's first node, into 40-float shared rows; a row's nodes start
// at the offset m = (element index of its first node) mod 4 of that row. Region rows need not
// be aligned: only the array bases must be (checked at launch). While the block computes plane
// l, the copies of the coefficients of planes up to l + kStAhead and of u up to l + 1 +
// kStAhead are in flight. Each node forms the products of stencil_row_half in the same slot
// order, so its row is bit for bit that of the other shapes.
#ifndef RMG_ST_AHEAD
#define RMG_ST_AHEAD 1
#endif
constexpr int kStX = 32, kStY = 8;
constexpr int kStRows = kStY + 2, kStRow = 40;           // window rows with the ring; floats
constexpr int kStPlane = kStRows * kStRow;               // one staged plane
constexpr int kStAhead = RMG_ST_AHEAD;                   // planes copied ahead of use
constexpr int kStCoef = kStAhead + 2, kStU = kStAhead + 3;   // ring depths
constexpr int kStSmemFloats = (kStCoef * 14 + kStU) * kStPlane;

__device__ __forceinline__ void cp_async16(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copy the windows of planes [0, np) of `src` (plane stride n_r, src 16-byte aligned, `total`
// floats long) at z-plane l of region R, tile corner (x0, y0), into dst[p][row][0..40). Only
// 16-byte chunks that hold a node of the region are copied; a chunk that would end past the
// array goes element by element. Other shared words keep stale values and are never read.
__device__ __forceinline__ void stage_windows(float* dst, const float* __restrict__ src, int np,
                                              long long n_r, long long total,
                                              const RegionDev& R, int x0, int y0, int l) {
  constexpr int kChunks = kStRow / 4;
  const int chunks = np * kStRows * kChunks;
  const int lo_cx = x0 == 0 ? 1 : 0, hi_cx = min(kStX + 1, R.nx - x0);
  for (int e = threadIdx.x; e < chunks; e += blockDim.x) {
    const int p = e / (kStRows * kChunks), rem = e - p * (kStRows * kChunks);
    const int row = rem / kChunks, k = rem - row * kChunks;
    const int j = y0 + row - 1;
    if (j < 0 || j >= R.ny) continue;
    const long long gs = (long long)p * n_r + R.off +
                         (long long)R.nx * (j + (long long)R.ny * l) + x0 - 1;   // node cx = 0
    const long long c = (gs & ~3LL) + 4 * k;
    if (c + 3 < gs + lo_cx || c > gs + hi_cx) continue;
    float* d = dst + p * kStPlane + row * kStRow + 4 * k;
    if (c + 4 <= total) {
      cp_async16(d, src + c);
    } else {
      for (int q = 0; q < 4 && c + q < total; ++q) cp_async4(d + q, src + c + q);
    }
  }
}

template <class Epi>
__global__ void __launch_bounds__(kStX * kStY)
k_stencil_half27_staged(Grid G, const float* __restrict__ coef, const float* __restrict__ half,
                        const int* __restrict__ asym, const float* __restrict__ u,
                        const uint8_t* __restrict__ mult, float* __restrict__ y, Epi epi) {
  extern __shared__ __align__(16) float st_smem[];
  float* CS = st_smem;                                // [kStCoef][14][kStPlane]
  float* US = st_smem + kStCoef * 14 * kStPlane;      // [kStU][kStPlane]
  const int tx = threadIdx.x % kStX, ty = threadIdx.x / kStX;
  const bool full = *asym != 0;
  const long long n_r = G.n_r;
  const unsigned nr3 = (unsigned)G.n_r & 3u;
  for (int t = blockIdx.x; t < G.ntiles; t += gridDim.x) {
    const Tile tile = G.tiles[t];
    const RegionDev R = G.regions[tile.region];
    const int x0 = tile.x0, y0 = tile.y0;
    const int i = x0 + tx, j = y0 + ty;
    const bool in = i < R.nx && j < R.ny;
    if (full) {                                       // asymmetric operator: full planes
      for (int l = 0; l < R.nz && in; ++l) {
        const int n = R.off + i + R.nx * (j + R.ny * l);
        const float au = stencil_row<27, float, float, float>(coef, u, n, G.n_r, i, j, l, R);
        if (mult[n] > 1) y[n] = au; else epi(n, au, 1);
      }
      continue;
    }
    // prologue: u planes 0 .. kStAhead and the coefficients of planes 0 .. kStAhead - 1, one
    // group per plane (u plane 0 joins the first)
    for (int q = 0; q < kStAhead; ++q) {
      if (q == 0) stage_windows(US, u, 1, n_r, n_r, R, x0, y0, 0);
      if (q + 1 < R.nz)
        stage_windows(US + ((q + 1) % kStU) * kStPlane, u, 1, n_r, n_r, R, x0, y0, q + 1);
      if (q < R.nz)
        stage_windows(CS + (q % kStCoef) * 14 * kStPlane, half, 14, n_r, 14 * n_r, R, x0, y0, q);
      cp_async_commit();
    }
    // m of window row ty + ri at z-plane z: (off + x0 - 1 + nx (y0 - 1 + ty + ri + ny z)) mod 4;
    // half plane q adds q n_r
    const unsigned cst = (unsigned)(R.off + x0 - 1) + (unsigned)R.nx * (unsigned)(y0 - 1 + ty);
    const bool xm = i > 0, xp = i < R.nx - 1, ym = j > 0, yp = j < R.ny - 1;
    for (int l = 0; l < R.nz; ++l) {
      // copies for later planes: coefficients of l + kStAhead, u of l + 1 + kStAhead
      const int lc = l + kStAhead, lu = l + 1 + kStAhead;
      if (lc < R.nz)
        stage_windows(CS + (lc % kStCoef) * 14 * kStPlane, half, 14, n_r, 14 * n_r, R, x0, y0, lc);
      if (lu < R.nz) stage_windows(US + (lu % kStU) * kStPlane, u, 1, n_r, n_r, R, x0, y0, lu);
      cp_async_commit();
      cp_async_wait<kStAhead>();                      // the groups of planes <= l have landed
      __syncthreads();
      if (in) {
        const bool zm = l > 0, zp = l < R.nz - 1;
        const float* Cc = CS + (l % kStCoef) * 14 * kStPlane;                    // plane l
        const float* Cp = CS + ((l + kStCoef - 1) % kStCoef) * 14 * kStPlane;    // plane l - 1
        const float* Uz[3] = {US + ((l + kStU - 1) % kStU) * kStPlane, US + (l % kStU) * kStPlane,
                              US + ((l + 1) % kStU) * kStPlane};
        unsigned m[3][3];                              // [z-plane l-1..l+1][window row ty..ty+2]
#pragma unroll
        for (int zi = 0; zi < 3; ++zi)
#pragma unroll
          for (int ri = 0; ri < 3; ++ri)
            m[zi][ri] = (cst + (unsigned)R.nx * (unsigned)(ri + R.ny * (l - 1 + zi))) & 3u;
        float au = 0.f;
#pragma unroll
        for (int s = 0; s < 27; ++s) {
          const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
          bool ok = true;
          if (dx < 0) ok &= xm;
          if (dx > 0) ok &= xp;
          if (dy < 0) ok &= ym;
          if (dy > 0) ok &= yp;
          if (dz < 0) ok &= zm;
          if (dz > 0) ok &= zp;
          if (ok) {
            const int cell = (ty + 1 + dy) * kStRow + tx + 1 + dx;
            float c;
            if (s < 13) {                              // mirror slot, at the neighbour
              const int q = 13 - s;
              const unsigned mq = (q * nr3 + m[dz + 1][dy + 1]) & 3u;
              c = (dz < 0 ? Cp : Cc)[q * kStPlane + cell + mq];
            } else {                                   // own slot
              const int q = s - 13;
              const unsigned mq = (q * nr3 + m[1][1]) & 3u;
              c = Cc[q * kStPlane + (ty + 1) * kStRow + tx + 1 + mq];
            }
            const float v = Uz[dz + 1][cell + m[dz + 1][dy + 1]];
            au = fmaf(c, v, au);
          }
        }
        const int n = R.off + i + R.nx * (j + R.ny * l);
        if (mult[n] > 1) y[n] = au; else epi(n, au, 1);
      }
      __syncthreads();                                // before the rings are overwritten
    }
    cp_async_wait<0>();
    __syncthreads();
  }
}

// Phase B: interface groups. y holds the partial row results of every copy. One thread per
// copy: it sums the partial results of its group in ascending slot order (every copy of a group
// forms the identical sum) and applies the epilogue to its own copy.
template <typename AT, class Epi>
__global__ void __launch_bounds__(256)
k_groups(int nslots, const int* __restrict__ sgrp, const int* __restrict__ gptr,
         const int* __restrict__ gslot, const AT* __restrict__ y, Epi epi) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nslots; q += gridDim.x * blockDim.x) {
    const int g = sgrp[q];
    const int a = gptr[g], e = gptr[g + 1];
    AT s = AT(0);
    for (int k = a; k < e; ++k) s += y[gslot[k]];
    epi(gslot[q], s, e - a);
  }
}

// ---- block operators (B dofs per node; elasticity: B = 3) ---------------------------------
// Coefficients of block (c, c') are a scalar stencil: coef[((c * B + c') * S + s) * n_r + n];
// vectors are component-major: v[c * n_r + n]. The epilogues receive the flat index c * n_r + n.
template <int KIND, int B, typename CT, typename VT, typename AT, class Epi>
__global__ void __launch_bounds__(kTile)
k_bstencil(Grid G, const CT* __restrict__ coef, const VT* __restrict__ u,
           const uint8_t* __restrict__ mult, AT* __restrict__ y, Epi epi) {
  using S = Sten<KIND>;
  RMG_FOR_NODES(G)
    int i, j, l;
    RMG_DECODE(i, j, l);
    AT au[B];
#pragma unroll
    for (int c = 0; c < B; ++c) au[c] = AT(0);
    const int sy = R.nx, sz = R.nx * R.ny;
#pragma unroll
    for (int s = 0; s < S::S; ++s) {
      const int dx = S::dx(s), dy = S::dy(s), dz = S::dz(s);
      bool ok = true;
      if (dx < 0) ok &= (i > 0);
      if (dx > 0) ok &= (i < R.nx - 1);
      if (dy < 0) ok &= (j > 0);
      if (dy > 0) ok &= (j < R.ny - 1);
      if (dz < 0) ok &= (l > 0);
      if (dz > 0) ok &= (l < R.nz - 1);
      if (!ok) continue;
      const int nb = n + dx + dy * sy + dz * sz;
      AT uv[B];
#pragma unroll
      for (int c2 = 0; c2 < B; ++c2) uv[c2] = AT(u[(size_t)c2 * G.n_r + nb]);
#pragma unroll
      for (int c = 0; c < B; ++c)
#pragma unroll
        for (int c2 = 0; c2 < B; ++c2)
          au[c] = fma(AT(coef[((size_t)(c * B + c2) * S::S + s) * G.n_r + n]), uv[c2], au[c]);
    }
    if (mult[n] > 1) {
#pragma unroll
      for (int c = 0; c < B; ++c) y[(size_t)c * G.n_r + n] = au[c];
    } else {
#pragma unroll
      for (int c = 0; c < B; ++c) epi(c * G.n_r + n, au[c], 1);
    }
  RMG_END_FOR_NODES
}

template <typename AT, class Epi>
__global__ void __launch_bounds__(256)
k_groups_b(int ngroups, int B, int n_r, const int* __restrict__ gptr,
           const int* __restrict__ gslot, const AT* __restrict__ y, Epi epi) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += gridDim.x * blockDim.x) {
    const int a = gptr[g], e = gptr[g + 1];
    for (int c = 0; c < B; ++c) {
      AT s = AT(0);
      for (int k = a; k < e; ++k) s += y[(size_t)c * n_r + gslot[k]];
      for (int k = a; k < e; ++k) epi(c * n_r + gslot[k], s, e - a);
    }
  }
}

// ------------------------------------------------------------------ epilogues
// An epilogue receives the node, the composite row result (A u)_n and the multiplicity m of
// the node (1 in phase A, the group size in phase B).

// 1/m without a division for the multiplicities of box tilings (1, 2, 4, 8).
template <typename T>
__device__ __forceinline__ T inv_mult(int m) {
  switch (m) {
    case 1: return T(1);
    case 2: return T(0.5);
    case 4: return T(0.25);
    case 8: return T(0.125);
    default: return T(1) / T(m);
  }
}

template <typename T>
struct EpiStore {                 // out = A u
  T* out;
  __device__ void operator()(int n, T au, int) const { out[n] = au; }
};

template <typename T>
struct EpiScaled {                // out = D~^-1 A u (power method)
  const T* dinv; T* out;
  __device__ void operator()(int n, T au, int) const { out[n] = dinv[n] * au; }
};

template <typename T>
struct EpiResid {                 // r = b - A u
  const T* b; T* r;
  __device__ void operator()(int n, T au, int) const { r[n] = b[n] - au; }
};

template <typename T>
struct EpiResidScaled {           // r = (b - A u) / mult: the [[Psi Psi^T]]^-1 of restriction
  const T* b; T* r;
  __device__ void operator()(int n, T au, int m) const { r[n] = (b[n] - au) * inv_mult<T>(m); }
};

template <typename T>
struct EpiJacobi {                // u_out = u + omega D~^-1 (b - A u)
  const T* u; const T* b; const T* dinv; T omega; T* uo;
  __device__ void operator()(int n, T au, int) const {
    const T r = b[n] - au;
    uo[n] = fma(omega * dinv[n], r, u[n]);
  }
};

// The Chebyshev coefficients are read in the cycle's own precision (a per-node conversion
// from FP64 would occupy the slow FP64 pipe of the FP32 cycle).
template <typename T>
struct EpiCheb0 {                 // first Chebyshev step: d = D~^-1 r / theta, u_out = u + d
  const T* u; const T* b; const T* dinv; const T* c2; T* d; T* uo;
  __device__ void operator()(int n, T au, int) const {
    const T r = b[n] - au;
    const T dn = (dinv[n] * r) * (*c2);
    d[n] = dn;
    uo[n] = u[n] + dn;
  }
};

template <typename T>
struct EpiCheb {                  // d = c1 d + c2 D~^-1 r, u_out = u + d
  const T* u; const T* b; const T* dinv; const T* c1; const T* c2; T* d; T* uo;
  __device__ void operator()(int n, T au, int) const {
    const T r = b[n] - au;
    const T dn = (*c1) * d[n] + ((*c2) * dinv[n]) * r;
    d[n] = dn;
    uo[n] = u[n] + dn;
  }
};

// ------------------------------------------------------------------ elementwise
template <typename T>
__global__ void k_jacobi_zero(int n, const T* __restrict__ b, const T* __restrict__ dinv,
                              T omega, T* __restrict__ uo) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    uo[k] = (omega * dinv[k]) * b[k];
}

template <typename T>
__global__ void k_cheb0_zero(int n, const T* __restrict__ b, const T* __restrict__ dinv,
                             const T* __restrict__ c2, T* __restrict__ d,
                             T* __restrict__ uo) {
  const T c = *c2;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const T dn = (dinv[k] * b[k]) * c;
    d[k] = dn;
    uo[k] = dn;
  }
}

// ------------------------------------------------------------------ region Gauss-Seidel
// Algorithm 1 in multicolour order. A sweep starts with r = b - Psi^T Psi [[A]] u at every copy
// (the stencil pair with EpiResidZero, which also sets delta = 0), then runs one launch per
// colour class.
template <typename T>
struct EpiResidZero {              // r = b - A u, delta = 0
  const T* b; T* r; T* delta;
  __device__ void operator()(int n, T au, int) const {
    r[n] = b[n] - au;
    delta[n] = T(0);
  }
};

// The composite value (mean over the copies) of an interface node, written to `out` at every
// copy: the last step of a Gauss-Seidel cycle, whose copies drift apart within a sweep.
template <typename T>
struct EpiMean {
  T* out;
  __device__ void operator()(int n, T s, int m) const { out[n] = s * inv_mult<T>(m); }
};

// dst[gslot[q]] = src[gslot[q]] for every copy of every interface node.
template <typename T>
__global__ void k_copy_slots(int nslots, const int* __restrict__ gslot, const T* __restrict__ src,
                             T* __restrict__ dst) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nslots; q += gridDim.x * blockDim.x)
    dst[gslot[q]] = src[gslot[q]];
}

// A sweep from u = 0: r = b, delta = 0, u = 0.
template <typename VT>
__global__ void k_gs_zero(int n, const VT* __restrict__ b, VT* __restrict__ r,
                          VT* __restrict__ delta, VT* __restrict__ u) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    r[k] = b[k];
    delta[k] = VT(0);
    u[k] = VT(0);
  }
}

// Colour of a regional node: parity of i + j + l for 5/7-point stencils (2 colours), the
// parities of i, j, l for 9/27-point ones (4 colours in 2D, 8 in 3D). Nodes of one colour are
// never coupled by the stencil.
template <int KIND>
__device__ __forceinline__ int gs_colour_of(int i, int j, int l) {
  return (KIND == 5 || KIND == 7) ? ((i + j + l) & 1) : ((i & 1) | ((j & 1) << 1) | ((l & 1) << 2));
}

// One colour class of the region Gauss-Seidel: at the nodes of colour `colour` of every
// region, delta_i = omega (r_i - sum_j A^(k)_ij delta_j) / d~_ii with the region's own stencil
// (no interface sum; delta is zero at the nodes not yet visited in this sweep, the node itself
// included) and u_i += delta_i.
template <int KIND, typename CT, typename VT>
__global__ void __launch_bounds__(kTile)
k_gs_colour(Grid G, const CT* __restrict__ coef, const VT* __restrict__ r,
            const VT* __restrict__ dinv, VT* delta, VT* __restrict__ u, int colour, VT omega) {
  RMG_FOR_NODES(G)
    int i, j, l;
    RMG_DECODE(i, j, l);
    if (gs_colour_of<KIND>(i, j, l) != colour) continue;
    const VT au = stencil_row<KIND, CT, VT, VT>(coef, delta, n, G.n_r, i, j, l, R);
    const VT d = omega * (r[n] - au) * dinv[n];
    delta[n] = d;
    u[n] = u[n] + d;
  RMG_END_FOR_NODES
}

// ------------------------------------------------------------------ transfers (Sec. 3.3)
// 1D linear 3:1 interpolation: a fine node with remainder rem = i mod 3 takes weight
// 1 - rem/3 from coarse node i/3 and rem/3 from coarse node i/3 + 1. Seen from a coarse node,
// the fine node at offset a in [-2, 2] carries w1d(a). All weights are compile-time constants.
__host__ __device__ constexpr double w1d(int a) {
  return a == -2 ? 1.0 / 3.0 : a == -1 ? 2.0 / 3.0 : a == 0 ? 1.0
       : a == 1 ? 1.0 - 1.0 / 3.0 : 1.0 - 2.0 / 3.0;
}
// Weight of the left (side 0) or right (side 1) coarse node of a fine node with remainder rem.
__host__ __device__ constexpr double wrem(int rem, int side) {
  return rem == 0 ? (side == 0 ? 1.0 : 0.0)
       : side == 1 ? rem / 3.0 : 1.0 - rem / 3.0;
}
// The same weights as compile-time constants in precision T (selects only, no division).
template <typename T>
__host__ __device__ constexpr T wrem_t(int rem, int side) {
  return rem == 0 ? (side == 0 ? T(1) : T(0))
       : rem == 1 ? (side == 1 ? T(wrem(1, 1)) : T(wrem(1, 0)))
                  : (side == 1 ? T(wrem(2, 1)) : T(wrem(2, 0)));
}

// Region-local restriction w = [[R]] rs for every coarse node, rs = r / mult being the
// residual already scaled by [[Psi Psi^T]]^-1. Zero at masked coarse nodes (their column of
// P is zero). Shared coarse nodes store into yc for the coarse interface sum.
template <typename T, typename W>
__device__ __forceinline__ T pw_seen_from_coarse(const W* __restrict__ wr, int n_f, int f,
                                                 int axis, int off);

// sum over the fine nodes f = 3C + (a, b, c) of the support of coarse node C of P(f, C) rs[f];
// P(f, C) is a compile-time constant for linear interpolation (STORED = false) or the FP32
// product of the stored per-axis weights of f.
template <int DIM, bool CHECK, bool STORED, typename VT>
__device__ __forceinline__ VT restrict_sum(const VT* __restrict__ rs, const RegionDev& F,
                                           const float* __restrict__ wr, int fn_r,
                                           int I, int J, int L) {
  VT acc = VT(0);
  constexpr int ZL = DIM == 3 ? -2 : 0, ZH = DIM == 3 ? 2 : 0;
#pragma unroll
  for (int c = ZL; c <= ZH; ++c) {
    const int fz = DIM == 3 ? 3 * L + c : 0;
    if (CHECK && (fz < 0 || fz >= F.nz)) continue;
#pragma unroll
    for (int b = -2; b <= 2; ++b) {
      const int fy = 3 * J + b;
      if (CHECK && (fy < 0 || fy >= F.ny)) continue;
      const int row = F.off + F.nx * (fy + F.ny * fz);
#pragma unroll
      for (int a = -2; a <= 2; ++a) {
        const int fx = 3 * I + a;
        if (CHECK && (fx < 0 || fx >= F.nx)) continue;
        VT wgt;
        if (STORED) {
          const int f = row + fx;
          const float wz = DIM == 3 ? pw_seen_from_coarse<float>(wr, fn_r, f, 2, c) : 1.f;
          wgt = VT(wz * (pw_seen_from_coarse<float>(wr, fn_r, f, 1, b) *
                         pw_seen_from_coarse<float>(wr, fn_r, f, 0, a)));
        } else {
          wgt = VT((DIM == 3 ? w1d(c) : 1.0) * (w1d(b) * w1d(a)));
        }
        acc = fma(wgt, rs[row + fx], acc);
      }
    }
  }
  return acc;
}

template <int DIM, typename VT>
__global__ void __launch_bounds__(kTile)
k_restrict(Grid Gc, const RegionDev* __restrict__ fregions, const VT* __restrict__ rs,
           const uint8_t* __restrict__ cmask, const uint8_t* __restrict__ cmult,
           VT* __restrict__ w, VT* __restrict__ yc) {
  RMG_FOR_NODES(Gc)
    int I, J, L;
    decode(li, R, I, J, L);
    VT acc = VT(0);
    if (!cmask[n]) {
      const RegionDev F = fregions[tile_.region];
      const bool inner = I > 0 && I < R.nx - 1 && J > 0 && J < R.ny - 1 &&
                         (DIM == 2 || (L > 0 && L < R.nz - 1));
      acc = inner ? restrict_sum<DIM, false, false, VT>(rs, F, nullptr, 0, I, J, L)
                  : restrict_sum<DIM, true, false, VT>(rs, F, nullptr, 0, I, J, L);
    }
    if (cmult[n] > 1) yc[n] = acc; else w[n] = acc;
  RMG_END_FOR_NODES
}

// Weight of the right coarse neighbour of a fine node with remainder rem (the left one takes
// 1 - w): 0, 1/3, 2/3, compile-time constants in the vector precision.
template <typename VT>
__device__ __forceinline__ VT rem_weight(int rem) {
  return rem == 0 ? VT(0) : (rem == 1 ? VT(1.0 / 3.0) : VT(2.0 / 3.0));
}

// Region-local interpolation and correction u += [[P]] ubar (no inter-region exchange). Every
// fine node gathers the 2 x 2 (x 2) coarse nodes around it and combines them axis by axis with
// the weights (1 - w, w) of its remainders; a right neighbour past the region edge only occurs
// with remainder 0 (weight 0) and is clamped onto the left one.
template <int DIM, typename VT>
__global__ void __launch_bounds__(kTile)
k_prolong(Grid Gf, const RegionDev* __restrict__ cregions, const uint8_t* __restrict__ fmask,
          const VT* __restrict__ ubar, VT* __restrict__ u) {
  RMG_FOR_NODES(Gf)
    if (fmask[n]) continue;
    int i, j, l;
    decode(li, R, i, j, l);
    const RegionDev C = cregions[tile_.region];
    const int cx = i / 3, rx = i - 3 * cx;
    const int cy = j / 3, ry = j - 3 * cy;
    const int cz = DIM == 3 ? l / 3 : 0, rz = DIM == 3 ? l - 3 * cz : 0;
    const int sy = C.nx, sz = C.nx * C.ny;
    const int dx = cx + 1 < C.nx ? 1 : 0;
    const int dy = cy + 1 < C.ny ? sy : 0;
    const int dz = (DIM == 3 && cz + 1 < C.nz) ? sz : 0;
    const VT* b0 = ubar + C.off + cx + sy * cy + sz * cz;
    const VT wx1 = rem_weight<VT>(rx), wx0 = VT(1) - wx1;
    const VT wy1 = rem_weight<VT>(ry), wy0 = VT(1) - wy1;
    auto xline = [&](const VT* p) { return fma(wx1, p[dx], wx0 * p[0]); };
    const VT a0 = fma(wy1, xline(b0 + dy), wy0 * xline(b0));
    VT acc = a0;
    if (DIM == 3) {
      const VT wz1 = rem_weight<VT>(rz), wz0 = VT(1) - wz1;
      const VT a1 = fma(wy1, xline(b0 + dz + dy), wy0 * xline(b0 + dz));
      acc = fma(wz1, a1, wz0 * a0);
    }
    u[n] = u[n] + acc;
  RMG_END_FOR_NODES
}

// ---- transfers with stored per-node weights ------------------------------------------
// wr[a * n_f + f] is the weight fine node f takes from its right coarse neighbour along axis a
// (the left one gets 1 - wr); along an axis where f sits on a coarse index the weight is 1.
// Seen from coarse node C, the fine node f = 3C + offset carries, per axis, 1 for offset 0,
// 1 - wr for offsets 1, 2 (C is f's left neighbour) and wr for offsets -1, -2.
template <typename T, typename W>
__device__ __forceinline__ T pw_seen_from_coarse(const W* __restrict__ wr, int n_f, int f,
                                                 int axis, int off) {
  return off == 0 ? T(1) : (off > 0 ? T(1) - T(wr[(size_t)axis * n_f + f])
                                    : T(wr[(size_t)axis * n_f + f]));
}

template <int DIM, typename VT>
__global__ void __launch_bounds__(kTile)
k_restrict_w(Grid Gc, const RegionDev* __restrict__ fregions, int fn_r, const float* __restrict__ wr,
             const VT* __restrict__ rs, const uint8_t* __restrict__ cmask,
             const uint8_t* __restrict__ cmult, VT* __restrict__ w, VT* __restrict__ yc) {
  RMG_FOR_NODES(Gc)
    int I, J, L;
    decode(li, R, I, J, L);
    VT acc = VT(0);
    if (!cmask[n]) {
      const RegionDev F = fregions[tile_.region];
      const bool inner = I > 0 && I < R.nx - 1 && J > 0 && J < R.ny - 1 &&
                         (DIM == 2 || (L > 0 && L < R.nz - 1));
      acc = inner ? restrict_sum<DIM, false, true, VT>(rs, F, wr, fn_r, I, J, L)
                  : restrict_sum<DIM, true, true, VT>(rs, F, wr, fn_r, I, J, L);
    }
    if (cmult[n] > 1) yc[n] = acc; else w[n] = acc;
  RMG_END_FOR_NODES
}

template <int DIM, typename VT>
__global__ void __launch_bounds__(kTile)
k_prolong_w(Grid Gf, const RegionDev* __restrict__ cregions, const float* __restrict__ wr,
            const uint8_t* __restrict__ fmask, const VT* __restrict__ ubar, VT* __restrict__ u) {
  RMG_FOR_NODES(Gf)
    if (fmask[n]) continue;
    int i, j, l;
    decode(li, R, i, j, l);
    const RegionDev C = cregions[tile_.region];
    const int co[3] = {i / 3, j / 3, DIM == 3 ? l / 3 : 0};
    const int rm[3] = {i - 3 * co[0], j - 3 * co[1], DIM == 3 ? l - 3 * co[2] : 0};
    float w0[3], w1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float r = rm[a] ? wr[(size_t)a * Gf.n_r + n] : 0.f;
      w0[a] = 1.f - r;
      w1[a] = r;
    }
    const int base = C.off + co[0] + C.nx * (co[1] + C.ny * co[2]);
    VT acc = VT(0);
    for (int c = 0; c < (rm[2] ? 2 : 1); ++c)
      for (int b = 0; b < (rm[1] ? 2 : 1); ++b)
        for (int a = 0; a < (rm[0] ? 2 : 1); ++a) {
          const float wgt = (c ? w1[2] : w0[2]) * ((b ? w1[1] : w0[1]) * (a ? w1[0] : w0[0]));
          acc = fma(VT(wgt), ubar[base + a + C.nx * (b + C.ny * c)], acc);
        }
    u[n] = u[n] + acc;
  RMG_END_FOR_NODES
}

// Composite coupling of regional node n in stencil slot `slot`: the sum over the copies of
// the node (a copy in a region without that neighbour contributes zero).
template <int KIND>
__device__ __forceinline__ double comp_coupling(const double* __restrict__ coef, int n_r, int n,
                                                int slot, const uint8_t* __restrict__ mult,
                                                const int* __restrict__ gid,
                                                const int* __restrict__ cgrp,
                                                const int* __restrict__ gptr,
                                                const int* __restrict__ gslot) {
  if (mult[n] == 1) return coef[(size_t)slot * n_r + n];
  const int grp = cgrp[gid[n]];
  double s = 0.0;
  for (int q = gptr[grp]; q < gptr[grp + 1]; ++q) s += coef[(size_t)slot * n_r + gslot[q]];
  return s;
}

// ------------------------------------------------------------------ reductions
// Deterministic two-pass reductions: every block writes one partial sum; a single block
// adds the partials in order.
template <int BS>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[BS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  if (ln == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (ln < BS / 32) ? sh[ln] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;   // valid in thread 0
}

// Composite inner product of consistent regional vectors: sum x y / mult.
// n = B * n_nodes entries, component-major; the multiplicity is that of the node k mod n_nodes.
template <typename XT, typename YT>
__global__ void __launch_bounds__(256)
k_dot(int n, int n_nodes, const XT* __restrict__ x, const YT* __restrict__ y,
      const uint8_t* __restrict__ mult, double* __restrict__ partials) {
  double s = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    // with the multiplicities of box tilings (1, 2, 4, 8) x * (1/mult) is exact and the FMA
    // rounds once
    s = fma(double(x[k]) * inv_mult<double>(mult[k < n_nodes ? k : k % n_nodes]), double(y[k]), s);
  s = block_sum<256>(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__device__ __forceinline__ double sum_partials(const double* __restrict__ partials, int np) {
  double s = 0.0;
  for (int k = threadIdx.x; k < np; k += blockDim.x) s += partials[k];
  return block_sum<256>(s);
}

}  // namespace rmg
