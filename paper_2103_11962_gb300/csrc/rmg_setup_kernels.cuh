// Setup-phase kernels: coarse layouts, diagonals, regional Galerkin products, power method,
// coarsest composite operator and its dense factorisation.
#pragma once

#include "rmg_kernels.cuh"

namespace rmg {

// ------------------------------------------------------------------ inject (Psibar)
// A regional node is a coarse point when its local indices are multiples of 3 (Sec. 3.2,
// 3:1 structured coarsening). All copies of a composite node must agree.
__global__ void k_coarse_flags(Grid G, int dim, const int* __restrict__ gid, int* __restrict__ flag) {
  RMG_FOR_NODES(G)
    int i, j, l;
    decode(li, R, i, j, l);
    const bool cp = (i % 3 == 0) && (j % 3 == 0) && (dim == 2 || l % 3 == 0);
    atomicOr(&flag[gid[n]], cp ? 1 : 2);
  RMG_END_FOR_NODES
}

__global__ void k_coarse_select(int ncomp, const int* __restrict__ flag, int* __restrict__ sel,
                                int* err) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ncomp; g += gridDim.x * blockDim.x) {
    const int f = flag[g];
    if (f == 3) set_err(err, DERR_COARSE_MISMATCH);
    sel[g] = (f == 1) ? 1 : 0;
  }
}

// Coarse regional node (I, J, L) of region k is co-located with fine node (3I, 3J, 3L).
__global__ void k_coarse_gids(Grid Gc, int dim, const RegionDev* __restrict__ fregs,
                              const int* __restrict__ fgid, const uint8_t* __restrict__ fmask,
                              const int* __restrict__ cid, int* __restrict__ cgid,
                              uint8_t* __restrict__ cmask, int* __restrict__ count) {
  RMG_FOR_NODES(Gc)
    int I, J, L;
    decode(li, R, I, J, L);
    const RegionDev F = fregs[tile_.region];
    const int f = F.off + 3 * I + F.nx * (3 * J + F.ny * (dim == 3 ? 3 * L : 0));
    const int g = cid[fgid[f]];
    cgid[n] = g;
    cmask[n] = fmask[f];
    atomicAdd(&count[g], 1);
  RMG_END_FOR_NODES
}

// ------------------------------------------------------------------ diagonal (Sec. 3.2)
// D~ = Psi^T Psi diag([[A]]); stores D~^-1.
template <int KIND>
__global__ void k_diag_local(int n_r, const double* __restrict__ coef,
                             const uint8_t* __restrict__ mult, double* __restrict__ dinv,
                             double* __restrict__ y) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_r; k += gridDim.x * blockDim.x) {
    const double d = coef[(size_t)Sten<KIND>::CENTER * n_r + k];
    if (mult[k] > 1) y[k] = d; else dinv[k] = 1.0 / d;
  }
}

struct EpiRecip {
  double* dinv;
  __device__ void operator()(int n, double s, int) const { dinv[n] = 1.0 / s; }
};

// ------------------------------------------------------------------ Galerkin product
// [[Abar]] = [[R]] [[A]] [[P]] (eq. RegionalGalerkinProduct), region by region, in two steps
// following the product order R (A P):
//  1. k_ap: for every fine node f, row f of [[A]] [[P]], i.e. sum_s A_s(f) P(f + d_s, C') for
//     the (at most 3 per axis) coarse nodes C' near f, stored relative to the coarse node
//     (x - 1) div 3 on each axis: ap[o][f], o = ox + 3 oy + 9 oz.
//  2. k_rtap: for every coarse node C, sum over the fine nodes f = 3C + (a, b, c) of its
//     support of P(f, C) ap[.][f]; the weights P(f, C) are compile-time constants.
// Masked fine nodes have zero rows of P, masked coarse nodes zero columns; a masked coarse
// row becomes 1/mult on the diagonal so that the composite sum is the identity row.
// T is the arithmetic of the product: FP64 for the plain method; FP32 for the hierarchies of
// the mixed-precision cycle, whose coarse operators only ever enter an FP32 cycle (GB300's
// FP64 pipe would make these sums the largest part of the setup).
__device__ __forceinline__ int floor_div3m1(int x) { return (x + 2) / 3 - 1; }   // (x-1) div 3, x >= 0

template <int FK, int DIM, typename T>
__global__ void __launch_bounds__(kTile)
k_ap(Grid Gf, const RegionDev* __restrict__ cregs, const T* __restrict__ fcoef,
     const uint8_t* __restrict__ fmask, const uint8_t* __restrict__ cmask,
     T* __restrict__ ap) {
  using FS = Sten<FK>;
  constexpr int NO = DIM == 3 ? 27 : 9;
  __shared__ T tab[27 * 8];
  extern __shared__ __align__(16) unsigned char ap_smem[];   // NO x kTile accumulators
  T (*acc)[kTile] = reinterpret_cast<T (*)[kTile]>(ap_smem);
  for (int e = threadIdx.x; e < 27 * 8; e += blockDim.x) {
    const int r = e >> 3, combo = e & 7;
    tab[e] = wrem_t<T>(r / 9, combo >> 2) *
             (wrem_t<T>((r / 3) % 3, (combo >> 1) & 1) * wrem_t<T>(r % 3, combo & 1));
  }
  __syncthreads();
  const int tid = threadIdx.x;
  RMG_FOR_NODES(Gf)
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o][tid] = T(0);
    if (!fmask[n]) {
      int x, y, z;
      decode(li, R, x, y, z);
      const RegionDev C = cregs[tile_.region];
      const int cx0 = floor_div3m1(x), cy0 = floor_div3m1(y), cz0 = DIM == 3 ? floor_div3m1(z) : 0;
#pragma unroll
      for (int s = 0; s < FS::S; ++s) {
        const int gx = x + FS::dx(s), gy = y + FS::dy(s), gz = z + FS::dz(s);
        if (gx < 0 || gx >= R.nx || gy < 0 || gy >= R.ny || gz < 0 || gz >= R.nz) continue;
        const T v = fcoef[(size_t)s * Gf.n_r + n];
        if (v == T(0)) continue;
        if (fmask[R.off + gx + R.nx * (gy + R.ny * gz)]) continue;
        const int x0 = gx / 3, rx = gx - 3 * x0;
        const int y0 = gy / 3, ry = gy - 3 * y0;
        const int z0 = DIM == 3 ? gz / 3 : 0, rz = DIM == 3 ? gz - 3 * z0 : 0;
        const T* t = tab + 8 * (rx + 3 * ry + 9 * rz);
        for (int c = 0; c < (rz ? 2 : 1); ++c)
          for (int b = 0; b < (ry ? 2 : 1); ++b)
            for (int a = 0; a < (rx ? 2 : 1); ++a) {
              const int X = x0 + a, Y = y0 + b, Z = z0 + c;
              if (cmask[C.off + X + C.nx * (Y + C.ny * Z)]) continue;
              const int o = (X - cx0) + 3 * (Y - cy0) + 9 * (Z - cz0);
              acc[o][tid] = fma(v, t[a + 2 * b + 4 * c], acc[o][tid]);
            }
      }
    }
#pragma unroll
    for (int o = 0; o < NO; ++o) ap[(size_t)o * Gf.n_r + n] = acc[o][tid];
  RMG_END_FOR_NODES
}

// A P for any fine stencil in FP32, for the mixed hierarchies: every output o of the
// 3 x 3 (x 3) coarse neighbourhood of f (the same ap[o][f] layout as k_ap) is evaluated
// directly as sum_s A_s(f) wx(g_x - 3 X) wy(g_y - 3 Y) wz(g_z - 3 Z), g = f + d_s, with the
// linear weights w(t) = 1 - |t|/3 for |t| <= 2. No divergent loops and no shared memory; the
// 27 x S FMAs are cheap on the FP32 pipe (in FP64 they would not be, so the plain method keeps
// k_ap). Masked fine neighbours and masked coarse nodes contribute nothing.
__device__ __forceinline__ float lin_w(int t) {
  t = t < 0 ? -t : t;
  return t == 0 ? 1.f : (t == 1 ? 2.f / 3.f : (t == 2 ? 1.f / 3.f : 0.f));
}

template <int FK, int DIM>
__global__ void __launch_bounds__(kTile)
k_ap_axis32(Grid Gf, const RegionDev* __restrict__ cregs, const float* __restrict__ fcoef,
            const uint8_t* __restrict__ fmask, const uint8_t* __restrict__ cmask,
            float* __restrict__ ap) {
  using FS = Sten<FK>;
  constexpr int NO = DIM == 3 ? 27 : 9;
  constexpr int NZ = DIM == 3 ? 3 : 1;
  RMG_FOR_NODES(Gf)
    float out[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) out[o] = 0.f;
    if (!fmask[n]) {
      int x, y, z;
      decode(li, R, x, y, z);
      const int cx0 = floor_div3m1(x), cy0 = floor_div3m1(y), cz0 = DIM == 3 ? floor_div3m1(z) : 0;
#pragma unroll
      for (int s = 0; s < FS::S; ++s) {
        const int dx = FS::dx(s), dy = FS::dy(s), dz = FS::dz(s);
        const int gx = x + dx, gy = y + dy, gz = z + dz;
        if (gx < 0 || gx >= R.nx || gy < 0 || gy >= R.ny || gz < 0 || gz >= R.nz) continue;
        if (fmask[R.off + gx + R.nx * (gy + R.ny * gz)]) continue;
        const float v = fcoef[(size_t)s * Gf.n_r + n];
        float wx[3], wy[3], wz[NZ];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          wx[k] = lin_w(gx - 3 * (cx0 + k));
          wy[k] = lin_w(gy - 3 * (cy0 + k));
        }
#pragma unroll
        for (int k = 0; k < NZ; ++k) wz[k] = DIM == 3 ? lin_w(gz - 3 * (cz0 + k)) : 1.f;
#pragma unroll
        for (int kz = 0; kz < NZ; ++kz)
#pragma unroll
          for (int ky = 0; ky < 3; ++ky) {
            const float vyz = v * (wz[kz] * wy[ky]);
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) out[kx + 3 * ky + 9 * kz] = fmaf(vyz, wx[kx], out[kx + 3 * ky + 9 * kz]);
          }
      }
      const RegionDev C = cregs[tile_.region];
#pragma unroll
      for (int kz = 0; kz < NZ; ++kz)
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) {
            const int X = cx0 + kx, Y = cy0 + ky, Z = cz0 + kz;
            const int o = kx + 3 * ky + 9 * kz;
            if (X < 0 || X >= C.nx || Y < 0 || Y >= C.ny || Z < 0 || Z >= C.nz ||
                cmask[C.off + X + C.nx * (Y + C.ny * Z)])
              out[o] = 0.f;
          }
    }
#pragma unroll
    for (int o = 0; o < NO; ++o) ap[(size_t)o * Gf.n_r + n] = out[o];
  RMG_END_FOR_NODES
}

// k_ap_axis32 for a 27-point fine stencil in 3D. Its slots and the weights of P are both tensor
// products, so the contraction factorises axis by axis, sum_dz wz (sum_dy wy (sum_dx wx A_s)):
// 243 FMAs instead of 729, and 27 weights per node instead of 243 (the sums are in another
// order than k_ap_axis32's, equal to FP32 rounding). Bound for 3 blocks per SM (80 registers).
__global__ void __launch_bounds__(kTile, 3)
k_ap_tensor27(Grid Gf, const RegionDev* __restrict__ cregs, const float* __restrict__ fcoef,
              const uint8_t* __restrict__ fmask, const uint8_t* __restrict__ cmask,
              float* __restrict__ ap) {
  RMG_FOR_NODES(Gf)
    float out[27];
#pragma unroll
    for (int o = 0; o < 27; ++o) out[o] = 0.f;
    if (!fmask[n]) {
      int x, y, z;
      decode(li, R, x, y, z);
      const int cx0 = floor_div3m1(x), cy0 = floor_div3m1(y), cz0 = floor_div3m1(z);
      float wx[3][3], wy[3][3], wz[3][3];            // [d + 1][k]: weight of fine offset d - 1
                                                     // towards coarse node c*0 + k
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          wx[d][k] = lin_w(x + d - 1 - 3 * (cx0 + k));
          wy[d][k] = lin_w(y + d - 1 - 3 * (cy0 + k));
          wz[d][k] = lin_w(z + d - 1 - 3 * (cz0 + k));
        }
#pragma unroll
      for (int dz = 0; dz < 3; ++dz) {
        float t2[3][3];                                // [ky][kx]
#pragma unroll
        for (int k = 0; k < 9; ++k) t2[k / 3][k % 3] = 0.f;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          float t1[3] = {0.f, 0.f, 0.f};               // [kx]
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            const int gx = x + dx - 1, gy = y + dy - 1, gz = z + dz - 1;
            if (gx < 0 || gx >= R.nx || gy < 0 || gy >= R.ny || gz < 0 || gz >= R.nz) continue;
            // the coefficient and the neighbour's mask are loaded independently (no round trip
            // between them); a masked neighbour contributes a zero product
            const float cv = fcoef[(size_t)(dx + 3 * dy + 9 * dz) * Gf.n_r + n];
            const float v = fmask[R.off + gx + R.nx * (gy + R.ny * gz)] ? 0.f : cv;
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) t1[kx] = fmaf(v, wx[dx][kx], t1[kx]);
          }
#pragma unroll
          for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) t2[ky][kx] = fmaf(t1[kx], wy[dy][ky], t2[ky][kx]);
        }
#pragma unroll
        for (int kz = 0; kz < 3; ++kz)
#pragma unroll
          for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx)
              out[kx + 3 * ky + 9 * kz] = fmaf(t2[ky][kx], wz[dz][kz], out[kx + 3 * ky + 9 * kz]);
      }
      const RegionDev C = cregs[tile_.region];
#pragma unroll
      for (int kz = 0; kz < 3; ++kz)
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) {
            const int X = cx0 + kx, Y = cy0 + ky, Z = cz0 + kz;
            if (X < 0 || X >= C.nx || Y < 0 || Y >= C.ny || Z < 0 || Z >= C.nz ||
                cmask[C.off + X + C.nx * (Y + C.ny * Z)])
              out[kx + 3 * ky + 9 * kz] = 0.f;
          }
    }
#pragma unroll
    for (int o = 0; o < 27; ++o) ap[(size_t)o * Gf.n_r + n] = out[o];
  RMG_END_FOR_NODES
}

// Level 0 of the FP32 cycle in one pass over the FP64 coefficients: the FP32 copy of every
// plane (for the FP32 Galerkin chain and the asymmetric fallback) and the half planes of
// stencil_row_half (planes C..S-1). *asym becomes 1 when a mirrored pair of the FP32 copy
// inside a region differs in any bit (the sweeps then keep reading the full planes); the pair's
// far value is rounded here from its FP64 value, the same rounding that made the copy.
template <int KIND>
__global__ void __launch_bounds__(kTile)
k_level0_fp32(Grid G, const double* __restrict__ coef, float* __restrict__ coef32,
              float* __restrict__ half, int* __restrict__ asym) {
  using S = Sten<KIND>;
  static_assert(mirrored_slots<KIND>(), "half storage needs mirrored stencil slots");
  constexpr int C = S::CENTER;
  bool bad = false;
  RMG_FOR_NODES(G)
    int i, j, l;
    RMG_DECODE(i, j, l);
    const int sy = R.nx, sz = R.nx * R.ny;
#pragma unroll
    for (int s = 0; s < S::S; ++s) {
      const float cv = static_cast<float>(coef[(size_t)s * G.n_r + n]);
      coef32[(size_t)s * G.n_r + n] = cv;
      if (s < C) continue;
      half[(size_t)(s - C) * G.n_r + n] = cv;
      const int dx = S::dx(s), dy = S::dy(s), dz = S::dz(s);
      bool ok = s > C;
      if (dx < 0) ok &= (i > 0);
      if (dx > 0) ok &= (i < R.nx - 1);
      if (dy < 0) ok &= (j > 0);
      if (dy > 0) ok &= (j < R.ny - 1);
      if (dz < 0) ok &= (l > 0);
      if (dz > 0) ok &= (l < R.nz - 1);
      if (ok) {
        const float mv = static_cast<float>(
            coef[(size_t)(S::S - 1 - s) * G.n_r + n + dx + dy * sy + dz * sz]);
        bad |= __float_as_uint(cv) != __float_as_uint(mv);
      }
    }
  RMG_END_FOR_NODES
  if (__syncthreads_or(bad) && threadIdx.x == 0) *asym = 1;
}

template <int DIM, bool CHECK, bool STORED, typename T>
__device__ __forceinline__ void rtap_sum(const T* __restrict__ ap, int fn_r,
                                         const RegionDev& F, const float* __restrict__ wr,
                                         int I, int J, int L, T (&acc)[27]) {
  constexpr int ZL = DIM == 3 ? -2 : 0, ZH = DIM == 3 ? 2 : 0;
#pragma unroll
  for (int c = ZL; c <= ZH; ++c) {
    const int fz = DIM == 3 ? 3 * L + c : 0;
    if (CHECK && (fz < 0 || fz >= F.nz)) continue;
#pragma unroll
    for (int b = -2; b <= 2; ++b) {
      const int fy = 3 * J + b;
      if (CHECK && (fy < 0 || fy >= F.ny)) continue;
#pragma unroll
      for (int a = -2; a <= 2; ++a) {
        const int fx = 3 * I + a;
        if (CHECK && (fx < 0 || fx >= F.nx)) continue;
        const int f = F.off + fx + F.nx * (fy + F.ny * fz);
        T wf;
        if (STORED) {
          const float wz = DIM == 3 ? pw_seen_from_coarse<float>(wr, fn_r, f, 2, c) : 1.f;
          wf = T(wz * (pw_seen_from_coarse<float>(wr, fn_r, f, 1, b) *
                       pw_seen_from_coarse<float>(wr, fn_r, f, 0, a)));
        } else {
          wf = T((DIM == 3 ? w1d(c) : 1.0) * (w1d(b) * w1d(a)));   // compile-time constant
        }
        // ap of node f is stored relative to the coarse node (f - 1) div 3 on each axis,
        // which is C - 1 for offsets a <= 0 and C for a >= 1
        const int bx = a <= 0 ? 1 : 0, by = b <= 0 ? 1 : 0, bz = DIM == 3 ? (c <= 0 ? 1 : 0) : 0;
#pragma unroll
        for (int oz = (DIM == 3 ? -1 : 0); oz <= (DIM == 3 ? 1 : 0); ++oz)
#pragma unroll
          for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
            for (int ox = -1; ox <= 1; ++ox) {
              const int ix = ox + bx, iy = oy + by, iz = oz + bz;
              if (ix < 0 || ix > 2 || iy < 0 || iy > 2 || iz < 0 || iz > 2) continue;
              // (A P)(f, C + o) vanishes unless |f - 3 (C + o)| <= 3 on every axis (A reaches
              // one node, P two): skip those structural zeros (compile-time, exact)
              if (3 * ox - a > 3 || a - 3 * ox > 3 || 3 * oy - b > 3 || b - 3 * oy > 3) continue;
              if (DIM == 3 && (3 * oz - c > 3 || c - 3 * oz > 3)) continue;
              const int slot = (ox + 1) + 3 * (oy + 1) + (DIM == 3 ? 9 * (oz + 1) : 0);
              acc[slot] = fma(wf, ap[(size_t)(ix + 3 * iy + 9 * iz) * fn_r + f], acc[slot]);
            }
      }
    }
  }
}

template <int CK, int DIM, typename T>
__global__ void __launch_bounds__(kTile)
k_rtap(Grid Gc, const RegionDev* __restrict__ fregs, const T* __restrict__ ap, int fn_r,
       const uint8_t* __restrict__ cmask, const uint8_t* __restrict__ cmult, double mdiag,
       T* __restrict__ ccoef) {
  using CS = Sten<CK>;
  RMG_FOR_NODES(Gc)
    T acc[27];
#pragma unroll
    for (int o = 0; o < 27; ++o) acc[o] = T(0);
    if (cmask[n]) {
      acc[DIM == 3 ? 13 : 4] = T(mdiag) / T(cmult[n]);
    } else {
      int I, J, L;
      decode(li, R, I, J, L);
      const RegionDev F = fregs[tile_.region];
      const bool inner = I > 0 && I < R.nx - 1 && J > 0 && J < R.ny - 1 &&
                         (DIM == 2 || (L > 0 && L < R.nz - 1));
      if (inner) rtap_sum<DIM, false, false, T>(ap, fn_r, F, nullptr, I, J, L, acc);
      else rtap_sum<DIM, true, false, T>(ap, fn_r, F, nullptr, I, J, L, acc);
    }
#pragma unroll
    for (int s = 0; s < CS::S; ++s) ccoef[(size_t)s * Gc.n_r + n] = acc[s];
  RMG_END_FOR_NODES
}

// Galerkin product with stored per-node weights (same two steps as k_ap / k_rtap).
template <int FK, int DIM, typename T>
__global__ void __launch_bounds__(kTile)
k_ap_w(Grid Gf, const RegionDev* __restrict__ cregs, const T* __restrict__ fcoef,
       const float* __restrict__ wr, const uint8_t* __restrict__ fmask,
       const uint8_t* __restrict__ cmask, T* __restrict__ ap) {
  using FS = Sten<FK>;
  constexpr int NO = DIM == 3 ? 27 : 9;
  extern __shared__ __align__(16) unsigned char ap_smem[];
  T (*acc)[kTile] = reinterpret_cast<T (*)[kTile]>(ap_smem);
  const int tid = threadIdx.x;
  RMG_FOR_NODES(Gf)
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o][tid] = T(0);
    if (!fmask[n]) {
      int x, y, z;
      decode(li, R, x, y, z);
      const RegionDev C = cregs[tile_.region];
      const int cx0 = floor_div3m1(x), cy0 = floor_div3m1(y), cz0 = DIM == 3 ? floor_div3m1(z) : 0;
#pragma unroll
      for (int s = 0; s < FS::S; ++s) {
        const int gx = x + FS::dx(s), gy = y + FS::dy(s), gz = z + FS::dz(s);
        if (gx < 0 || gx >= R.nx || gy < 0 || gy >= R.ny || gz < 0 || gz >= R.nz) continue;
        const T v = fcoef[(size_t)s * Gf.n_r + n];
        if (v == T(0)) continue;
        const int f2 = R.off + gx + R.nx * (gy + R.ny * gz);
        if (fmask[f2]) continue;
        const int x0 = gx / 3, rx = gx - 3 * x0;
        const int y0 = gy / 3, ry = gy - 3 * y0;
        const int z0 = DIM == 3 ? gz / 3 : 0, rz = DIM == 3 ? gz - 3 * z0 : 0;
        const float wx = rx ? wr[f2] : 0.f;
        const float wy = ry ? wr[(size_t)Gf.n_r + f2] : 0.f;
        const float wz = rz ? wr[(size_t)2 * Gf.n_r + f2] : 0.f;
        for (int c = 0; c < (rz ? 2 : 1); ++c)
          for (int b = 0; b < (ry ? 2 : 1); ++b)
            for (int a = 0; a < (rx ? 2 : 1); ++a) {
              const int X = x0 + a, Y = y0 + b, Z = z0 + c;
              if (cmask[C.off + X + C.nx * (Y + C.ny * Z)]) continue;
              const float wgt = (c ? wz : 1.f - wz) * ((b ? wy : 1.f - wy) * (a ? wx : 1.f - wx));
              const int o = (X - cx0) + 3 * (Y - cy0) + 9 * (Z - cz0);
              acc[o][tid] = fma(v, T(wgt), acc[o][tid]);
            }
      }
    }
#pragma unroll
    for (int o = 0; o < NO; ++o) ap[(size_t)o * Gf.n_r + n] = acc[o][tid];
  RMG_END_FOR_NODES
}

template <int CK, int DIM, typename T>
__global__ void __launch_bounds__(kTile)
k_rtap_w(Grid Gc, const RegionDev* __restrict__ fregs, const T* __restrict__ ap, int fn_r,
         const float* __restrict__ wr, const uint8_t* __restrict__ cmask,
         const uint8_t* __restrict__ cmult, double mdiag, T* __restrict__ ccoef) {
  using CS = Sten<CK>;
  RMG_FOR_NODES(Gc)
    T acc[27];
#pragma unroll
    for (int o = 0; o < 27; ++o) acc[o] = T(0);
    if (cmask[n]) {
      acc[DIM == 3 ? 13 : 4] = T(mdiag) / T(cmult[n]);
    } else {
      int I, J, L;
      decode(li, R, I, J, L);
      const RegionDev F = fregs[tile_.region];
      const bool inner = I > 0 && I < R.nx - 1 && J > 0 && J < R.ny - 1 &&
                         (DIM == 2 || (L > 0 && L < R.nz - 1));
      if (inner) rtap_sum<DIM, false, true, T>(ap, fn_r, F, wr, I, J, L, acc);
      else rtap_sum<DIM, true, true, T>(ap, fn_r, F, wr, I, J, L, acc);
    }
#pragma unroll
    for (int s = 0; s < CS::S; ++s) ccoef[(size_t)s * Gc.n_r + n] = acc[s];
  RMG_END_FOR_NODES
}

// ---- operator-dependent interpolation weights (teacher of the learned prolongator) ----
// Along each axis a fine node between coarse nodes X0 and X0 + 3 lies on a line of three
// edges with composite conductances k_i = -A(p_i, p_i+1). Treating the line as resistors in
// series (the 1D A-harmonic extension), the weight of the right coarse node at position rem
// is (1/k_0 + ... + 1/k_{rem-1}) / (1/k_0 + 1/k_1 + 1/k_2). With equal conductances this is
// rem/3, the linear weight; with a non-positive conductance the linear weight is kept.
// Composite couplings are the sums over the copies of a node, so co-located copies obtain
// identical weights (the matching condition of Lemma 2).
template <int KIND>
__global__ void __launch_bounds__(kTile)
k_opdep(Grid G, const double* __restrict__ coef, const uint8_t* __restrict__ mult,
        const int* __restrict__ gid, const int* __restrict__ cgrp, const int* __restrict__ gptr,
        const int* __restrict__ gslot, float* __restrict__ wr) {
  constexpr int DIM = Sten<KIND>::DIM;
  RMG_FOR_NODES(G)
    int x[3];
    decode(li, R, x[0], x[1], x[2]);
    const int stride[3] = {1, R.nx, R.nx * R.ny};
    const int len[3] = {R.nx, R.ny, R.nz};
    for (int a = 0; a < 3; ++a) {
      int rem = (a < DIM) ? x[a] % 3 : 0;
      if (rem && x[a] - rem + 3 > len[a] - 1) rem = 0;   // no right coarse node in the region
      double w = 0.0;
      if (rem) {
        const int slot = sten_slot<KIND>(a == 0, a == 1, a == 2);   // coupling to +e_a
        const int p0 = n - rem * stride[a];
        double rsum[3];
        bool ok = slot >= 0;
        for (int e = 0; e < 3 && ok; ++e) {
          const double k = -comp_coupling<KIND>(coef, G.n_r, p0 + e * stride[a], slot, mult, gid,
                                                cgrp, gptr, gslot);
          if (!(k > 0.0)) ok = false;
          else rsum[e] = 1.0 / k;
        }
        if (ok) {
          const double tot = rsum[0] + rsum[1] + rsum[2];
          w = (rem == 1 ? rsum[0] : rsum[0] + rsum[1]) / tot;
        } else {
          w = rem / 3.0;
        }
      }
      wr[(size_t)a * G.n_r + n] = (float)w;
    }
  RMG_END_FOR_NODES
}

// Piecewise-constant 3:1 transfers (the "Const" grid transfers of Table 4): every fine node
// takes weight 1 from its nearest coarse node along each axis (remainder 1: the left one,
// remainder 2: the right one), so each row of P has a single unit entry.
__global__ void k_constant_weights(Grid G, int dim, float* __restrict__ wr) {
  RMG_FOR_NODES(G)
    int x[3];
    decode(li, R, x[0], x[1], x[2]);
    for (int a = 0; a < 3; ++a) {
      const int rem = a < dim ? x[a] % 3 : 0;
      wr[(size_t)a * G.n_r + n] = rem == 2 ? 1.f : 0.f;
    }
  RMG_END_FOR_NODES
}

// ------------------------------------------------------------------ power method (Sec. 3.4)
// SplitMix64 as a counter-based generator: value i of stream seed = output i+1 of a
// generator seeded with seed (Steele, Lea, Flood 2014). Doubles in [-1, 1) from the top 53 bits.
__device__ __forceinline__ double splitmix_pm1(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * 0x1.0p-52 - 1.0;
}

// Random start vector: value of composite dof g*B + b (dofs numbered node-major) at every
// copy of the node; zero at masked nodes. Regional vectors are component-major.
template <typename VT>
__global__ void k_power_init(int n_r, int B, const int* __restrict__ gid,
                             const uint8_t* __restrict__ mask, unsigned long long seed,
                             VT* __restrict__ x) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_r; k += gridDim.x * blockDim.x)
    for (int b = 0; b < B; ++b)
      x[(size_t)b * n_r + k] =
          mask[k] ? VT(0) : VT(splitmix_pm1(seed, (unsigned long long)gid[k] * B + b));
}

// out = sum of partials, then an operation on the scalar block.
// FIN_SQRT stores sqrt(sum) in dst[0] and its reciprocal in dst[1].
enum FinOp : int { FIN_SQRT = 0, FIN_STORE = 1 };
__global__ void k_finalize(const double* __restrict__ partials, int np, double* __restrict__ dst,
                           int op) {
  const double s = sum_partials(partials, np);
  if (threadIdx.x == 0) {
    if (op == FIN_SQRT) {
      const double r = sqrt(s);
      dst[0] = r;
      dst[1] = 1.0 / r;
    } else {
      dst[0] = s;
    }
  }
}

// out = x / ||x|| as a product with the stored reciprocal norm.
template <typename VT>
__global__ void k_scale_div(int n, const VT* __restrict__ x, const double* __restrict__ nrm,
                            VT* __restrict__ out) {
  const VT d = VT(nrm[1]);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    out[k] = x[k] * d;
}

// lambda = num / den, then the Chebyshev coefficient table of Algorithm 2 for this level.
__global__ void k_cheb_coeffs(Scalars* sc, int level, double eig_ratio, double boost, int degree) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double lam = sc->pw_num / sc->pw_den;
  sc->lam[level] = lam;
  const double alpha = lam / eig_ratio, beta = boost * lam;
  const double theta = 0.5 * (alpha + beta);
  const double delta = 2.0 / (beta - alpha);
  double rho = 1.0 / (theta * delta);
  sc->cheb_c1[level][0] = 0.0;
  sc->cheb_c2[level][0] = 1.0 / theta;
  for (int k = 1; k < degree && k < 8; ++k) {
    const double rho_old = rho;
    rho = 1.0 / (2.0 * theta * delta - rho_old);
    sc->cheb_c1[level][k] = rho * rho_old;
    sc->cheb_c2[level][k] = 2.0 * rho * delta;
  }
  for (int k = 0; k < 8; ++k) {
    sc->cheb_c1f[level][k] = (float)sc->cheb_c1[level][k];
    sc->cheb_c2f[level][k] = (float)sc->cheb_c2[level][k];
  }
}

// ------------------------------------------------------------------ coarsest composite level
__global__ void k_coarse_free(int ncomp, const int* __restrict__ c2r, const uint8_t* __restrict__ mask,
                              int* __restrict__ freeflag) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ncomp; g += gridDim.x * blockDim.x)
    freeflag[g] = mask[c2r[g]] ? 0 : 1;
}

__global__ void k_coarse_maps(int ncomp, const int* __restrict__ freeflag, const int* __restrict__ pos,
                              const int* __restrict__ c2r, int* __restrict__ cidx,
                              int* __restrict__ cu2slot, long long* __restrict__ cu2gid) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ncomp; g += gridDim.x * blockDim.x) {
    if (freeflag[g]) {
      cidx[g] = pos[g];
      cu2slot[pos[g]] = c2r[g];
      cu2gid[pos[g]] = g;
    } else {
      cidx[g] = -1;
    }
  }
}

// Abar = Psibar [[Abar]] Psibar^T restricted to unmasked nodes (eq. CoarseCompositeOperator):
// row of composite node g = sum over its regional copies of their region rows. With B dofs per
// node the dense matrix has dimension B * nc, dof cidx * B + b (blockIdx.y = row component).
template <int KIND>
__global__ void k_coarse_assemble(int ncomp, int B, const RegionDev* __restrict__ regs, int nreg,
                                  int n_r, const double* __restrict__ coef,
                                  const int* __restrict__ gid, const int* __restrict__ cidx,
                                  const int* __restrict__ c2r, const int* __restrict__ cgrp,
                                  const int* __restrict__ gptr, const int* __restrict__ gslot,
                                  int nd, double* __restrict__ M) {
  using S = Sten<KIND>;
  const int b = blockIdx.y;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ncomp; g += gridDim.x * blockDim.x) {
    const int rowc = cidx[g];
    if (rowc < 0) continue;
    const size_t row = (size_t)rowc * B + b;
    const int grp = cgrp[g];
    const int a = grp < 0 ? 0 : gptr[grp];
    const int e = grp < 0 ? 1 : gptr[grp + 1];
    for (int q = a; q < e; ++q) {
      const int n = grp < 0 ? c2r[g] : gslot[q];
      const RegionDev R = regs[region_of(regs, nreg, n)];
      int i, j, l;
      decode(n - R.off, R, i, j, l);
      for (int s = 0; s < S::S; ++s) {
        const int x = i + S::dx(s), y = j + S::dy(s), z = l + S::dz(s);
        if (x < 0 || x >= R.nx || y < 0 || y >= R.ny || z < 0 || z >= R.nz) continue;
        const int n2 = R.off + x + R.nx * (y + R.ny * z);
        const int col = cidx[gid[n2]];
        if (col < 0) continue;
        for (int b2 = 0; b2 < B; ++b2)
          M[row * nd + (size_t)col * B + b2] +=
              coef[((size_t)(b * B + b2) * S::S + s) * n_r + n];
      }
    }
  }
}

// Blocked right-looking Cholesky (lower), block width 32, in place in row-major M, followed by
// the explicit inverse Ainv = L^-T L^-1 for the coarse solve (one GEMV per cycle).
//  k_chol_diag   one warp factors the 32 x 32 diagonal block and inverts it (Dinv_k = L_kk^-1);
//  k_chol_panel  L_ik = A_ik L_kk^-T as a product with Dinv_k (no serial solve per row);
//  k_chol_update trailing update of the lower triangle;
//  k_inv_merge   X = L^-1 from the inverted diagonal blocks by recursive doubling;
//  k_xtx         Ainv = X^T X (lower tiles, mirrored).
// A partial last block is padded with the identity inside the kernels.
constexpr int kNB = 32;

template <typename F>
__global__ void __launch_bounds__(32)
k_chol_diag(F* M, int n, int k0, F* __restrict__ Dblk, int* err) {
  __shared__ F T[kNB][kNB + 1];
  __shared__ F X[kNB][kNB + 1];
  __shared__ F rdiag[kNB];
  const int nb = min(kNB, n - k0);
  const int ln = threadIdx.x;
  for (int i = 0; i < kNB; ++i)
    T[i][ln] = (i < nb && ln < nb) ? M[(size_t)(k0 + i) * n + k0 + ln] : F(i == ln ? 1 : 0);
  __syncwarp();
  for (int j = 0; j < kNB; ++j) {
    F p = T[j][j];
    if (!(p > F(0))) {
      if (ln == 0) set_err(err, DERR_NOT_SPD);
      p = F(1);
    }
    // 1/sqrt(p): FP32 seed, then two Newton steps in FP64 (relative error 1e-7 -> 1e-14 ->
    // rounding), far shorter on the FP64 pipe than a sqrt and a division; pivots outside the
    // FP32 range take the sqrt and the division
    F rd;
    if (sizeof(F) == 4) {
      rd = F(rsqrtf((float)p));
    } else if (p > F(1e-30) && p < F(1e30)) {
      rd = F(rsqrtf((float)p));
      rd = rd * (F(1.5) - F(0.5) * p * rd * rd);
      rd = rd * (F(1.5) - F(0.5) * p * rd * rd);
    } else {
      rd = F(1) / sqrt(p);
    }
    const F d = p * rd;
    __syncwarp();
    if (ln == j) { T[j][j] = d; rdiag[j] = rd; }
    if (ln > j) T[ln][j] *= rd;
    __syncwarp();
    if (ln > j) {
      const F lij = T[ln][j];
      for (int c = j + 1; c <= ln; ++c) T[ln][c] -= lij * T[c][j];
    }
    __syncwarp();
  }
  // column ln of L^-1 by forward substitution (each lane owns one column)
  for (int i = 0; i < kNB; ++i) {
    F x = F(0);
    if (i >= ln) {
      F s = F(i == ln ? 1 : 0);
      for (int m = ln; m < i; ++m) s -= T[i][m] * X[m][ln];
      x = s * rdiag[i];
    }
    X[i][ln] = x;
  }
  __syncwarp();
  F* D = Dblk + (size_t)(k0 / kNB) * kNB * kNB;
  for (int i = 0; i < kNB; ++i) {
    D[i * kNB + ln] = X[i][ln];
    if (i < nb && ln < nb) M[(size_t)(k0 + i) * n + k0 + ln] = ln <= i ? T[i][ln] : F(0);
  }
}

template <typename F>
__global__ void __launch_bounds__(256)
k_chol_panel(F* M, int n, int k0, const F* __restrict__ Dblk) {
  __shared__ F D[kNB][kNB + 1], A[8][kNB + 1];
  const int nb = min(kNB, n - k0);
  const F* Dk = Dblk + (size_t)(k0 / kNB) * kNB * kNB;
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) D[e / kNB][e % kNB] = Dk[e];
  const int tr = threadIdx.x >> 5, tc = threadIdx.x & 31;
  for (int rb = k0 + nb + blockIdx.x * 8; rb < n; rb += gridDim.x * 8) {
    __syncthreads();
    const int r = rb + tr;
    A[tr][tc] = (r < n && tc < nb) ? M[(size_t)r * n + k0 + tc] : F(0);
    __syncthreads();
    if (r < n && tc < nb) {
      F s = F(0);
      for (int m = 0; m <= tc; ++m) s = fma(A[tr][m], D[tc][m], s);
      M[(size_t)r * n + k0 + tc] = s;
    }
  }
}

// Trailing update of the lower triangle: M[i][j] -= sum_k L[i][k] L[j][k], i, j >= k1.
template <typename F>
__global__ void k_chol_update(F* M, int n, int k0, int k1) {
  __shared__ F Li[16][kNB + 1], Lj[16][kNB + 1];
  const int ti = blockIdx.y * 16, tj = blockIdx.x * 16;
  if (tj > ti + 15) return;     // tile strictly above the diagonal
  const int nb = k1 - k0;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int e = ty * 16 + tx; e < 16 * kNB; e += 256) {
    const int r = e / kNB, k = e % kNB;
    const int gi = k1 + ti + r, gj = k1 + tj + r;
    Li[r][k] = (gi < n && k < nb) ? M[(size_t)gi * n + k0 + k] : F(0);
    Lj[r][k] = (gj < n && k < nb) ? M[(size_t)gj * n + k0 + k] : F(0);
  }
  __syncthreads();
  const int i = k1 + ti + ty, j = k1 + tj + tx;
  if (i < n && j < n && j <= i) {
    F s = F(0);
    for (int k = 0; k < nb; ++k) s += Li[ty][k] * Lj[tx][k];
    M[(size_t)i * n + j] -= s;
  }
}

// X = L^-1 by recursive doubling. The diagonal 32 x 32 blocks of X are the inverted blocks
// Dinv_k; then, for s = 32, 64, ..., every pair of neighbouring inverted diagonal blocks of
// size s (rows/columns [p, p + s) and [p + s, p + s + s2), p = 2 s z) is merged into one of
// size s + s2 by the block formula X21 = -X22 L21 X11, in two tile products per pair:
//   step 1: T = L21 X11   (X11 lower: output column tile ct needs k >= 32 ct only)
//   step 2: X21 = -X22 T  (X22 lower: output row tile rt needs k < 32 (rt + 1) only)
// All pairs of a level run in one launch (blockIdx.z), so every launch fills the GPU with
// 32 x 32 output tiles; thread (ty, tx) owns rows ty, ty + 8, ty + 16, ty + 24 of column tx.
template <typename F>
__global__ void __launch_bounds__(256)
k_inv_diag_blocks(int n, const F* __restrict__ Dblk, F* __restrict__ X) {
  const int b = blockIdx.x, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const F* D = Dblk + (size_t)b * kNB * kNB;
  for (int q = 0; q < 4; ++q) {
    const int r = ty + 8 * q;
    if (b * kNB + r < n && b * kNB + tx < n)
      X[(size_t)(b * kNB + r) * n + b * kNB + tx] = D[r * kNB + tx];
  }
}

template <int STEP, typename F>
__global__ void __launch_bounds__(256)
k_inv_merge(const F* __restrict__ L, F* __restrict__ X, F* __restrict__ T, int n, int s) {
  __shared__ F As[kNB][kNB + 1], Bs[kNB][kNB + 1];
  const int p = blockIdx.z * 2 * s;
  const int s2 = min(s, n - p - s);
  const int rt = blockIdx.y, ct = blockIdx.x;
  if (s2 <= 0 || rt * kNB >= s2) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int kb = STEP == 1 ? ct * kNB : 0;
  const int ke = STEP == 1 ? s : min(s2, (rt + 1) * kNB);
  const F* A = STEP == 1 ? L : X;                // rows p + s + ..., k-columns from a0
  const F* B = STEP == 1 ? X : T;                // k-rows from a0, columns p + ...
  const int a0 = STEP == 1 ? p : p + s;
  const int r0 = p + s + rt * kNB, c0 = p + ct * kNB;
  const bool col_ok = ct * kNB + tx < s;
  F acc[4] = {F(0), F(0), F(0), F(0)};
  for (int k0 = kb; k0 < ke; k0 += kNB) {
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
      const int rr = ty + 8 * q;
      As[rr][tx] = (rt * kNB + rr < s2 && k0 + tx < ke)
                       ? A[(size_t)(r0 + rr) * n + a0 + k0 + tx] : F(0);
      Bs[rr][tx] = (k0 + rr < ke && col_ok) ? B[(size_t)(a0 + k0 + rr) * n + c0 + tx] : F(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int m = 0; m < kNB; ++m) {
      const F bv = Bs[m][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(As[ty + 8 * q][m], bv, acc[q]);
    }
  }
  for (int q = 0; q < 4; ++q) {
    const int rr = ty + 8 * q;
    if (rt * kNB + rr < s2 && col_ok) {
      const size_t idx = (size_t)(r0 + rr) * n + c0 + tx;
      if (STEP == 1) T[idx] = acc[q]; else X[idx] = -acc[q];
    }
  }
}

// Ainv = X^T X with X = L^-1 lower: Ainv[i][j] = sum_{k >= max(i, j)} X[k][i] X[k][j]. Lower
// tiles are computed and mirrored, so Ainv is exactly symmetric.
template <typename F>
__global__ void k_xtx(const F* __restrict__ X, int n, F* __restrict__ Ainv) {
  __shared__ F A[16][17], B[16][17];
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
  if (j0 > i0) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  F s = F(0);
  for (int k0 = i0; k0 < n; k0 += 16) {
    A[ty][tx] = (k0 + ty < n && i0 + tx < n) ? X[(size_t)(k0 + ty) * n + i0 + tx] : F(0);
    B[ty][tx] = (k0 + ty < n && j0 + tx < n) ? X[(size_t)(k0 + ty) * n + j0 + tx] : F(0);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) s = fma(A[k][ty], B[k][tx], s);
    __syncthreads();
  }
  const int i = i0 + ty, j = j0 + tx;
  if (i < n && j < n && j <= i) {
    Ainv[(size_t)i * n + j] = s;
    Ainv[(size_t)j * n + i] = s;
  }
}

}  // namespace rmg
