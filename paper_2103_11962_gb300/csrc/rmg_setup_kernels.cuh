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
  __device__ void operator()(int n, double s) const { dinv[n] = 1.0 / s; }
};

// ------------------------------------------------------------------ Galerkin product
// [[Abar]] = [[R]] [[A]] [[P]] for one coarse node per thread (eq. RegionalGalerkinProduct),
// evaluated region-locally from the definition: sum over the fine nodes f in the support of
// the coarse basis function, their stencil neighbours f', and the coarse nodes C' that f'
// interpolates from. Masked fine nodes have zero P rows, masked coarse nodes zero P
// columns; a masked coarse row becomes 1/mult on the diagonal.
constexpr int kRapBS = 128;

template <int FK, int CK, int DIM>
__global__ void __launch_bounds__(kRapBS)
k_rap(int cn_r, const RegionDev* __restrict__ cregs, int nreg, const RegionDev* __restrict__ fregs,
      const double* __restrict__ fcoef, int fn_r, const uint8_t* __restrict__ fmask,
      const uint8_t* __restrict__ cmask, const uint8_t* __restrict__ cmult,
      double* __restrict__ ccoef) {
  using FS = Sten<FK>;
  using CS = Sten<CK>;
  __shared__ double acc[CS::S][kRapBS];
  const int tid = threadIdx.x;
  for (int base = blockIdx.x * kRapBS; base < cn_r; base += gridDim.x * kRapBS) {
    const int C = base + tid;
    const bool live = C < cn_r;
#pragma unroll
    for (int s = 0; s < CS::S; ++s) acc[s][tid] = 0.0;
    if (live) {
      const int k = region_of(cregs, nreg, C);
      const RegionDev Cr = cregs[k];
      const RegionDev F = fregs[k];
      int I, J, L;
      decode(C - Cr.off, Cr, I, J, L);
      if (cmask[C]) {
        acc[CS::CENTER][tid] = 1.0 / (double)cmult[C];
      } else {
        const int zlo = DIM == 3 ? -2 : 0, zhi = DIM == 3 ? 2 : 0;
        for (int c = zlo; c <= zhi; ++c) {
          const int fz = 3 * L + c;
          if (fz < 0 || fz >= F.nz) continue;
          const double wz = DIM == 3 ? w1d(c) : 1.0;
          for (int b = -2; b <= 2; ++b) {
            const int fy = 3 * J + b;
            if (fy < 0 || fy >= F.ny) continue;
            const double wy = w1d(b);
            for (int a = -2; a <= 2; ++a) {
              const int fx = 3 * I + a;
              if (fx < 0 || fx >= F.nx) continue;
              const int f = F.off + fx + F.nx * (fy + F.ny * fz);
              if (fmask[f]) continue;
              const double wf = wz * (wy * w1d(a));
#pragma unroll
              for (int s = 0; s < FS::S; ++s) {
                const int gx = fx + FS::dx(s), gy = fy + FS::dy(s), gz = fz + FS::dz(s);
                if (gx < 0 || gx >= F.nx || gy < 0 || gy >= F.ny || gz < 0 || gz >= F.nz) continue;
                const double v = fcoef[(size_t)s * fn_r + f];
                if (v == 0.0) continue;
                const int f2 = F.off + gx + F.nx * (gy + F.ny * gz);
                if (fmask[f2]) continue;
                const double wv = wf * v;
                // coarse nodes that f2 interpolates from
                const int x0 = gx / 3, rx = gx - 3 * x0;
                const int y0 = gy / 3, ry = gy - 3 * y0;
                const int z0 = gz / 3, rz = gz - 3 * z0;
                const int nxs = rx ? 2 : 1, nys = ry ? 2 : 1, nzs = (DIM == 3 && rz) ? 2 : 1;
                for (int zc = 0; zc < nzs; ++zc) {
                  const double wcz = DIM == 3 ? (rz ? (zc ? rz / 3.0 : 1.0 - rz / 3.0) : 1.0) : 1.0;
                  const int Z = z0 + zc;
                  for (int yc = 0; yc < nys; ++yc) {
                    const double wcy = ry ? (yc ? ry / 3.0 : 1.0 - ry / 3.0) : 1.0;
                    const int Y = y0 + yc;
                    for (int xc = 0; xc < nxs; ++xc) {
                      const double wcx = rx ? (xc ? rx / 3.0 : 1.0 - rx / 3.0) : 1.0;
                      const int X = x0 + xc;
                      const int Cn = Cr.off + X + Cr.nx * (Y + Cr.ny * Z);
                      if (cmask[Cn]) continue;
                      const int slot = sten_slot<CK>(X - I, Y - J, DIM == 3 ? Z - L : 0);
                      acc[slot][tid] += wv * (wcz * (wcy * wcx));
                    }
                  }
                }
              }
            }
          }
        }
      }
#pragma unroll
      for (int s = 0; s < CS::S; ++s) ccoef[(size_t)s * cn_r + C] = acc[s][tid];
    }
  }
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

__global__ void k_power_init(int n_r, const int* __restrict__ gid, const uint8_t* __restrict__ mask,
                             unsigned long long seed, double* __restrict__ x) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_r; k += gridDim.x * blockDim.x)
    x[k] = mask[k] ? 0.0 : splitmix_pm1(seed, (unsigned long long)gid[k]);
}

// out = sum of partials, then an operation on the scalar block.
enum FinOp : int { FIN_SQRT = 0, FIN_STORE = 1 };
__global__ void k_finalize(const double* __restrict__ partials, int np, double* __restrict__ dst,
                           int op) {
  const double s = sum_partials(partials, np);
  if (threadIdx.x == 0) *dst = (op == FIN_SQRT) ? sqrt(s) : s;
}

__global__ void k_scale_div(int n, const double* __restrict__ x, const double* __restrict__ nrm,
                            double* __restrict__ out) {
  const double d = *nrm;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    out[k] = x[k] / d;
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
// row of composite node g = sum over its regional copies of their region rows.
template <int KIND>
__global__ void k_coarse_assemble(int ncomp, int nc, const RegionDev* __restrict__ regs, int nreg,
                                  int n_r, const double* __restrict__ coef,
                                  const int* __restrict__ gid, const int* __restrict__ cidx,
                                  const int* __restrict__ c2r, const int* __restrict__ cgrp,
                                  const int* __restrict__ gptr, const int* __restrict__ gslot,
                                  double* __restrict__ M) {
  using S = Sten<KIND>;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ncomp; g += gridDim.x * blockDim.x) {
    const int row = cidx[g];
    if (row < 0) continue;
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
        M[(size_t)row * nc + col] += coef[(size_t)s * n_r + n];
      }
    }
  }
}

// Blocked right-looking Cholesky (lower), block width 32, in place in row-major M.
constexpr int kNB = 32;

__global__ void k_chol_diag(double* M, int n, int k0, int* err) {
  __shared__ double T[kNB][kNB + 1];
  const int nb = min(kNB, n - k0);
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int i = e / kNB, j = e % kNB;
    T[i][j] = (i < nb && j < nb) ? M[(size_t)(k0 + i) * n + k0 + j] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      const double p = T[j][j];
      if (!(p > 0.0)) { set_err(err, DERR_NOT_SPD); T[j][j] = 1.0; }
      else T[j][j] = sqrt(p);
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) T[i][j] /= T[j][j];
    __syncthreads();
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
      const int i = e / nb, c = e % nb;
      if (i > j && c > j && c <= i) T[i][c] -= T[i][j] * T[c][j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    M[(size_t)(k0 + i) * n + k0 + j] = (j <= i) ? T[i][j] : 0.0;
  }
}

__global__ void k_chol_panel(double* M, int n, int k0) {
  __shared__ double Lk[kNB][kNB + 1];
  const int nb = min(kNB, n - k0);
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int i = e / kNB, j = e % kNB;
    Lk[i][j] = (i < nb && j < nb) ? M[(size_t)(k0 + i) * n + k0 + j] : 0.0;
  }
  __syncthreads();
  for (int i = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double x[kNB];
    for (int j = 0; j < nb; ++j) {
      double a = M[(size_t)i * n + k0 + j];
      for (int k = 0; k < j; ++k) a -= x[k] * Lk[j][k];
      x[j] = a / Lk[j][j];
    }
    for (int j = 0; j < nb; ++j) M[(size_t)i * n + k0 + j] = x[j];
  }
}

// Trailing update of the lower triangle: M[i][j] -= sum_k L[i][k] L[j][k], i, j >= k1.
__global__ void k_chol_update(double* M, int n, int k0, int k1) {
  __shared__ double Li[16][kNB + 1], Lj[16][kNB + 1];
  const int ti = blockIdx.y * 16, tj = blockIdx.x * 16;
  if (tj > ti + 15) return;     // tile strictly above the diagonal
  const int nb = k1 - k0;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int e = ty * 16 + tx; e < 16 * kNB; e += 256) {
    const int r = e / kNB, k = e % kNB;
    const int gi = k1 + ti + r, gj = k1 + tj + r;
    Li[r][k] = (gi < n && k < nb) ? M[(size_t)gi * n + k0 + k] : 0.0;
    Lj[r][k] = (gj < n && k < nb) ? M[(size_t)gj * n + k0 + k] : 0.0;
  }
  __syncthreads();
  const int i = k1 + ti + ty, j = k1 + tj + tx;
  if (i < n && j < n && j <= i) {
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += Li[ty][k] * Lj[tx][k];
    M[(size_t)i * n + j] -= s;
  }
}

// X = L^-1 (lower), one thread per column, X row-major (coalesced across columns).
__global__ void k_trinv(const double* __restrict__ L, int n, double* __restrict__ X) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    for (int i = 0; i < j; ++i) X[(size_t)i * n + j] = 0.0;
    for (int i = j; i < n; ++i) {
      double acc = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) acc -= L[(size_t)i * n + k] * X[(size_t)k * n + j];
      X[(size_t)i * n + j] = acc / L[(size_t)i * n + i];
    }
  }
}

// Ainv = X^T X (X = L^-1 lower triangular).
__global__ void k_xtx(const double* __restrict__ X, int n, double* __restrict__ Ainv) {
  __shared__ double A[16][17], B[16][17];
  const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
  double s = 0.0;
  const int kstart = (min(blockIdx.y, blockIdx.x) * 16);
  for (int k0 = kstart; k0 < n; k0 += 16) {
    const int kr = k0 + threadIdx.y;
    A[threadIdx.y][threadIdx.x] =
        (kr < n && blockIdx.y * 16 + threadIdx.x < n) ? X[(size_t)kr * n + blockIdx.y * 16 + threadIdx.x] : 0.0;
    B[threadIdx.y][threadIdx.x] = (kr < n && j < n) ? X[(size_t)kr * n + j] : 0.0;
    __syncthreads();
    for (int k = 0; k < 16; ++k) s += A[k][threadIdx.y] * B[k][threadIdx.x];
    __syncthreads();
  }
  if (i < n && j < n) Ainv[(size_t)i * n + j] = s;
}

}  // namespace rmg
