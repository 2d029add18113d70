// Hierarchy setup (regional mgSetup), the regional V-cycle (regional mgCycle) and PCG.
#include <chrono>
#include <cmath>

#include "rmg_hier.cuh"
#include "rmg_launch.cuh"
#include "rmg_layout.cuh"
#include "rmg_setup_kernels.cuh"

namespace rmg {

Hier::~Hier() {
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  if (graph_stream) cudaStreamDestroy(graph_stream);
  if (pinned) cudaFreeHost(pinned);
  for (auto e : probe_ev) if (e) cudaEventDestroy(e);
}

const int* Hier::half_flag() const { return &sc.get()->half_asym; }

// the mixed-precision dense coarse solve (defined with the coarse factorisation below)
static int mixed_coarse_solve(Hier& h, cudaStream_t st, int nd, int steps, double* nrm);

namespace {

template <typename T>
__global__ void k_copy(int n, const T* __restrict__ a, T* __restrict__ b) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) b[k] = a[k];
}

template <typename S, typename D>
__global__ void k_convert(size_t n, const S* __restrict__ a, D* __restrict__ b) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x)
    b[k] = D(a[k]);
}

__global__ void k_to_bf16(size_t n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x)
    b[k] = __float2bfloat16_rn(a[k]);
}

// coarse solve: gather the averaged composite right-hand side, x = Abar^-1 rhs, replicate
template <typename VT>
__global__ void k_coarse_gather(int nc, int B, int n_r, const VT* __restrict__ w,
                                const int* __restrict__ cu2slot, double* __restrict__ rc) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nc; k += gridDim.x * blockDim.x)
    for (int b = 0; b < B; ++b) rc[(size_t)k * B + b] = double(w[(size_t)b * n_r + cu2slot[k]]);
}

__global__ void k_gemv(int nc, const double* __restrict__ A, const double* __restrict__ v,
                       double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int i = warp; i < nc; i += nwarps) {
    double s = 0.0;
    const double* row = A + (size_t)i * nc;
    for (int j = lane; j < nc; j += 32) s = fma(row[j], v[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[i] = s;
  }
}

// ---- mixed-precision dense coarse solve ------------------------------------------------
// s_i = 1 / sqrt(Abar_ii): the symmetric diagonal scaling that takes the coefficient contrast
// out of the coarse matrix before it is factored in FP32.
__global__ void k_dense_scale(int nd, const double* __restrict__ A, double* __restrict__ s) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += gridDim.x * blockDim.x)
    s[i] = 1.0 / sqrt(A[(size_t)i * nd + i]);
}

// M = S A S rounded to FP32 (row blockIdx.y).
__global__ void k_dense_scaled32(int nd, const double* __restrict__ A,
                                 const double* __restrict__ s, float* __restrict__ M) {
  const int i = blockIdx.y;
  const double si = s[i];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nd; j += gridDim.x * blockDim.x)
    M[(size_t)i * nd + j] = (float)(si * A[(size_t)i * nd + j] * s[j]);
}

// w = FP32(s .* r * 2^-e) with 2^e near max |s_i r_i|, and back = 2^e: the FP32 solve then
// sees values of order one whatever the scale of r (no FP32 underflow or overflow), and the
// scaling is exact. One block of 1024 threads (the coarse dimension is at most 16384).
__global__ void __launch_bounds__(1024)
k_scale_vec32(int nd, const double* __restrict__ s, const double* __restrict__ r,
              float* __restrict__ w, double* __restrict__ back) {
  __shared__ double red[32];
  __shared__ double pw;
  double m = 0.0;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) m = fmax(m, fabs(s[i] * r[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) {
      const int e = (m > 0.0 && m <= 1.7e308) ? ilogb(m) : 0;
      pw = ldexp(1.0, -e);
      *back = ldexp(1.0, e);
    }
  }
  __syncthreads();
  const double p = pw;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) w[i] = (float)(s[i] * r[i] * p);
}

// x = s .* (M w) * back (accumulate = 0) or x += s .* (M w) * back: one warp per row, FP32
// products and sums; back undoes the power-of-two scaling of w.
__global__ void k_gemv32(int nd, const float* __restrict__ M, const float* __restrict__ w,
                         const double* __restrict__ s, const double* __restrict__ back,
                         double* __restrict__ x, int accumulate) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const double bk = *back;
  for (int i = warp; i < nd; i += nwarps) {
    float acc = 0.f;
    const float* row = M + (size_t)i * nd;
    for (int j = lane; j < nd; j += 32) acc = fmaf(row[j], w[j], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) x[i] = (accumulate ? x[i] : 0.0) + s[i] * ((double)acc * bk);
  }
}

// res = rc - A x in FP64: one warp per row.
__global__ void k_resid_dense(int nd, const double* __restrict__ A, const double* __restrict__ x,
                              const double* __restrict__ rc, double* __restrict__ res) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int i = warp; i < nd; i += nwarps) {
    double acc = 0.0;
    const double* row = A + (size_t)i * nd;
    for (int j = lane; j < nd; j += 32) acc = fma(row[j], x[j], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) res[i] = rc[i] - acc;
  }
}

// out[0] = sum v^2 (one block).
__global__ void k_norm2_dense(int nd, const double* __restrict__ v, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) acc = fma(v[i], v[i], acc);
  acc = block_sum<256>(acc);
  if (threadIdx.x == 0) out[0] = acc;
}

// SplitMix64 test vector for measuring the refinement's contraction.
__global__ void k_dense_random(int nd, unsigned long long seed, double* __restrict__ v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nd; i += gridDim.x * blockDim.x)
    v[i] = splitmix_pm1(seed, (unsigned long long)i);
}

template <typename VT>
__global__ void k_coarse_scatter(int n_r, int B, const int* __restrict__ gid,
                                 const int* __restrict__ cidx, const double* __restrict__ xc,
                                 VT* __restrict__ u) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_r; k += gridDim.x * blockDim.x) {
    const int c = cidx[gid[k]];
    for (int b = 0; b < B; ++b)
      u[(size_t)b * n_r + k] = c >= 0 ? VT(xc[(size_t)c * B + b]) : VT(0);
  }
}

// PCG scalar updates (single thread)
__global__ void k_alpha(Scalars* sc) { sc->alpha = sc->rz / sc->pq; }
__global__ void k_beta(Scalars* sc, int flexible) {
  // flexible (Polak-Ribiere) form: beta = r.(z - z_old) / rz_old, with r.z_old in sc->beta
  const double num = flexible ? sc->rz_new - sc->beta : sc->rz_new;
  sc->beta = num / sc->rz;
  sc->rz = sc->rz_new;
}

// x += alpha p, r -= alpha q, partial sums of r.r (all FP64).
__global__ void __launch_bounds__(256)
k_cg_update(int n, int n_nodes, const double* __restrict__ p, const double* __restrict__ q,
            const uint8_t* __restrict__ mult, const Scalars* __restrict__ sc,
            double* __restrict__ x, double* __restrict__ r, double* __restrict__ partials) {
  const double a = sc->alpha;
  double s = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    x[k] = x[k] + a * p[k];
    const double rk = r[k] - a * q[k];
    r[k] = rk;
    s = fma(rk * inv_mult<double>(mult[k < n_nodes ? k : k % n_nodes]), rk, s);
  }
  s = block_sum<256>(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Mixed-precision cycle. The FP32 (or BF16-coefficient) V-cycle is the preconditioner of a
// flexible CG that keeps x, r and p in FP64 and forms every inner product in FP64: r.r for the
// stopping test, r.z and r.z_old for alpha and beta. The cycle's right-hand side is the FP64
// residual times rscale = 2^-e, a power of two near 1/||b||, rounded to FP32: the scaling is
// exact and the cycle is linear, so its output is z / rscale and the iteration does not depend
// on the scale of b (without it, residual entries below ~1e-19 or above ~1e19 would underflow
// or overflow in FP32 squares and products). zscale = 1 / rscale undoes it (exactly).

// x += alpha p, r -= alpha q (FP64); r32 = FP32(r * rscale), the cycle's right-hand side;
// partial sums of r.r / mult in FP64.
__global__ void __launch_bounds__(256)
k_cg_update_mixed(int n, int n_nodes, const double* __restrict__ p, const double* __restrict__ q,
                  const uint8_t* __restrict__ mult, const Scalars* __restrict__ sc,
                  double rscale, double* __restrict__ x, double* __restrict__ r,
                  float* __restrict__ r32, double* __restrict__ partials) {
  const double a = sc->alpha;
  double s = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    x[k] = fma(a, p[k], x[k]);
    const double rk = fma(-a, q[k], r[k]);
    r[k] = rk;
    r32[k] = (float)(rk * rscale);
    s = fma(rk * inv_mult<double>(mult[k < n_nodes ? k : k % n_nodes]), rk, s);
  }
  s = block_sum<256>(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// r32 = FP32(r * rscale): the cycle's right-hand side at a (re)start of the iteration.
__global__ void k_to_f32_scaled(int n, const double* __restrict__ r, double rscale,
                                float* __restrict__ r32) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    r32[k] = (float)(r[k] * rscale);
}

// Partial sums of r.z and r.z_old in FP64 (the FP32 values convert exactly), times zscale;
// the FP32 cycle output z then becomes z_old. Partials of r.z go to partials[0, gridDim), those
// of r.z_old to partials[gridDim, 2 gridDim). Four consecutive FP32 entries per thread step
// (16-byte loads); the entries past the last multiple of four take a scalar tail.
__global__ void __launch_bounds__(256)
k_flex_dots(int n, int n_nodes, const double* __restrict__ r, const float* __restrict__ z,
            float* __restrict__ zold, const uint8_t* __restrict__ mult, double zscale,
            double* __restrict__ partials) {
  double s0 = 0.0, s1 = 0.0;
  const int n4 = n >> 2;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  auto im_of = [&](int k) { return inv_mult<double>(mult[k < n_nodes ? k : k % n_nodes]); };
  auto term = [&](int k, float zk, float ok) {
    const double rk = r[k] * im_of(k);
    s0 = fma(rk, (double)zk, s0);
    s1 = fma(rk, (double)ok, s1);
  };
  for (int q = tid; q < n4; q += nth) {
    const float4 zv = reinterpret_cast<const float4*>(z)[q];
    const float4 ov = reinterpret_cast<const float4*>(zold)[q];
    const int k = 4 * q;
    term(k, zv.x, ov.x);
    term(k + 1, zv.y, ov.y);
    term(k + 2, zv.z, ov.z);
    term(k + 3, zv.w, ov.w);
    reinterpret_cast<float4*>(zold)[q] = zv;
  }
  for (int k = 4 * n4 + tid; k < n; k += nth) {
    term(k, z[k], zold[k]);
    zold[k] = z[k];
  }
  s0 = block_sum<256>(s0 * zscale);
  s1 = block_sum<256>(s1 * zscale);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s0;
    partials[gridDim.x + blockIdx.x] = s1;
  }
}

// First direction after a (re)start: partial sums of r.z in FP64, p = z * zscale (FP64),
// z_old = z.
__global__ void __launch_bounds__(256)
k_start_dir(int n, int n_nodes, const double* __restrict__ r, const float* __restrict__ z,
            const uint8_t* __restrict__ mult, double zscale, double* __restrict__ p,
            float* __restrict__ zold, double* __restrict__ partials) {
  double s = 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const float zk = z[k];
    const double zd = (double)zk * zscale;
    s = fma(r[k] * inv_mult<double>(mult[k < n_nodes ? k : k % n_nodes]), zd, s);
    p[k] = zd;
    zold[k] = zk;
  }
  s = block_sum<256>(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_axpy_neg(int n, const double* __restrict__ z, double* __restrict__ e) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    e[k] -= z[k];
}

// p = z * zscale + beta p (zscale = 1 for the FP64 cycle).
template <typename ZT>
__global__ void k_p_update(int n, const ZT* __restrict__ z, double zscale,
                           const Scalars* __restrict__ sc, double* __restrict__ p) {
  const double b = sc->beta;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    p[k] = fma(double(z[k]), zscale, b * p[k]);
}

// Composite inner product of consistent regional vectors with n entries (B components of
// n_nodes nodes each, component-major).
void dot(Ctx& c, int n, int n_nodes, const double* x, const double* y, const uint8_t* mult,
         double* dst, int op, cudaStream_t st) {
  const int g = std::min(c.max_partials, persistent_grid(c, (n + 255) / 256));
  k_dot<double, double><<<g, 256, 0, st>>>(n, n_nodes, x, y, mult, c.partials.get());
  RMG_LAUNCHED();
  k_finalize<<<1, 256, 0, st>>>(c.partials.get(), g, dst, op);
  RMG_LAUNCHED();
}

// ---------------------------------------------------------------------- V-cycle executor
template <typename VT, typename CT>
struct Exec {
  Hier& h;
  cudaStream_t st;
  int launches = 0;
  bool probe = false;        // time the next level-0 phase-A launch with the probe events
  std::vector<VT*> cur, oth;

  Exec(Hier& hh, cudaStream_t s) : h(hh), st(s) {}

  LevelVecs<VT>& V(int l);
  const CT* coef(int l) const;
  const VT* dinv(int l) const;
  Scalars* sc() const { return h.sc.get(); }
  Ctx& c() const { return *h.c; }
  void flip(int l) { std::swap(cur[l], oth[l]); }

  template <class Epi>
  void stencil(int l, const VT* u, Epi epi) {
    const bool pr = probe && l == 0 && h.probe_ev[0];
    launch_stencil(c(), *h.lv[l], coef(l), u, V(l).y.get(), epi, st, &launches,
                   pr ? h.probe_ev[0] : nullptr, pr ? h.probe_ev[1] : nullptr, h.sweep(l),
                   h.half(l), h.half_flag());
    if (pr) probe = false;
  }

  int elementwise_grid(int n) const { return persistent_grid(c(), (n + 255) / 256); }

  // Chebyshev coefficients of level l, step k, in the cycle's precision
  const VT* c1(int l, int k) const;
  const VT* c2(int l, int k) const;

  void cheb_step(int l, int k, bool probe_it = false) {   // k >= 1
    probe = probe_it;
    EpiCheb<VT> e{cur[l], V(l).b.get(), dinv(l), c1(l, k), c2(l, k), V(l).d.get(), oth[l]};
    stencil(l, cur[l], e);
    flip(l);
  }

  // One colour class of the region Gauss-Seidel on level l.
  void gs_colour(int l, int colour, VT omega) {
    const Level& L = *h.lv[l];
    const Grid G = h.sweep(l) ? *h.sweep(l) : L.grid();
    const int gb = persistent_grid(c(), G.ntiles);
    VT* u = cur[l];
#define RMG_GS(K)                                                                             \
  k_gs_colour<K, CT, VT><<<gb, kTile, 0, st>>>(G, coef(l), V(l).r.get(), dinv(l),               \
                                               V(l).d.get(), u, colour, omega)
    switch (L.kind) {
      case 5: RMG_GS(5); break;
      case 7: RMG_GS(7); break;
      case 9: RMG_GS(9); break;
      default: RMG_GS(27); break;
    }
#undef RMG_GS
    RMG_LAUNCHED();
    ++launches;
  }

  void smooth(int l, int nu, bool from_zero, bool probe_it = false, bool post = false) {
    const Level& L = *h.lv[l];
    const int n = L.B * L.n_r;
    const VT omega = VT(h.o.omega);
    if (h.o.smoother == RMG_SMOOTHER_GS) {
      const int ncol = (L.kind == 5 || L.kind == 7) ? 2 : (L.dim == 3 ? 8 : 4);
      for (int s = 0; s < nu; ++s) {
        if (s == 0 && from_zero) {
          k_gs_zero<VT><<<elementwise_grid(n), 256, 0, st>>>(n, V(l).b.get(), V(l).r.get(),
                                                             V(l).d.get(), cur[l]);
          RMG_LAUNCHED();
          ++launches;
        } else {
          probe = probe_it && s == 0;
          stencil(l, cur[l], EpiResidZero<VT>{V(l).b.get(), V(l).r.get(), V(l).d.get()});
        }
        for (int k = 0; k < ncol; ++k) gs_colour(l, post ? ncol - 1 - k : k, omega);
      }
      return;
    }
    if (h.o.smoother == RMG_SMOOTHER_JACOBI) {
      for (int s = 0; s < nu; ++s) {
        if (s == 0 && from_zero) {
          k_jacobi_zero<VT><<<elementwise_grid(n), 256, 0, st>>>(n, V(l).b.get(), dinv(l), omega,
                                                                 oth[l]);
          RMG_LAUNCHED();
          ++launches;
        } else {
          probe = probe_it && s == 0;
          stencil(l, cur[l], EpiJacobi<VT>{cur[l], V(l).b.get(), dinv(l), omega, oth[l]});
        }
        flip(l);
      }
    } else {
      for (int a = 0; a < nu; ++a) {
        if (a == 0 && from_zero) {
          k_cheb0_zero<VT><<<elementwise_grid(n), 256, 0, st>>>(n, V(l).b.get(), dinv(l),
                                                                c2(l, 0), V(l).d.get(), oth[l]);
          RMG_LAUNCHED();
          ++launches;
        } else {
          probe = probe_it && a == 0 && h.o.cheb_degree == 1;
          stencil(l, cur[l], EpiCheb0<VT>{cur[l], V(l).b.get(), dinv(l), c2(l, 0),
                                          V(l).d.get(), oth[l]});
        }
        flip(l);
        for (int k = 1; k < h.o.cheb_degree; ++k) cheb_step(l, k, probe_it && a == 0 && k == 1);
      }
    }
  }

  // r = ([[b]] - Psi^T Psi [[A]] [[u]]) / mult: the regional residual already carrying the
  // [[Psi Psi^T]]^-1 scaling of the restriction
  void residual(int l) { stencil(l, cur[l], EpiResidScaled<VT>{V(l).b.get(), V(l).r.get()}); }

  const float* pw(int l) const { return h.pw[l].get(); }

  void restrict_to(int l) {
    const Level& F = *h.lv[l];
    const Level& C = *h.lv[l + 1];
    if (F.B > 1) {   // B x B block operators: the scalar transfer on every component
      const Grid Gc = C.grid();
      const int gb = persistent_grid(c(), Gc.ntiles);
      for (int b = 0; b < F.B; ++b) {
        VT* wb = V(l + 1).b.get() + (size_t)b * C.n_r;
        VT* yb = V(l + 1).y.get() + (size_t)b * C.n_r;
        const VT* rb = V(l).r.get() + (size_t)b * F.n_r;
        k_restrict<3, VT><<<gb, kTile, 0, st>>>(Gc, F.regions.get(), rb, C.mask.get(),
                                                C.mult.get(), wb, yb);
        RMG_LAUNCHED();
        ++launches;
        if (C.ngroups) {
          launch_groups(c(), C, (const VT*)yb, EpiStore<VT>{wb}, st);
          ++launches;
        }
      }
      return;
    }
    const Grid Gc = C.grid();
    const int gb = persistent_grid(c(), Gc.ntiles);
    if (h.stored[l]) {
      if (F.dim == 3)
        k_restrict_w<3, VT><<<gb, kTile, 0, st>>>(Gc, F.regions.get(), F.n_r, pw(l), V(l).r.get(),
                                                  C.mask.get(), C.mult.get(), V(l + 1).b.get(),
                                                  V(l + 1).y.get());
      else
        k_restrict_w<2, VT><<<gb, kTile, 0, st>>>(Gc, F.regions.get(), F.n_r, pw(l), V(l).r.get(),
                                                  C.mask.get(), C.mult.get(), V(l + 1).b.get(),
                                                  V(l + 1).y.get());
    } else if (F.dim == 3)
      k_restrict<3, VT><<<gb, kTile, 0, st>>>(Gc, F.regions.get(), V(l).r.get(), C.mask.get(),
                                              C.mult.get(), V(l + 1).b.get(), V(l + 1).y.get());
    else
      k_restrict<2, VT><<<gb, kTile, 0, st>>>(Gc, F.regions.get(), V(l).r.get(), C.mask.get(),
                                              C.mult.get(), V(l + 1).b.get(), V(l + 1).y.get());
    RMG_LAUNCHED();
    ++launches;
    if (C.ngroups) {
      launch_groups(c(), C, (const VT*)V(l + 1).y.get(), EpiStore<VT>{V(l + 1).b.get()}, st);
      ++launches;
    }
  }

  void prolong(int l) {
    const Level& F = *h.lv[l];
    const Level& C = *h.lv[l + 1];
    const Grid Gf = F.grid();
    const int gb = persistent_grid(c(), Gf.ntiles);
    if (F.B > 1) {
      for (int b = 0; b < F.B; ++b) {
        k_prolong<3, VT><<<gb, kTile, 0, st>>>(Gf, C.regions.get(), F.mask.get(),
                                               cur[l + 1] + (size_t)b * C.n_r,
                                               cur[l] + (size_t)b * F.n_r);
        RMG_LAUNCHED();
        ++launches;
      }
      return;
    }
    if (h.stored[l]) {
      if (F.dim == 3)
        k_prolong_w<3, VT><<<gb, kTile, 0, st>>>(Gf, C.regions.get(), pw(l), F.mask.get(),
                                                 cur[l + 1], cur[l]);
      else
        k_prolong_w<2, VT><<<gb, kTile, 0, st>>>(Gf, C.regions.get(), pw(l), F.mask.get(),
                                                 cur[l + 1], cur[l]);
    } else if (F.dim == 3)
      k_prolong<3, VT><<<gb, kTile, 0, st>>>(Gf, C.regions.get(), F.mask.get(), cur[l + 1], cur[l]);
    else
      k_prolong<2, VT><<<gb, kTile, 0, st>>>(Gf, C.regions.get(), F.mask.get(), cur[l + 1], cur[l]);
    RMG_LAUNCHED();
    ++launches;
  }

  void coarse(int l) {
    const Level& L = *h.lv[l];
    const int nc = h.nc;
    if (nc > 0) {
      k_coarse_gather<VT><<<elementwise_grid(nc), 256, 0, st>>>(nc, L.B, L.n_r, V(l).b.get(),
                                                                h.cu2slot.get(), h.rc.get());
      RMG_LAUNCHED();
      const int nd = nc * L.B;
      if (h.coarse_refine > 0) {
        launches += 1 + mixed_coarse_solve(h, st, nd, h.coarse_refine, nullptr);
      } else {
        const int blocks = std::max(1, std::min(c().nsm * 4, (nd * 32 + 255) / 256));
        k_gemv<<<blocks, 256, 0, st>>>(nd, h.Ainv.get(), h.rc.get(), h.xc.get());
        RMG_LAUNCHED();
        launches += 2;
      }
    }
    k_coarse_scatter<VT><<<elementwise_grid(L.n_r), 256, 0, st>>>(L.n_r, L.B, L.gid.get(),
                                                                  h.cidx.get(), h.xc.get(), cur[l]);
    RMG_LAUNCHED();
    ++launches;
  }

  int level0_flips() const {
    if (h.o.smoother == RMG_SMOOTHER_GS) return 0;       // Gauss-Seidel updates u in place
    const int per = (h.o.smoother == RMG_SMOOTHER_JACOBI) ? 1 : h.o.cheb_degree;
    return (h.o.nu1 + h.o.nu2) * per;
  }

  void run() {
    const int Lv = h.levels();
    cur.assign(Lv, nullptr);
    oth.assign(Lv, nullptr);
    for (int l = 0; l < Lv; ++l) { cur[l] = V(l).u.get(); oth[l] = V(l).u2.get(); }
    if (Lv > 1 && (level0_flips() & 1)) std::swap(cur[0], oth[0]);
    for (int l = 0; l < Lv - 1; ++l) {
      smooth(l, h.o.nu1, true);
      residual(l);
      restrict_to(l);
    }
    coarse(Lv - 1);
    for (int l = Lv - 2; l >= 0; --l) {
      prolong(l);
      smooth(l, h.o.nu2, false, l == 0, true);
    }
    if (h.o.smoother == RMG_SMOOTHER_GS && Lv > 1) consistent_output();
  }

  // The cycle's output as a consistent regional vector: the copies of an interface node take
  // their mean, the composite value (Psi Psi^T)^-1 Psi u of the preconditioner's output.
  void consistent_output() {
    const Level& L = *h.lv[0];
    if (!L.ngroups) return;
    launch_groups(c(), L, (const VT*)cur[0], EpiMean<VT>{V(0).y.get()}, st);
    ++launches;
    k_copy_slots<VT><<<persistent_grid(c(), (L.nslots + 255) / 256), 256, 0, st>>>(
        L.nslots, L.gslot.get(), V(0).y.get(), cur[0]);
    RMG_LAUNCHED();
    ++launches;
  }
};

template <> const double* Exec<double, double>::c1(int l, int k) const { return &h.sc.get()->cheb_c1[l][k]; }
template <> const double* Exec<double, double>::c2(int l, int k) const { return &h.sc.get()->cheb_c2[l][k]; }
template <> const float* Exec<float, float>::c1(int l, int k) const { return &h.sc.get()->cheb_c1f[l][k]; }
template <> const float* Exec<float, float>::c2(int l, int k) const { return &h.sc.get()->cheb_c2f[l][k]; }
template <> const float* Exec<float, __nv_bfloat16>::c1(int l, int k) const { return &h.sc.get()->cheb_c1f[l][k]; }
template <> const float* Exec<float, __nv_bfloat16>::c2(int l, int k) const { return &h.sc.get()->cheb_c2f[l][k]; }
template <> LevelVecs<double>& Exec<double, double>::V(int l) { return h.v64[l]; }
template <> const double* Exec<double, double>::coef(int l) const { return h.lv[l]->coef.get(); }
template <> const double* Exec<double, double>::dinv(int l) const { return h.lv[l]->dinv.get(); }
template <> LevelVecs<float>& Exec<float, float>::V(int l) { return h.v32[l]; }
template <> const float* Exec<float, float>::coef(int l) const { return h.lv[l]->coef32.get(); }
template <> const float* Exec<float, float>::dinv(int l) const { return h.lv[l]->dinv32.get(); }
template <> LevelVecs<float>& Exec<float, __nv_bfloat16>::V(int l) { return h.v32[l]; }
template <> const __nv_bfloat16* Exec<float, __nv_bfloat16>::coef(int l) const {
  return h.lv[l]->coef16.get();
}
template <> const float* Exec<float, __nv_bfloat16>::dinv(int l) const {
  return h.lv[l]->dinv32.get();
}

int run_cycle(Hier& h, cudaStream_t st) {
  if (h.o.precision == RMG_PREC_FP64) {
    Exec<double, double> e(h, st);
    e.run();
    return e.launches;
  } else if (h.o.precision == RMG_PREC_FP32) {
    Exec<float, float> e(h, st);
    e.run();
    return e.launches;
  } else {
    Exec<float, __nv_bfloat16> e(h, st);
    e.run();
    return e.launches;
  }
}

}  // namespace

// ---------------------------------------------------------------------- setup
static void coarsen_level(Hier& h, const Level& F, Level& C) {
  Ctx& c = *h.c;
  std::vector<int> cd(3 * F.nreg);
  for (int r = 0; r < F.nreg; ++r)
    for (int a = 0; a < 3; ++a) {
      const int n = F.hdims[3 * r + a];
      if (n == 1 && (F.dim == 2 && a == 2)) { cd[3 * r + a] = 1; continue; }
      RMG_REQUIRE(n >= 4 && (n - 1) % 3 == 0, RMG_ERR_LAYOUT,
                  "region " + std::to_string(r) + " has " + std::to_string(n) +
                      " nodes along an axis; 3:1 coarsening needs 3k+1 with k >= 1");
      cd[3 * r + a] = (n - 1) / 3 + 1;
    }
  set_geometry(C, F.dim, F.nreg, cd.data());
  DBuf<int> flag(F.ncomp), sel(F.ncomp), cid(F.ncomp);
  RMG_CUDA(cudaMemsetAsync(flag.get(), 0, flag.bytes(), c.stream));
  const Grid Gf = F.grid();
  k_coarse_flags<<<persistent_grid(c, Gf.ntiles), kTile, 0, c.stream>>>(Gf, F.dim, F.gid.get(),
                                                                         flag.get());
  RMG_LAUNCHED();
  k_coarse_select<<<persistent_grid(c, (F.ncomp + 255) / 256), 256, 0, c.stream>>>(
      F.ncomp, flag.get(), sel.get(), c.d_err.get());
  RMG_LAUNCHED();
  C.ncomp = exclusive_scan(c, sel.get(), cid.get(), F.ncomp);
  c.check_device_error("rmg_setup");
  C.gid.alloc(C.n_r);
  DBuf<uint8_t> cmask(C.n_r);
  DBuf<int> count(C.ncomp);
  RMG_CUDA(cudaMemsetAsync(count.get(), 0, count.bytes(), c.stream));
  const Grid Gc = C.grid();
  k_coarse_gids<<<persistent_grid(c, Gc.ntiles), kTile, 0, c.stream>>>(
      Gc, F.dim, F.regions.get(), F.gid.get(), F.mask.get(), cid.get(), C.gid.get(), cmask.get(),
      count.get());
  RMG_LAUNCHED();
  build_groups(c, C, nullptr, cmask.get(), count);
  c.check_device_error("rmg_setup");
  C.kind = coarse_kind(F.kind);
  C.B = F.B;
  C.coef.alloc((size_t)C.B * C.B * C.kind * C.n_r);
}

void hier_build(Hier& h) {
  Ctx& c = *h.c;
  RMG_REQUIRE(h.layout->has_operator, RMG_ERR_STATE, "rmg_setup needs an operator on the layout");
  const rmg_options& o = h.o;
  RMG_REQUIRE(o.levels >= 1 && o.levels <= 16, RMG_ERR_ARG, "levels must be in [1, 16]");
  RMG_REQUIRE(o.nu1 >= 0 && o.nu2 >= 0 && o.nu1 + o.nu2 >= 0, RMG_ERR_ARG, "bad nu1/nu2");
  RMG_REQUIRE(o.smoother == RMG_SMOOTHER_JACOBI || o.smoother == RMG_SMOOTHER_CHEBYSHEV ||
                  o.smoother == RMG_SMOOTHER_GS,
              RMG_ERR_ARG, "unknown smoother");
  RMG_REQUIRE(o.cheb_degree >= 1 && o.cheb_degree <= 8, RMG_ERR_ARG, "cheb_degree in [1, 8]");
  RMG_REQUIRE(o.precision >= 0 && o.precision <= 2, RMG_ERR_ARG, "unknown precision");
  RMG_REQUIRE(o.tile_shape >= -1 && o.tile_shape < kNumTileShapes, RMG_ERR_ARG,
              "tile_shape must be -1 (autotune) or a shape index");
  RMG_REQUIRE(o.symmetric_storage == 0 || o.symmetric_storage == 1, RMG_ERR_ARG,
              "symmetric_storage must be 0 or 1");
  RMG_REQUIRE(o.eig_ratio > 1.0 && o.boost > 0.0 && o.power_iters >= 1 &&
              o.power_iters <= 100, RMG_ERR_ARG, "bad Chebyshev options");
  RMG_REQUIRE(o.smoother != RMG_SMOOTHER_GS || h.layout->L0.B == 1, RMG_ERR_ARG,
              "the region Gauss-Seidel smoother is for scalar operators");
  h.lv.push_back(&h.layout->L0);
  for (int l = 1; l < o.levels; ++l) {
    h.own.emplace_back(new Level());
    coarsen_level(h, *h.lv.back(), *h.own.back());
    h.lv.push_back(h.own.back().get());
  }
  const int Lv = h.levels();
  h.stored.assign(Lv, 0);
  h.pw.resize(Lv);
  h.shape.assign(Lv, -1);
  h.stiles.resize(Lv);
  h.sgrid.resize(Lv);
  h.v64.resize(Lv);
  for (int l = 0; l < Lv; ++l) {
    const size_t nb = (size_t)h.lv[l]->B * h.lv[l]->n_r;
    h.lv[l]->dinv.ensure(nb);   // level 0 belongs to the layout and may be shared
    h.v64[l].alloc((int)nb);
  }
  if (h.mixed()) {
    h.v32.resize(Lv);
    for (int l = 0; l < Lv; ++l) {
      Level& L = *h.lv[l];
      h.v32[l].alloc(L.B * L.n_r);
      L.dinv32.ensure((size_t)L.B * L.n_r);
      // FP32 coefficients on every level of a mixed hierarchy (the FP32 Galerkin chain runs
      // on them); the BF16 cycle reads its own copy
      L.coef32.ensure((size_t)L.B * L.B * L.kind * L.n_r);
      if (o.precision == RMG_PREC_FP32_BF16COEF) L.coef16.ensure((size_t)L.B * L.B * L.kind * L.n_r);
    }
  }
  // half planes for the FP32 cycle's level-0 sweeps of a scalar operator
  h.half_on = o.symmetric_storage != 0 && o.precision == RMG_PREC_FP32 && h.lv[0]->B == 1;
  if (Lv > 1) h.layout->apbuf.ensure((size_t)(h.lv[0]->dim == 3 ? 27 : 9) * h.lv[0]->n_r);
  h.sc.alloc(1);
  RMG_CUDA(cudaMemsetAsync(h.sc.get(), 0, sizeof(Scalars), c.stream));
  const int n0 = h.lv[0]->B * h.lv[0]->n_r;
  h.x.alloc(n0); h.p.alloc(n0); h.q.alloc(n0); h.tmp.alloc(n0);
  h.r.alloc(n0); h.z.alloc(n0); h.zold.alloc(n0);
  if (h.mixed()) h.zold32.alloc(n0);
  RMG_CUDA(cudaHostAlloc(&h.pinned, 64 * sizeof(double), cudaHostAllocDefault));
  RMG_CUDA(cudaEventCreate(&h.probe_ev[0]));
  RMG_CUDA(cudaEventCreate(&h.probe_ev[1]));
  // coarsest composite maps
  Level& Lc = *h.lv[Lv - 1];
  DBuf<int> freeflag(Lc.ncomp), pos(Lc.ncomp);
  k_coarse_free<<<persistent_grid(c, (Lc.ncomp + 255) / 256), 256, 0, c.stream>>>(
      Lc.ncomp, Lc.c2r.get(), Lc.mask.get(), freeflag.get());
  RMG_LAUNCHED();
  h.nc = exclusive_scan(c, freeflag.get(), pos.get(), Lc.ncomp);
  const long long ncd = (long long)h.nc * Lc.B;
  // a coarsest level above the dense solver's size leaves a hierarchy for setup and
  // introspection only (cycles fail with RMG_ERR_STATE)
  h.dense_ok = ncd <= kMaxDense;
  h.cidx.alloc(Lc.ncomp);
  h.cu2slot.alloc(std::max(1, h.nc));
  h.cu2gid.alloc(std::max(1, h.nc));
  k_coarse_maps<<<persistent_grid(c, (Lc.ncomp + 255) / 256), 256, 0, c.stream>>>(
      Lc.ncomp, freeflag.get(), pos.get(), Lc.c2r.get(), h.cidx.get(), h.cu2slot.get(),
      h.cu2gid.get());
  RMG_LAUNCHED();
  const size_t nd = h.dense_ok ? (size_t)std::max(1LL, ncd) : 1;
  const size_t nblk = (nd + kNB - 1) / kNB;
  h.Mfac.alloc(nd * nd); h.X.alloc(nd * nd); h.Ainv.alloc(nd * nd); h.Linv.alloc(nd * nd);
  h.Tinv.alloc(nd * nd);
  h.Dblk.alloc(nblk * kNB * kNB);
  h.M32.alloc(nd * nd); h.Ainv32.alloc(nd * nd); h.Linv32.alloc(nd * nd); h.Tinv32.alloc(nd * nd);
  h.Dblk32.alloc(nblk * kNB * kNB);
  h.cscale.alloc(nd); h.cres.alloc(nd); h.cw32.alloc(nd); h.cnorm.alloc(5); h.cerr.alloc(1);
  h.xc.alloc(nd); h.rc.alloc(nd);
  RMG_CUDA(cudaMemsetAsync(h.xc.get(), 0, h.xc.bytes(), c.stream));
  RMG_CUDA(cudaStreamSynchronize(c.stream));
}

// D~^-1 = (Psi^T Psi diag([[A]]))^-1, per component of a block operator (diagonal of A_cc).
static void compute_dinv(Hier& h, Level& L) {
  Ctx& c = *h.c;
  const int gb = persistent_grid(c, (L.n_r + 255) / 256);
  double* y = nullptr;
  for (int l = 0; l < h.levels(); ++l) if (h.lv[l] == &L) y = h.v64[l].y.get();
  for (int b = 0; b < L.B; ++b) {
    const double* cb = L.coef.get() + (size_t)(b * L.B + b) * L.kind * L.n_r;
    double* db = L.dinv.get() + (size_t)b * L.n_r;
    double* yb = y + (size_t)b * L.n_r;
    switch (L.kind) {
      case 5: k_diag_local<5><<<gb, 256, 0, c.stream>>>(L.n_r, cb, L.mult.get(), db, yb); break;
      case 7: k_diag_local<7><<<gb, 256, 0, c.stream>>>(L.n_r, cb, L.mult.get(), db, yb); break;
      case 9: k_diag_local<9><<<gb, 256, 0, c.stream>>>(L.n_r, cb, L.mult.get(), db, yb); break;
      default: k_diag_local<27><<<gb, 256, 0, c.stream>>>(L.n_r, cb, L.mult.get(), db, yb); break;
    }
    RMG_LAUNCHED();
    if (L.ngroups) {
      launch_groups(c, L, (const double*)yb, EpiRecip{db}, c.stream);
    }
  }
}

template <typename T>
static void galerkin_t(Hier& h, int l, const Level& F, Level& C, const T* fcoef, T* ccoef) {
  Ctx& c = *h.c;
  T* ap = reinterpret_cast<T*>(h.layout->apbuf.get());
  const Grid Gf = F.grid(), Gc = C.grid();
  const int gf = persistent_grid(c, Gf.ntiles), gc = persistent_grid(c, Gc.ntiles);
  // (P x I)^T A (P x I) of a B x B block operator is the scalar product on every block; a
  // masked coarse row is the identity row in the diagonal blocks and zero elsewhere
  for (int blk = 0; blk < F.B * F.B; ++blk) {
  const T* fco = fcoef + (size_t)blk * F.kind * F.n_r;
  T* cco = ccoef + (size_t)blk * C.kind * C.n_r;
  const double mdiag = (blk / F.B == blk % F.B) ? 1.0 : 0.0;
#define RMG_RAP(FK, CK, D)                                                                    \
  if (sizeof(T) == 4 && FK == 27 && D == 3) {                                                \
    const int ga = persistent_grid(c, Gf.ntiles, resident_per_sm((const void*)k_ap_tensor27)); \
    k_ap_tensor27<<<ga, kTile, 0, c.stream>>>(Gf, C.regions.get(), (const float*)fco,          \
                                              F.mask.get(), C.mask.get(), (float*)ap);        \
  } else if (sizeof(T) == 4) {                                                                \
    k_ap_axis32<FK, D><<<gf, kTile, 0, c.stream>>>(Gf, C.regions.get(), (const float*)fco,     \
                                                   F.mask.get(), C.mask.get(), (float*)ap);   \
  } else {                                                                                    \
    const int smem = (D == 3 ? 27 : 9) * kTile * (int)sizeof(T);                              \
    RMG_CUDA(cudaFuncSetAttribute(k_ap<FK, D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                  smem));                                                     \
    k_ap<FK, D, T><<<gf, kTile, smem, c.stream>>>(Gf, C.regions.get(), fco, F.mask.get(),        \
                                               C.mask.get(), ap);                             \
  }                                                                                           \
  RMG_LAUNCHED();                                                                             \
  k_rtap<CK, D, T><<<gc, kTile, 0, c.stream>>>(Gc, F.regions.get(), ap, F.n_r, C.mask.get(),     \
                                            C.mult.get(), mdiag, cco)
#define RMG_RAPW(FK, CK, D)                                                                   \
  {                                                                                           \
    const int smem = (D == 3 ? 27 : 9) * kTile * (int)sizeof(T);                         \
    RMG_CUDA(cudaFuncSetAttribute(k_ap_w<FK, D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                  smem));                                                     \
    k_ap_w<FK, D, T><<<gf, kTile, smem, c.stream>>>(Gf, C.regions.get(), fco, h.pw[l].get(),       \
                                                 F.mask.get(), C.mask.get(), ap);             \
  }                                                                                           \
  RMG_LAUNCHED();                                                                             \
  k_rtap_w<CK, D, T><<<gc, kTile, 0, c.stream>>>(Gc, F.regions.get(), ap, F.n_r, h.pw[l].get(),   \
                                              C.mask.get(), C.mult.get(), mdiag, cco)
  if (h.stored[l]) {
    switch (F.kind) {
      case 5: RMG_RAPW(5, 9, 2); break;
      case 9: RMG_RAPW(9, 9, 2); break;
      case 7: RMG_RAPW(7, 27, 3); break;
      default: RMG_RAPW(27, 27, 3); break;
    }
  } else {
    switch (F.kind) {
      case 5: RMG_RAP(5, 9, 2); break;
      case 9: RMG_RAP(9, 9, 2); break;
      case 7: RMG_RAP(7, 27, 3); break;
      default: RMG_RAP(27, 27, 3); break;
    }
  }
  RMG_LAUNCHED();
  }
#undef RMG_RAP
#undef RMG_RAPW
}

// Level l + 1 = Galerkin product of level l: in FP64 for the plain method; for a mixed
// hierarchy in FP32 on the FP32 coefficients, then widened to FP64 (exactly) for the dense
// coarse solve, the diagonal and introspection.
static void galerkin(Hier& h, int l, Level& F, Level& C) {
  if (!h.mixed()) {
    galerkin_t<double>(h, l, F, C, F.coef.get(), C.coef.get());
    return;
  }
  galerkin_t<float>(h, l, F, C, F.coef32.get(), C.coef32.get());
  const size_t nco = (size_t)C.B * C.B * C.kind * C.n_r;
  const int g = persistent_grid(*h.c, (int)std::min<size_t>((nco + 255) / 256, 1 << 20));
  k_convert<float, double><<<g, 256, 0, h.c->stream>>>(nco, C.coef32.get(), C.coef.get());
  RMG_LAUNCHED();
}

// Recompute the Galerkin product of level -> level + 1 alone (with the level's current
// transfer), as the numeric setup does it.
void galerkin_level(Hier& h, int level) {
  RMG_REQUIRE(level >= 0 && level + 1 < h.levels(), RMG_ERR_ARG,
              "Galerkin products exist for levels 0 .. levels-2");
  galerkin(h, level, *h.lv[level], *h.lv[level + 1]);
}

// Stored transfer weights for level -> level+1 (NULL restores linear interpolation). The
// numeric setup must run afterwards; it re-captures the V-cycle graph when the kind of
// transfer of a level changed.
void set_transfer_weights(Hier& h, int level, const float* wr) {
  RMG_REQUIRE(level >= 0 && level + 1 < h.levels(), RMG_ERR_ARG,
              "transfer weights exist for levels 0 .. levels-2");
  RMG_REQUIRE(h.lv[level]->B == 1 || !wr, RMG_ERR_ARG,
              "stored transfer weights are for scalar operators");
  Level& L = *h.lv[level];
  if (!wr) {
    h.stored[level] = 0;
    return;
  }
  h.pw[level].ensure((size_t)3 * L.n_r);
  RMG_CUDA(cudaMemcpyAsync(h.pw[level].get(), wr, h.pw[level].bytes(), cudaMemcpyDeviceToDevice,
                           h.c->stream));
  h.stored[level] = 1;
}

void constant_weights(Hier& h, int level, float* wr) {
  RMG_REQUIRE(level >= 0 && level < h.levels(), RMG_ERR_ARG, "bad level");
  Level& L = *h.lv[level];
  const Grid G = L.grid();
  k_constant_weights<<<persistent_grid(*h.c, G.ntiles), kTile, 0, h.c->stream>>>(G, L.dim, wr);
  RMG_LAUNCHED();
}

// Operator-dependent (series-resistance) weights of a level from its current operator.
void opdep_weights(Hier& h, int level, float* wr) {
  RMG_REQUIRE(level >= 0 && level < h.levels(), RMG_ERR_ARG, "bad level");
  RMG_REQUIRE(h.lv[level]->B == 1, RMG_ERR_ARG, "operator-dependent weights are for scalar operators");
  Level& L = *h.lv[level];
  Ctx& c = *h.c;
  const Grid G = L.grid();
  const int gb = persistent_grid(c, G.ntiles);
#define RMG_OPD(K)                                                                             \
  k_opdep<K><<<gb, kTile, 0, c.stream>>>(G, L.coef.get(), L.mult.get(), L.gid.get(),           \
                                         L.cgrp.get(), L.gptr.get(), L.gslot.get(), wr)
  switch (L.kind) {
    case 5: RMG_OPD(5); break;
    case 7: RMG_OPD(7); break;
    case 9: RMG_OPD(9); break;
    default: RMG_OPD(27); break;
  }
#undef RMG_OPD
  RMG_LAUNCHED();
}

// Composite inner product of two FP32 vectors (the mixed cycle's power method): FP32 products
// added in runs of 16 before the FP64 accumulation, four entries per thread step.
__global__ void __launch_bounds__(256)
k_dot_f32(int n, int n_nodes, const float* __restrict__ x, const float* __restrict__ y,
          const uint8_t* __restrict__ mult, double* __restrict__ partials) {
  double s = 0.0;
  float run = 0.f;
  const int n4 = n >> 2;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  auto im_of = [&](int k) { return inv_mult<float>(mult[k < n_nodes ? k : k % n_nodes]); };
  int cnt = 0;
  for (int q = tid; q < n4; q += nth) {
    const float4 a = reinterpret_cast<const float4*>(x)[q];
    const float4 b = reinterpret_cast<const float4*>(y)[q];
    const int k = 4 * q;
    run = fmaf(a.x * im_of(k), b.x, run);
    run = fmaf(a.y * im_of(k + 1), b.y, run);
    run = fmaf(a.z * im_of(k + 2), b.z, run);
    run = fmaf(a.w * im_of(k + 3), b.w, run);
    if (++cnt == 4) { s += (double)run; run = 0.f; cnt = 0; }
  }
  for (int k = 4 * n4 + tid; k < n; k += nth) run = fmaf(x[k] * im_of(k), y[k], run);
  s += (double)run;
  s = block_sum<256>(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Composite inner product of two consistent regional vectors of any precision (FP64 sums).
template <typename VT>
static void dot_t(Ctx& c, int n, int n_nodes, const VT* x, const VT* y, const uint8_t* mult,
                  double* dst, int op, cudaStream_t st) {
  const int g = std::min(c.max_partials, persistent_grid(c, (n + 255) / 256));
  if constexpr (sizeof(VT) == 4)
    k_dot_f32<<<g, 256, 0, st>>>(n, n_nodes, x, y, mult, c.partials.get());
  else
    k_dot<VT, VT><<<g, 256, 0, st>>>(n, n_nodes, x, y, mult, c.partials.get());
  RMG_LAUNCHED();
  k_finalize<<<1, 256, 0, st>>>(c.partials.get(), g, dst, op);
  RMG_LAUNCHED();
}

// lambda~_max(D~^-1 A) by the power method (Sec. 3.4), on the operator the cycle smooths with:
// FP64 coefficients for the plain method, the FP32 or BF16 copies for the mixed cycle. The
// start vector is normalised once; the power_iters steps y <- D~^-1 A y then run without
// normalising (the direction is the same as with a normalisation per step; the norm grows like
// lambda_max^k, and Gershgorin bounds lambda_max(D~^-1 A) by 1 + sum_j |a_ij| / a_ii, a few
// units for the stencils here, so 100 steps stay far inside the FP64 range). In FP32 the
// iterate is renormalised every 8 steps instead. The estimate is the Rayleigh quotient
// y^T D~^-1 A y / y^T y of the last iterate.
template <typename VT, typename CT>
static void power_method_t(Hier& h, int l) {
  Ctx& c = *h.c;
  Level& L = *h.lv[l];
  cudaStream_t st = c.stream;
  Exec<VT, CT> ex(h, st);
  LevelVecs<VT>& V = ex.V(l);
  const CT* coef = ex.coef(l);
  const VT* dinv = ex.dinv(l);
  const int n = L.B * L.n_r, eg = persistent_grid(c, (n + 255) / 256);
  Scalars* sc = h.sc.get();
  auto normalise = [&](VT* v) {
    dot_t<VT>(c, n, L.n_r, v, v, L.mult.get(), &sc->pw_norm, FIN_SQRT, st);
    k_scale_div<VT><<<eg, 256, 0, st>>>(n, v, &sc->pw_norm, v);
    RMG_LAUNCHED();
  };
  k_power_init<VT><<<eg, 256, 0, st>>>(L.n_r, L.B, L.gid.get(), L.mask.get(),
                                       (unsigned long long)(h.o.power_seed_base + l), V.u.get());
  RMG_LAUNCHED();
  normalise(V.u.get());
  VT* a = V.u.get();
  VT* b = V.r.get();
  for (int it = 0; it < h.o.power_iters; ++it) {
    launch_stencil(c, L, coef, a, V.y.get(), EpiScaled<VT>{dinv, b}, st, nullptr, nullptr,
                   nullptr, h.sweep(l), h.half(l), h.half_flag());
    std::swap(a, b);
    if (sizeof(VT) < 8 && (it + 1) % 8 == 0 && it + 1 < h.o.power_iters) normalise(a);
  }
  launch_stencil(c, L, coef, a, V.y.get(), EpiScaled<VT>{dinv, b}, st, nullptr, nullptr,
                 nullptr, h.sweep(l), h.half(l), h.half_flag());
  dot_t<VT>(c, n, L.n_r, a, b, L.mult.get(), &sc->pw_num, FIN_STORE, st);
  dot_t<VT>(c, n, L.n_r, a, a, L.mult.get(), &sc->pw_den, FIN_STORE, st);
  k_cheb_coeffs<<<1, 1, 0, st>>>(sc, l, h.o.eig_ratio, h.o.boost, h.o.cheb_degree);
  RMG_LAUNCHED();
}

static void power_method(Hier& h, int l) {
  switch (h.o.precision) {
    case RMG_PREC_FP64: power_method_t<double, double>(h, l); break;
    case RMG_PREC_FP32: power_method_t<float, float>(h, l); break;
    default: power_method_t<float, __nv_bfloat16>(h, l); break;
  }
}

static bool coarse_factor_mixed(Hier& h, int nd);
static void coarse_factor_fp64(Hier& h, int nc);

static void coarse_factor(Hier& h) {
  Ctx& c = *h.c;
  cudaStream_t st = c.stream;
  Level& L = *h.lv[h.levels() - 1];
  if (h.nc == 0 || !h.dense_ok) return;
  const int nc = h.nc * L.B;     // dense dimension: B dofs per free composite node
  RMG_CUDA(cudaMemsetAsync(h.Mfac.get(), 0, (size_t)nc * nc * sizeof(double), st));
  const dim3 gb(persistent_grid(c, (L.ncomp + 127) / 128), L.B);
#define RMG_ASM(K)                                                                              \
  k_coarse_assemble<K><<<gb, 128, 0, st>>>(L.ncomp, L.B, L.regions.get(), L.nreg, L.n_r,        \
                                           L.coef.get(), L.gid.get(), h.cidx.get(), L.c2r.get(), \
                                           L.cgrp.get(), L.gptr.get(), L.gslot.get(), nc,          \
                                           h.Mfac.get())
  switch (L.kind) {
    case 5: RMG_ASM(5); break;
    case 7: RMG_ASM(7); break;
    case 9: RMG_ASM(9); break;
    default: RMG_ASM(27); break;
  }
#undef RMG_ASM
  RMG_LAUNCHED();
  // keep the assembled matrix for introspection and for the refinement residuals in X
  RMG_CUDA(cudaMemcpyAsync(h.X.get(), h.Mfac.get(), (size_t)nc * nc * sizeof(double),
                           cudaMemcpyDeviceToDevice, st));
  if (!coarse_factor_mixed(h, nc)) coarse_factor_fp64(h, nc);
}

// Dense inverse in precision F of the nd x nd matrix in M (overwritten by its Cholesky factor):
// blocked Cholesky, L^-1 by recursive doubling, Ainv = L^-T L^-1.
template <typename F>
static void dense_inverse(Ctx& c, cudaStream_t st, int nd, F* M, F* Dblk, F* Linv, F* Tinv,
                          F* Ainv, int* err) {
  for (int k0 = 0; k0 < nd; k0 += kNB) {
    k_chol_diag<F><<<1, 32, 0, st>>>(M, nd, k0, Dblk, err);
    RMG_LAUNCHED();
    const int k1 = std::min(nd, k0 + kNB);
    if (k1 < nd) {
      const int rows = nd - k1;
      k_chol_panel<F><<<std::min(1024, (rows + 7) / 8), 256, 0, st>>>(M, nd, k0, Dblk);
      RMG_LAUNCHED();
      const int tiles = (rows + 15) / 16;
      k_chol_update<F><<<dim3(tiles, tiles), dim3(16, 16), 0, st>>>(M, nd, k0, k1);
      RMG_LAUNCHED();
    }
  }
  RMG_CUDA(cudaMemsetAsync(Linv, 0, (size_t)nd * nd * sizeof(F), st));
  const int nblk = (nd + kNB - 1) / kNB;
  k_inv_diag_blocks<F><<<nblk, 256, 0, st>>>(nd, Dblk, Linv);
  RMG_LAUNCHED();
  for (int s = kNB; s < nd; s *= 2) {
    const int tiles = (s + kNB - 1) / kNB, pairs = (nd + 2 * s - 1) / (2 * s);
    const dim3 grid(tiles, tiles, pairs);
    k_inv_merge<1, F><<<grid, 256, 0, st>>>(M, Linv, Tinv, nd, s);
    RMG_LAUNCHED();
    k_inv_merge<2, F><<<grid, 256, 0, st>>>(M, Linv, Tinv, nd, s);
    RMG_LAUNCHED();
  }
  const int t = (nd + 15) / 16;
  k_xtx<F><<<dim3(t, t), dim3(16, 16), 0, st>>>(Linv, nd, Ainv);
  RMG_LAUNCHED();
}

static void coarse_factor_fp64(Hier& h, int nc) {
  Ctx& c = *h.c;
  dense_inverse<double>(c, c.stream, nc, h.Mfac.get(), h.Dblk.get(), h.Linv.get(), h.Tinv.get(),
                        h.Ainv.get(), c.d_err.get());
  c.check_device_error("rmg_setup (coarse factorisation)");
  h.coarse_refine = 0;
}

// One mixed-precision coarse solve xc = Abar^-1 rc: x = S Ainv32 S rc, then `steps` FP64
// refinement steps x += S Ainv32 S (rc - Abar x). nrm (optional) receives ||rc - Abar x||^2
// before every refinement step.
static int mixed_coarse_solve(Hier& h, cudaStream_t st, int nd, int steps, double* nrm) {
  Ctx& c = *h.c;
  const int wg = std::max(1, std::min(c.nsm * 4, (nd * 32 + 255) / 256));
  int launches = 0;
  double* back = h.cnorm.get() + 4;
  k_scale_vec32<<<1, 1024, 0, st>>>(nd, h.cscale.get(), h.rc.get(), h.cw32.get(), back);
  RMG_LAUNCHED();
  k_gemv32<<<wg, 256, 0, st>>>(nd, h.Ainv32.get(), h.cw32.get(), h.cscale.get(), back,
                               h.xc.get(), 0);
  RMG_LAUNCHED();
  launches += 2;
  for (int k = 0; k < steps; ++k) {
    k_resid_dense<<<wg, 256, 0, st>>>(nd, h.X.get(), h.xc.get(), h.rc.get(), h.cres.get());
    RMG_LAUNCHED();
    if (nrm) {
      k_norm2_dense<<<1, 256, 0, st>>>(nd, h.cres.get(), nrm + k);
      RMG_LAUNCHED();
    }
    k_scale_vec32<<<1, 1024, 0, st>>>(nd, h.cscale.get(), h.cres.get(), h.cw32.get(), back);
    RMG_LAUNCHED();
    k_gemv32<<<wg, 256, 0, st>>>(nd, h.Ainv32.get(), h.cw32.get(), h.cscale.get(), back,
                                 h.xc.get(), 1);
    RMG_LAUNCHED();
    launches += 3;
  }
  return launches;
}

// FP32 factorisation of S Abar S (GB300's FP32 pipe is 64x its FP64 one) with FP64 iterative
// refinement in every coarse solve. The number of refinement steps comes from the contraction
// measured here on a test vector (it must bring the relative residual to 1e-15); a breakdown of
// the FP32 factorisation or a contraction above 0.1 leaves the FP64 inverse to the caller.
static bool coarse_factor_mixed(Hier& h, int nd) {
  Ctx& c = *h.c;
  cudaStream_t st = c.stream;
  const int eg = std::max(1, std::min(c.nsm * 4, (nd + 255) / 256));
  k_dense_scale<<<eg, 256, 0, st>>>(nd, h.X.get(), h.cscale.get());
  RMG_LAUNCHED();
  k_dense_scaled32<<<dim3((nd + 255) / 256, nd), 256, 0, st>>>(nd, h.X.get(), h.cscale.get(),
                                                               h.M32.get());
  RMG_LAUNCHED();
  RMG_CUDA(cudaMemsetAsync(h.cerr.get(), 0, sizeof(int), st));
  dense_inverse<float>(c, st, nd, h.M32.get(), h.Dblk32.get(), h.Linv32.get(), h.Tinv32.get(),
                       h.Ainv32.get(), h.cerr.get());
  // contraction of the refinement on a SplitMix64 test right-hand side
  k_dense_random<<<eg, 256, 0, st>>>(nd, 0x5eedull, h.rc.get());
  RMG_LAUNCHED();
  k_norm2_dense<<<1, 256, 0, st>>>(nd, h.rc.get(), h.cnorm.get());
  RMG_LAUNCHED();
  mixed_coarse_solve(h, st, nd, 3, h.cnorm.get() + 1);
  int err = 0;
  RMG_CUDA(cudaMemcpyAsync(h.pinned, h.cnorm.get(), 4 * sizeof(double), cudaMemcpyDeviceToHost,
                           st));
  RMG_CUDA(cudaMemcpyAsync(&err, h.cerr.get(), sizeof(int), cudaMemcpyDeviceToHost, st));
  RMG_CUDA(cudaStreamSynchronize(st));
  const double b2 = h.pinned[0], r0 = h.pinned[1], r1 = h.pinned[2], r2 = h.pinned[3];
  if (err || !(b2 > 0.0) || !std::isfinite(r0) || !std::isfinite(r2) || !(r0 > 0.0)) return false;
  // per-step contraction from the last two steps (the first one also removes the FP32
  // rounding of the right-hand side), in norms
  const double rho = std::sqrt(std::max(r2, 1e-300) / std::max(r1, 1e-300));
  const double rel0 = std::sqrt(r0 / b2);
  if (!(rho < 0.1)) return false;
  int steps = 1;
  double rel = rel0 * std::max(rho, 1e-16);
  while (rel > 1e-15 && steps < 8) {
    rel *= std::max(rho, 1e-16);
    ++steps;
  }
  if (rel > 1e-15) return false;
  h.coarse_rho = rho;
  h.coarse_refine = steps;
  return true;
}

// FP32 copy of the level-0 coefficients for the mixed hierarchy's FP32 Galerkin chain.
static void level0_to_fp32(Hier& h) {
  Ctx& c = *h.c;
  Level& L = *h.lv[0];
  if (!h.half_on) {
    const size_t nco = (size_t)L.B * L.B * L.kind * L.n_r;
    const int g = persistent_grid(c, (int)std::min<size_t>((nco + 255) / 256, 1 << 20));
    k_convert<double, float><<<g, 256, 0, c.stream>>>(nco, L.coef.get(), L.coef32.get());
    RMG_LAUNCHED();
    return;
  }
  // with the FP32 cycle's half planes and the flag that says whether they hold the operator,
  // in the same pass
  h.half32.ensure((size_t)(L.kind + 1) / 2 * L.n_r);
  int* flag = &h.sc.get()->half_asym;
  RMG_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c.stream));
  const Grid G = L.grid();
  const int gb = persistent_grid(c, G.ntiles);
#define RMG_L0(K)                                                                              \
  k_level0_fp32<K><<<gb, kTile, 0, c.stream>>>(G, L.coef.get(), L.coef32.get(), h.half32.get(), \
                                               flag)
  switch (L.kind) {
    case 5: RMG_L0(5); break;
    case 7: RMG_L0(7); break;
    case 9: RMG_L0(9); break;
    default: RMG_L0(27); break;
  }
#undef RMG_L0
  RMG_LAUNCHED();
}

// The mixed cycle's remaining copies: FP32 D~^-1 on every level and, for the BF16 variant, the
// BF16 coefficients (from the FP32 ones).
static void make_low_precision(Hier& h) {
  Ctx& c = *h.c;
  for (int l = 0; l < h.levels(); ++l) {
    Level& L = *h.lv[l];
    const size_t nco = (size_t)L.B * L.B * L.kind * L.n_r;
    const int g = persistent_grid(c, (int)std::min<size_t>((nco + 255) / 256, 1 << 20));
    if (h.o.precision == RMG_PREC_FP32_BF16COEF) {
      k_to_bf16<<<g, 256, 0, c.stream>>>(nco, L.coef32.get(), L.coef16.get());
      RMG_LAUNCHED();
    }
    k_convert<double, float><<<g, 256, 0, c.stream>>>((size_t)L.B * L.n_r, L.dinv.get(),
                                                      L.dinv32.get());
    RMG_LAUNCHED();
  }
}

// ---------------------------------------------------------------------- tile-shape autotuner
// Candidate tile shapes of the stencil sweeps: index 0 = runs of kTile consecutive nodes,
// 1..8 = boxes tx x ty x tz (tx * ty * tz = kTile, given as log2 tx, log2 ty), 9 = 32 x 8
// columns staged through shared memory (27-point FP32 half planes). Boxes hand every thread
// its (i, j, l) without a decode and keep stencil neighbours inside the block, at the price of
// idle threads where a box overhangs the region; which wins depends on the region sizes, the
// stencil and the precision, so each hierarchy times them.

static bool shape_fits(const Hier& h, int l, int k) {
  const Level& L = *h.lv[l];
  const TileShape t = kTileShapes[k];
  if (k == kStagedShape) {     // FP32 half-plane sweeps of a 3D 27-point scalar stencil only
    if (!(h.half(l) != nullptr && L.B == 1 && L.dim == 3 && L.kind == 27 &&
          h.o.smoother != RMG_SMOOTHER_GS))
      return false;
    for (int d : L.hdims)
      if (d >= 32768) return false;                       // tile corners are 16-bit
    return true;
  }
  if (t.lx < 0) return true;
  if (L.dim == 2 && t.lx + t.ly != 8) return false;      // 2D levels need tz = 1
  for (int d : L.hdims)
    if (d >= 32768) return false;                         // box corners are 16-bit
  return true;
}

static void set_shape(Hier& h, int l, int k) {
  Level& L = *h.lv[l];
  h.shape[l] = k;
  const TileShape t = kTileShapes[k];
  if (t.lx == -1) {
    h.sgrid[l] = L.grid();
    return;
  }
  std::vector<Tile> tl;
  if (t.lx == -3) {
    // staged columns: one 32 x 8 tile of the x-y planes per block, through all z-planes
    for (int r = 0; r < L.nreg; ++r) {
      const int nx = L.hdims[3 * r], ny = L.hdims[3 * r + 1];
      for (int y = 0; y < ny; y += kStY)
        for (int x = 0; x < nx; x += kStX) tl.push_back(Tile{r, 0, (short)x, (short)y, 0, 0});
    }
  }
  const int tx = t.lx < 0 ? 1 : 1 << t.lx, ty = t.lx < 0 ? 1 : 1 << t.ly;
  const int tz = t.lx < 0 ? 1 : kTile >> (t.lx + t.ly);
  for (int r = 0; r < L.nreg && t.lx >= 0; ++r) {
    const int nx = L.hdims[3 * r], ny = L.hdims[3 * r + 1], nz = L.hdims[3 * r + 2];
    for (int z = 0; z < nz; z += tz)
      for (int y = 0; y < ny; y += ty)
        for (int x = 0; x < nx; x += tx)
          tl.push_back(Tile{r, 0, (short)x, (short)y, (short)z, 0});
  }
  h.stiles[l].alloc(tl.size());
  RMG_CUDA(cudaMemcpy(h.stiles[l].get(), tl.data(), tl.size() * sizeof(Tile),
                      cudaMemcpyHostToDevice));
  Grid G = L.grid();
  G.tiles = h.stiles[l].get();
  G.ntiles = (int)tl.size();
  G.lx = t.lx;
  G.ly = t.ly;
  h.sgrid[l] = G;
}

// Time the candidate shapes on every smoothed level with the residual sweep in the cycle's
// precision (3 launches after a warm-up, CUDA events on the library stream) and keep the
// fastest; tile_shape >= 0 in the options forces one shape where it fits.
template <typename VT, typename CT>
static void autotune_t(Hier& h) {
  Ctx& c = *h.c;
  cudaStream_t st = c.stream;
  Exec<VT, CT> ex(h, st);
  cudaEvent_t e0, e1;
  RMG_CUDA(cudaEventCreate(&e0));
  RMG_CUDA(cudaEventCreate(&e1));
  for (int l = 0; l + 1 < h.levels(); ++l) {
    const Level& L = *h.lv[l];
    LevelVecs<VT>& V = ex.V(l);
    const size_t nv = (size_t)L.B * L.n_r;
    RMG_CUDA(cudaMemsetAsync(V.u.get(), 0, nv * sizeof(VT), st));
    RMG_CUDA(cudaMemsetAsync(V.b.get(), 0, nv * sizeof(VT), st));
    if (h.o.tile_shape >= 0) {
      set_shape(h, l, shape_fits(h, l, h.o.tile_shape) ? h.o.tile_shape : 0);
      continue;
    }
    int best = 0;
    float best_ms = 0.f;
    for (int k = 0; k < kNumTileShapes; ++k) {
      if (!shape_fits(h, l, k)) continue;
      set_shape(h, l, k);
      auto run = [&]() {
        launch_stencil(c, L, ex.coef(l), (const VT*)V.u.get(), V.y.get(),
                       EpiResid<VT>{V.b.get(), V.r.get()}, st, nullptr, nullptr, nullptr,
                       &h.sgrid[l], h.half(l), h.half_flag());
      };
      run();
      RMG_CUDA(cudaEventRecord(e0, st));
      for (int rep = 0; rep < 3; ++rep) run();
      RMG_CUDA(cudaEventRecord(e1, st));
      RMG_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      RMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (k == 0 || ms < best_ms) { best = k; best_ms = ms; }
    }
    set_shape(h, l, best);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

static void autotune(Hier& h) {
  switch (h.o.precision) {
    case RMG_PREC_FP64: autotune_t<double, double>(h); break;
    case RMG_PREC_FP32: autotune_t<float, float>(h); break;
    default: autotune_t<float, __nv_bfloat16>(h); break;
  }
  h.tuned = true;
}

void tile_shape(const Hier& h, int l, int* tx, int* ty, int* tz) {
  if (h.shape[l] == kStagedShape) {
    *tx = kStX; *ty = kStY; *tz = 0;
    return;
  }
  const TileShape t = kTileShapes[h.shape[l]];
  *tx = t.lx < 0 ? 0 : 1 << t.lx;
  *ty = t.lx < 0 ? 0 : 1 << t.ly;
  *tz = t.lx < 0 ? 0 : kTile >> (t.lx + t.ly);
}

void hier_numeric(Hier& h) {
  Ctx& c = *h.c;
  const int Lv = h.levels();
  Level& L0 = *h.lv[0];
  if (h.gexec) {
    RMG_REQUIRE(L0.kind == h.kind0 && L0.coef.get() == h.coef0, RMG_ERR_STATE,
                "the layout's operator changed its stencil since rmg_setup; create a new "
                "hierarchy");
  }
  h.kind0 = L0.kind;
  h.coef0 = L0.coef.get();
  compute_dinv(h, *h.lv[0]);
  if (h.mixed()) level0_to_fp32(h);
  for (int l = 0; l + 1 < Lv; ++l) {
    galerkin(h, l, *h.lv[l], *h.lv[l + 1]);
    compute_dinv(h, *h.lv[l + 1]);
  }
  // the mixed cycle's coefficient copies first: its power method runs on them
  if (h.mixed()) make_low_precision(h);
  if (!h.tuned) autotune(h);
  if (h.o.smoother == RMG_SMOOTHER_CHEBYSHEV)
    for (int l = 0; l + 1 < Lv; ++l) power_method(h, l);
  coarse_factor(h);
  RMG_CUDA(cudaMemcpyAsync(&h.hsc, h.sc.get(), sizeof(Scalars), cudaMemcpyDeviceToHost, c.stream));
  RMG_CUDA(cudaStreamSynchronize(c.stream));
  const std::vector<char>& stored = h.stored;
  if (h.gexec && (stored != h.graph_stored || h.coarse_refine != h.graph_refine)) {
    cudaGraphExecDestroy(h.gexec);
    cudaGraphDestroy(h.graph);
    h.gexec = nullptr;
    h.graph = nullptr;
  }
  h.graph_stored = stored;
  h.graph_refine = h.coarse_refine;
  if (h.o.use_graph && !h.gexec && h.dense_ok) {
    if (!h.graph_stream) RMG_CUDA(cudaStreamCreateWithFlags(&h.graph_stream, cudaStreamNonBlocking));
    RMG_CUDA(cudaStreamBeginCapture(h.graph_stream, cudaStreamCaptureModeThreadLocal));
    int launches = 0;
    g_capturing = true;
    try {
      launches = run_cycle(h, h.graph_stream);
      g_capturing = false;
    } catch (...) {
      g_capturing = false;
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(h.graph_stream, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    RMG_CUDA(cudaStreamEndCapture(h.graph_stream, &h.graph));
    RMG_CUDA(cudaGraphInstantiate(&h.gexec, h.graph, 0));
    h.launches = launches;
  }
}

void require_dense(const Hier& h) {
  RMG_REQUIRE(h.dense_ok, RMG_ERR_STATE,
              "the coarsest level has more unknowns than the dense coarse solver takes (" +
                  std::to_string(kMaxDense) + "); use more levels");
}

void vcycle(Hier& h) {
  require_dense(h);
  h.probe_pending = h.levels() > 1 && (h.o.nu2 > 0);
  if (h.gexec) {
    RMG_CUDA(cudaGraphLaunch(h.gexec, h.c->stream));
    g_launches += (unsigned long long)h.launches;
  } else {
    h.launches = run_cycle(h, h.c->stream);
  }
}

// r, z: FP64 regional or composite device vectors.
void vcycle_apply(Hier& h, const double* r, double* z, int regional) {
  Ctx& c = *h.c;
  const Level& L0 = *h.lv[0];
  const int n = L0.B * L0.n_r, g = persistent_grid(c, (n + 255) / 256);
  double* b64 = h.v64[0].b.get();
  if (regional) k_copy<double><<<g, 256, 0, c.stream>>>(n, r, b64);
  else comp_to_reg(c, L0, r, b64, true);
  RMG_LAUNCHED();
  if (h.mixed()) {
    k_convert<double, float><<<g, 256, 0, c.stream>>>((size_t)n, b64, h.v32[0].b.get());
    RMG_LAUNCHED();
  }
  vcycle(h);
  double* u64 = h.v64[0].u.get();
  if (h.mixed()) {
    k_convert<float, double><<<g, 256, 0, c.stream>>>((size_t)n, h.v32[0].u.get(), u64);
    RMG_LAUNCHED();
  }
  if (regional) k_copy<double><<<g, 256, 0, c.stream>>>(n, u64, z);
  else reg_to_comp(c, L0, u64, z, 1);
  RMG_LAUNCHED();
}

// Accumulate the timed level-0 smoother launch of the last V-cycle (stream must be idle).
void probe_collect(Hier& h) {
  if (!h.probe_pending || !h.probe_ev[0]) return;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, h.probe_ev[0], h.probe_ev[1]) == cudaSuccess) {
    h.probe_ms += ms;
    h.probe_count += 1;
  } else {
    cudaGetLastError();
  }
  h.probe_pending = false;
}

// V-cycle as a stationary solver on A e = 0 from a SplitMix64 random error:
// e <- e - M^-1 A e. Returns (||e_K||_A / ||e_0||_A)^(1/K), the mean A-norm error reduction
// per cycle (FP64 A-norm; the cycle in the hierarchy's own precision).
double convergence_factor(Hier& h, int iters, unsigned long long seed) {
  require_dense(h);
  Ctx& c = *h.c;
  cudaStream_t st = c.stream;
  const Level& L0 = *h.lv[0];
  const int n = L0.B * L0.n_r, eg = persistent_grid(c, (n + 255) / 256);
  Scalars* sc = h.sc.get();
  double* e = h.x.get();
  double* Ae = h.v64[0].b.get();      // the cycle's right-hand side buffer
  double* z = h.v64[0].u.get();
  k_power_init<<<eg, 256, 0, st>>>(L0.n_r, L0.B, L0.gid.get(), L0.mask.get(), seed, e);
  RMG_LAUNCHED();
  auto anorm2 = [&]() {
    launch_stencil(c, L0, L0.coef.get(), e, h.v64[0].y.get(), EpiStore<double>{Ae}, st, nullptr);
    dot(c, n, L0.n_r, e, Ae, L0.mult.get(), &sc->pq, FIN_STORE, st);
    RMG_CUDA(cudaMemcpyAsync(h.pinned, &sc->pq, sizeof(double), cudaMemcpyDeviceToHost, st));
    RMG_CUDA(cudaStreamSynchronize(st));
    return h.pinned[0];
  };
  const double e0 = anorm2();
  double ek = e0;
  for (int k = 0; k < iters; ++k) {
    if (h.mixed()) {
      k_convert<double, float><<<eg, 256, 0, st>>>((size_t)n, Ae, h.v32[0].b.get());
      RMG_LAUNCHED();
      vcycle(h);
      k_convert<float, double><<<eg, 256, 0, st>>>((size_t)n, h.v32[0].u.get(), z);
      RMG_LAUNCHED();
    } else {
      vcycle(h);
    }
    k_axpy_neg<<<eg, 256, 0, st>>>(n, z, e);
    RMG_LAUNCHED();
    ek = anorm2();
  }
  if (!(e0 > 0.0) || iters <= 0) return 0.0;
  return std::pow(std::max(ek, 0.0) / e0, 0.5 / iters);
}

// ---------------------------------------------------------------------- per-region energies
// E_k(e) = e_k^T A^(k) e_k for every region k: the region's own (split) matrix applied to the
// region's copy of e, without the interface sum. By Lemma 1 the E_k add up to e^T A e; for the
// M-matrix operators here every A^(k) is positive semi-definite (row sums zero or positive,
// non-positive couplings), so E_k is a local energy of the error. One partial sum per run tile,
// then the tiles of each region (contiguous in the tile list) in order.
template <int KIND>
__global__ void __launch_bounds__(kTile)
k_region_energy(Grid G, const double* __restrict__ coef, const double* __restrict__ e,
                double* __restrict__ part) {
  for (int t = blockIdx.x; t < G.ntiles; t += gridDim.x) {
    const Tile tile = G.tiles[t];
    const RegionDev R = G.regions[tile.region];
    const int li = tile.start + (int)threadIdx.x;
    double v = 0.0;
    if (li < R.nx * R.ny * R.nz) {
      int i, j, l;
      decode(li, R, i, j, l);
      const int n = R.off + li;
      v = e[n] * stencil_row<KIND, double, double, double>(coef, e, n, G.n_r, i, j, l, R);
    }
    v = block_sum<kTile>(v);
    if (threadIdx.x == 0) part[t] = v;
  }
}

__global__ void k_region_sum(int nreg, const int* __restrict__ tstart,
                             const double* __restrict__ part, double* __restrict__ out) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreg; r += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int t = tstart[r]; t < tstart[r + 1]; ++t) s += part[t];
    out[r] = s;
  }
}

static void region_energy(Hier& h, const double* e, double* host_out) {
  Ctx& c = *h.c;
  const Level& L = *h.lv[0];
  const Grid G = L.grid();
  if (h.energy_tiles.n != (size_t)L.nreg + 1) {
    std::vector<int> ts(L.nreg + 1, 0);
    for (size_t t = 0; t < L.htiles.size(); ++t) ts[L.htiles[t].region + 1] = (int)t + 1;
    for (int r = 0; r < L.nreg; ++r) ts[r + 1] = std::max(ts[r + 1], ts[r]);
    h.energy_tiles.alloc(L.nreg + 1);
    RMG_CUDA(cudaMemcpy(h.energy_tiles.get(), ts.data(), ts.size() * sizeof(int),
                        cudaMemcpyHostToDevice));
    h.energy_part.alloc(std::max<size_t>(1, L.htiles.size()));
    h.energy_out.alloc(L.nreg);
  }
  const int gb = persistent_grid(c, G.ntiles);
  switch (L.kind) {
    case 5: k_region_energy<5><<<gb, kTile, 0, c.stream>>>(G, L.coef.get(), e, h.energy_part.get()); break;
    case 7: k_region_energy<7><<<gb, kTile, 0, c.stream>>>(G, L.coef.get(), e, h.energy_part.get()); break;
    case 9: k_region_energy<9><<<gb, kTile, 0, c.stream>>>(G, L.coef.get(), e, h.energy_part.get()); break;
    default: k_region_energy<27><<<gb, kTile, 0, c.stream>>>(G, L.coef.get(), e, h.energy_part.get()); break;
  }
  RMG_LAUNCHED();
  k_region_sum<<<persistent_grid(c, (L.nreg + 255) / 256), 256, 0, c.stream>>>(
      L.nreg, h.energy_tiles.get(), h.energy_part.get(), h.energy_out.get());
  RMG_LAUNCHED();
  RMG_CUDA(cudaMemcpyAsync(host_out, h.energy_out.get(), (size_t)L.nreg * sizeof(double),
                           cudaMemcpyDeviceToHost, c.stream));
  RMG_CUDA(cudaStreamSynchronize(c.stream));
}

// The V-cycle as a stationary solver (as convergence_factor) with the region energies of the
// error before and after `iters` cycles.
void region_energies(Hier& h, int iters, unsigned long long seed, double* e0, double* eK) {
  require_dense(h);
  Ctx& c = *h.c;
  cudaStream_t st = c.stream;
  const Level& L0 = *h.lv[0];
  RMG_REQUIRE(L0.B == 1, RMG_ERR_ARG, "region energies are for scalar operators");
  const int n = L0.n_r, eg = persistent_grid(c, (n + 255) / 256);
  double* e = h.x.get();
  double* Ae = h.v64[0].b.get();
  double* z = h.v64[0].u.get();
  k_power_init<<<eg, 256, 0, st>>>(L0.n_r, L0.B, L0.gid.get(), L0.mask.get(), seed, e);
  RMG_LAUNCHED();
  region_energy(h, e, e0);
  for (int k = 0; k < iters; ++k) {
    launch_stencil(c, L0, L0.coef.get(), e, h.v64[0].y.get(), EpiStore<double>{Ae}, st, nullptr);
    if (h.mixed()) {
      k_convert<double, float><<<eg, 256, 0, st>>>((size_t)n, Ae, h.v32[0].b.get());
      RMG_LAUNCHED();
      vcycle(h);
      k_convert<float, double><<<eg, 256, 0, st>>>((size_t)n, h.v32[0].u.get(), z);
      RMG_LAUNCHED();
    } else {
      vcycle(h);
    }
    k_axpy_neg<<<eg, 256, 0, st>>>(n, z, e);
    RMG_LAUNCHED();
  }
  region_energy(h, e, eK);
}

// Transfer weights of a level from `learned` where every region containing the node accepts,
// linear interpolation (rem / 3) elsewhere; zero along axes where the node sits on a coarse
// index. Copies of an interface node see the same regions, so they get the same weights.
__global__ void __launch_bounds__(kTile)
k_blend_weights(Grid G, int dim, const uint8_t* __restrict__ accept,
                const uint8_t* __restrict__ mult, const int* __restrict__ gid,
                const int* __restrict__ cgrp, const int* __restrict__ gptr,
                const int* __restrict__ gslot, const float* __restrict__ learned,
                float* __restrict__ out) {
  RMG_FOR_NODES(G)
    int x[3];
    decode(li, R, x[0], x[1], x[2]);
    bool ok = accept[tile_.region] != 0;
    if (ok && mult[n] > 1) {
      const int grp = cgrp[gid[n]];
      for (int q = gptr[grp]; q < gptr[grp + 1]; ++q)
        ok = ok && accept[region_of(G.regions, G.nreg, gslot[q])] != 0;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int rem = a < dim ? x[a] % 3 : 0;
      const size_t k = (size_t)a * G.n_r + n;
      out[k] = rem == 0 ? 0.f : (ok ? learned[k] : (rem == 1 ? (float)(1.0 / 3.0)
                                                             : (float)(2.0 / 3.0)));
    }
  RMG_END_FOR_NODES
}

void blend_weights(Hier& h, int level, const uint8_t* accept_host, const float* learned,
                   float* out) {
  RMG_REQUIRE(level >= 0 && level + 1 < h.levels(), RMG_ERR_ARG,
              "transfer weights exist for levels 0 .. levels-2");
  Level& L = *h.lv[level];
  RMG_REQUIRE(L.B == 1, RMG_ERR_ARG, "stored transfer weights are for scalar operators");
  Ctx& c = *h.c;
  h.accept.ensure(L.nreg);
  RMG_CUDA(cudaMemcpyAsync(h.accept.get(), accept_host, (size_t)L.nreg, cudaMemcpyHostToDevice,
                           c.stream));
  const Grid G = L.grid();
  k_blend_weights<<<persistent_grid(c, G.ntiles), kTile, 0, c.stream>>>(
      G, L.dim, h.accept.get(), L.mult.get(), L.gid.get(), L.cgrp.get(), L.gptr.get(),
      L.gslot.get(), learned, out);
  RMG_LAUNCHED();
  RMG_CUDA(cudaStreamSynchronize(c.stream));      // the host accept array may be reused
}

// Greedy colouring of the region graph of level 0: two regions are adjacent when they share a
// composite node (an interface group holds copies in both). Regions of one colour never touch,
// so a transfer changed in the regions of one colour alone leaves every interface node with
// linear weights (rmg_hier_blend_weights) and the other regions' own rows unchanged.
int region_colours(Hier& h, int* colours) {
  const Level& L = *h.lv[0];
  std::vector<int> gptr(L.ngroups + 1), gslot(L.nslots);
  if (L.ngroups) {
    RMG_CUDA(cudaMemcpy(gptr.data(), L.gptr.get(), gptr.size() * sizeof(int),
                        cudaMemcpyDeviceToHost));
    RMG_CUDA(cudaMemcpy(gslot.data(), L.gslot.get(), gslot.size() * sizeof(int),
                        cudaMemcpyDeviceToHost));
  }
  auto region = [&](int slot) {
    return (int)(std::upper_bound(L.hoff.begin(), L.hoff.begin() + L.nreg, slot) -
                 L.hoff.begin()) - 1;
  };
  std::vector<std::vector<int>> adj(L.nreg);
  for (int g = 0; g < L.ngroups; ++g)
    for (int a = gptr[g]; a < gptr[g + 1]; ++a)
      for (int b = a + 1; b < gptr[g + 1]; ++b) {
        const int ra = region(gslot[a]), rb = region(gslot[b]);
        if (ra != rb) { adj[ra].push_back(rb); adj[rb].push_back(ra); }
      }
  int ncol = 0;
  std::vector<int> col(L.nreg, -1);
  for (int r = 0; r < L.nreg; ++r) {
    std::vector<char> used(ncol + 1, 0);
    for (int q : adj[r])
      if (col[q] >= 0) used[col[q]] = 1;
    int c = 0;
    while (used[c]) ++c;
    col[r] = c;
    ncol = std::max(ncol, c + 1);
  }
  std::copy(col.begin(), col.end(), colours);
  return ncol;
}

// ---------------------------------------------------------------------- PCG
// Textbook PCG for the plain FP64 cycle, flexible CG (Polak-Ribiere beta) for the FP32/BF16
// cycles and for the region Gauss-Seidel cycle; every inner product and update in FP64. When
// the recurrence residual passes the tolerance the true residual b - A x is recomputed; the
// solve ends only if it passes too, otherwise the iteration restarts from the true residual.
void pcg_solve(Hier& h, const double* b, double* xout, double rtol, int maxit, double* history,
               rmg_solve_info* info) {
  require_dense(h);
  Ctx& c = *h.c;
  cudaStream_t st = c.stream;
  const Level& L0 = *h.lv[0];
  const int n = L0.B * L0.n_r, eg = persistent_grid(c, (n + 255) / 256);
  const int dg = std::min(c.max_partials, persistent_grid(c, (n + 255) / 256));
  Scalars* sc = h.sc.get();
  const bool mixed = h.mixed();
  // the Gauss-Seidel cycle is not exactly symmetric (interface copies drift apart within a
  // sweep): flexible CG for it in FP64 too
  const bool flex64 = !mixed && h.o.smoother == RMG_SMOOTHER_GS;
  double* rvec = h.v64[0].b.get();     // the V-cycle reads its right-hand side here
  double* zvec = h.v64[0].u.get();     // and leaves its result here (FP64 cycle)
  double* breg = h.tmp.get();
  const auto t0 = std::chrono::steady_clock::now();
  comp_to_reg(c, L0, b, breg, true);
  comp_to_reg(c, L0, xout, h.x.get(), true);
  auto read2 = [&](double* a, double* bb) {
    RMG_CUDA(cudaMemcpyAsync(h.pinned, &sc->rr, sizeof(double), cudaMemcpyDeviceToHost, st));
    RMG_CUDA(cudaMemcpyAsync(h.pinned + 1, &sc->bb, sizeof(double), cudaMemcpyDeviceToHost, st));
    RMG_CUDA(cudaStreamSynchronize(st));
    probe_collect(h);
    *a = h.pinned[0];
    *bb = h.pinned[1];
  };
  // out = b - A x and its squared composite norm into sc->rr
  auto true_residual = [&](double* out) {
    launch_stencil(c, L0, L0.coef.get(), h.x.get(), h.v64[0].y.get(),
                   EpiResid<double>{breg, out}, st, nullptr);
    dot(c, n, L0.n_r, out, out, L0.mult.get(), &sc->rr, FIN_STORE, st);
  };
  true_residual(rvec);
  dot(c, n, L0.n_r, breg, breg, L0.mult.get(), &sc->bb, FIN_STORE, st);
  double rr = 0, bb = 0;
  read2(&rr, &bb);
  const double bnorm = std::sqrt(bb);
  double relres = bnorm > 0 ? std::sqrt(rr) / bnorm : 0.0;
  double rtrue = relres;
  if (history) history[0] = relres;
  // the FP32 cycle's input scaling: a power of two near 1 / ||b|| (exact both ways)
  const int eb = (bnorm > 0 && std::isfinite(bnorm)) ? std::ilogb(bnorm) : 0;
  const double rscale = std::ldexp(1.0, -eb), zscale = std::ldexp(1.0, eb);
  int it = 0, ncyc = 0;
  // The FP32 cycle reads its right-hand side from r32 and leaves z32; in the loop, r32 is
  // written by the CG update and z32 is read directly by the dots and the direction update
  // (the cycle does not modify its level-0 right-hand side).
  float* r32 = mixed ? h.v32[0].b.get() : nullptr;
  const float* z32 = mixed ? h.v32[0].u.get() : nullptr;
  bool converged = !(relres > rtol) || !(bnorm > 0);
  while (!converged && it < maxit) {
    // (re)start: z = M^-1 r, p = z
    if (mixed) {
      k_to_f32_scaled<<<eg, 256, 0, st>>>(n, rvec, rscale, r32);
      RMG_LAUNCHED();
    }
    vcycle(h);
    ++ncyc;
    if (mixed) {
      k_start_dir<<<dg, 256, 0, st>>>(n, L0.n_r, rvec, z32, L0.mult.get(), zscale, h.p.get(),
                                      h.zold32.get(), c.partials.get());
      RMG_LAUNCHED();
      k_finalize<<<1, 256, 0, st>>>(c.partials.get(), dg, &sc->rz, FIN_STORE);
      RMG_LAUNCHED();
    } else {
      dot(c, n, L0.n_r, rvec, zvec, L0.mult.get(), &sc->rz, FIN_STORE, st);
      k_copy<double><<<eg, 256, 0, st>>>(n, zvec, h.p.get());
      RMG_LAUNCHED();
      if (flex64) {
        k_copy<double><<<eg, 256, 0, st>>>(n, zvec, h.zold.get());
        RMG_LAUNCHED();
      }
    }
    while (it < maxit) {
      ++it;
      launch_stencil(c, L0, L0.coef.get(), h.p.get(), h.v64[0].y.get(),
                     EpiStore<double>{h.q.get()}, st, nullptr);
      dot(c, n, L0.n_r, h.p.get(), h.q.get(), L0.mult.get(), &sc->pq, FIN_STORE, st);
      k_alpha<<<1, 1, 0, st>>>(sc);
      RMG_LAUNCHED();
      if (mixed)
        k_cg_update_mixed<<<dg, 256, 0, st>>>(n, L0.n_r, h.p.get(), h.q.get(), L0.mult.get(), sc,
                                              rscale, h.x.get(), rvec, r32, c.partials.get());
      else
        k_cg_update<<<dg, 256, 0, st>>>(n, L0.n_r, h.p.get(), h.q.get(), L0.mult.get(), sc,
                                        h.x.get(), rvec, c.partials.get());
      RMG_LAUNCHED();
      k_finalize<<<1, 256, 0, st>>>(c.partials.get(), dg, &sc->rr, FIN_STORE);
      RMG_LAUNCHED();
      read2(&rr, &bb);
      relres = std::sqrt(rr) / bnorm;
      if (history) history[it] = relres;
      if (relres <= rtol) {
        // confirm on the true residual; q is free until the next product
        true_residual(h.q.get());
        double rt = 0;
        read2(&rt, &bb);
        rtrue = std::sqrt(rt) / bnorm;
        if (rtrue <= rtol) {
          converged = true;
        } else {
          // the recurrence drifted from b - A x: restart from the true residual
          RMG_CUDA(cudaMemcpyAsync(rvec, h.q.get(), (size_t)n * sizeof(double),
                                   cudaMemcpyDeviceToDevice, st));
          relres = rtrue;
        }
        break;
      }
      vcycle(h);
      ++ncyc;
      if (mixed) {
        k_flex_dots<<<dg, 256, 0, st>>>(n, L0.n_r, rvec, z32, h.zold32.get(), L0.mult.get(),
                                        zscale, c.partials.get());
        RMG_LAUNCHED();
        k_finalize<<<1, 256, 0, st>>>(c.partials.get(), dg, &sc->rz_new, FIN_STORE);
        RMG_LAUNCHED();
        k_finalize<<<1, 256, 0, st>>>(c.partials.get() + dg, dg, &sc->beta, FIN_STORE);
        RMG_LAUNCHED();
        k_beta<<<1, 1, 0, st>>>(sc, 1);
        RMG_LAUNCHED();
        k_p_update<float><<<eg, 256, 0, st>>>(n, z32, zscale, sc, h.p.get());
        RMG_LAUNCHED();
      } else {
        dot(c, n, L0.n_r, rvec, zvec, L0.mult.get(), &sc->rz_new, FIN_STORE, st);
        if (flex64) {
          dot(c, n, L0.n_r, rvec, h.zold.get(), L0.mult.get(), &sc->beta, FIN_STORE, st);
          k_copy<double><<<eg, 256, 0, st>>>(n, zvec, h.zold.get());
          RMG_LAUNCHED();
        }
        k_beta<<<1, 1, 0, st>>>(sc, flex64 ? 1 : 0);
        RMG_LAUNCHED();
        k_p_update<double><<<eg, 256, 0, st>>>(n, zvec, 1.0, sc, h.p.get());
        RMG_LAUNCHED();
      }
    }
  }
  reg_to_comp(c, L0, h.x.get(), xout, 1);
  if (!converged || it == 0) {
    // true residual of the returned iterate (already known after a confirmed convergence)
    true_residual(h.q.get());
    double rt = 0;
    read2(&rt, &bb);
    rtrue = bnorm > 0 ? std::sqrt(rt) / bnorm : 0.0;
  } else {
    RMG_CUDA(cudaStreamSynchronize(st));
  }
  const auto t1 = std::chrono::steady_clock::now();
  if (info) {
    info->iterations = it;
    info->relres = relres;
    info->true_relres = rtrue;
    info->seconds = std::chrono::duration<double>(t1 - t0).count();
    info->vcycles = ncyc;
  }
  if (!converged)
    throw Error(RMG_ERR_NOT_CONVERGED, "PCG reached maxit with relres " + std::to_string(relres));
}

}  // namespace rmg
