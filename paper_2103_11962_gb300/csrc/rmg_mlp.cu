// Learned prolongator: a small MLP that maps a fine node's local operator to its interpolation
// weights, with hand-written training and inference kernels.
//
// Network: 27 features (padded to 32) -> 64 -> 64 -> 3, ReLU, ReLU, sigmoid. The three outputs
// are the weights a fine node takes from its right coarse neighbour along x, y and z (the left
// one gets 1 - w), so every predicted row of P sums to one and constants are preserved.
//
// Forward pass: BF16 tensor-core MMA (mma.sync m16n8k16, FP32 accumulate); a CTA of 8 warps
// takes 128 samples, each warp 16 rows. Backward pass: FP32 CUDA cores on the same tile, one
// atomic add per parameter per CTA. Adam updates FP32 master weights.
//
// Features of fine node n (9 per axis, zero along axes where n sits on a coarse index): for
// the line of three edges between its two coarse neighbours along the axis, log10 of the three
// composite conductances -A(p_e, p_e+1) and of the four composite diagonals, each divided by
// the node's own diagonal, then rem/3 and an active flag. Composite values are sums over the
// copies of a node, so co-located copies see the same features and get identical weights.
#include <cuda_bf16.h>

#include <algorithm>

#include "rmg_hier.cuh"
#include "rmg_kernels.cuh"

namespace rmg {
namespace {

constexpr int NF = 32, NH = 64, NOUT = 3;
constexpr int NPARAMS = NH * NF + NH + NH * NH + NH + NOUT * NH + NOUT;
constexpr int O_W1 = 0, O_B1 = O_W1 + NH * NF, O_W2 = O_B1 + NH, O_B2 = O_W2 + NH * NH,
              O_W3 = O_B2 + NH, O_B3 = O_W3 + NOUT * NH;
constexpr int kRows = 128, kThreads = 256;
// padded shared-memory strides (elements)
constexpr int SX = NF + 8, SH = NH + 8, SD = NH + 1;

struct MlpSmem {
  __nv_bfloat16 Xb[kRows * SX];
  __nv_bfloat16 W1b[NH * SX];
  __nv_bfloat16 H1b[kRows * SH];
  __nv_bfloat16 W2b[NH * SH];
  __nv_bfloat16 H2b[kRows * SH];
  __nv_bfloat16 W3b[8 * SH];
  float O[kRows * 4];
  float Y[kRows * 4];
  float M[kRows * 4];
  float W2f[NH * NH];
  float W3f[NOUT * NH];
  float dZ3[kRows * 4];
  float dZ2[kRows * SD];
  float dZ1[kRows * SD];
  float red[kThreads / 32];
};

__device__ __forceinline__ uint32_t pack2(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);    // two consecutive bf16 (4-byte aligned)
}

// acc[nt][4] += A[16 x K] * B[K x 8*NT] for one warp. A rows come from row-major bf16 smem
// (row stride lda, first row r0); B is given transposed: Bt[n][k] (row-major, stride ldb),
// which is how the layer weights are stored ([out][in]).
template <int NT, int K>
__device__ __forceinline__ void warp_mma(const __nv_bfloat16* A, int lda, int r0,
                                         const __nv_bfloat16* Bt, int ldb, float (&acc)[NT][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int k0 = 0; k0 < K; k0 += 16) {
    const uint32_t a0 = pack2(A + (r0 + g) * lda + k0 + 2 * t);
    const uint32_t a1 = pack2(A + (r0 + g + 8) * lda + k0 + 2 * t);
    const uint32_t a2 = pack2(A + (r0 + g) * lda + k0 + 2 * t + 8);
    const uint32_t a3 = pack2(A + (r0 + g + 8) * lda + k0 + 2 * t + 8);
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const uint32_t b0 = pack2(Bt + (nt * 8 + g) * ldb + k0 + 2 * t);
      const uint32_t b1 = pack2(Bt + (nt * 8 + g) * ldb + k0 + 2 * t + 8);
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
          "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
          : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
  }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// mode 0: inference (rows = samples base..base+127, outputs written to out[n][3]).
// mode 1: gradient (rows sampled or taken in order; gradients and loss accumulated).
__global__ void __launch_bounds__(kThreads)
k_mlp(const float* __restrict__ params, int n, long long ntiles, const float* __restrict__ feats,
      const float* __restrict__ labels, const float* __restrict__ mask, int mode, int sample,
      unsigned long long seed, float inv_norm, float* __restrict__ out, float* __restrict__ grads,
      float* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;

  // ---- stage weights (bf16 copies for the MMA, fp32 copies for the backward pass)
  for (int e = tid; e < NH * NF; e += kThreads)
    S.W1b[(e / NF) * SX + e % NF] = __float2bfloat16_rn(params[O_W1 + e]);
  for (int e = tid; e < NH * NH; e += kThreads) {
    const float w = params[O_W2 + e];
    S.W2b[(e / NH) * SH + e % NH] = __float2bfloat16_rn(w);
    S.W2f[e] = w;
  }
  for (int e = tid; e < 8 * NH; e += kThreads) {
    const int j = e / NH, k = e % NH;
    const float w = j < NOUT ? params[O_W3 + j * NH + k] : 0.f;
    S.W3b[j * SH + k] = __float2bfloat16_rn(w);
    if (j < NOUT) S.W3f[j * NH + k] = w;
  }
  // persistent loop over tiles of 128 samples; the weights above are staged once per CTA
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
  const long long base = tile * kRows;
  __syncthreads();
  // ---- stage the samples
  for (int e = tid; e < kRows * NF; e += kThreads) {
    const int r = e / NF, k = e % NF;
    long long i = base + r;
    float v = 0.f;
    bool valid;
    if (sample) {
      i = (long long)(mix64(seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(base + r + 1)) %
                      (unsigned long long)n);
      valid = true;
    } else {
      valid = i < n;
    }
    if (valid) v = feats[i * NF + k];
    S.Xb[r * SX + k] = __float2bfloat16_rn(v);
    if (k < 4) {
      float y = 0.f, m = 0.f;
      if (mode == 1 && valid && k < NOUT) {
        y = labels[i * NOUT + k];
        m = mask[i * NOUT + k];
      }
      S.Y[r * 4 + k] = y;
      S.M[r * 4 + k] = m;
    }
  }
  __syncthreads();

  const int r0 = warp * 16;
  // ---- layer 1: H1 = relu(X W1^T + b1)
  {
    float acc[8][4] = {};
    warp_mma<8, NF>(S.Xb, SX, r0, S.W1b, SX, acc);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int c = nt * 8 + 2 * t;
      const float b0 = params[O_B1 + c], b1 = params[O_B1 + c + 1];
      S.H1b[(r0 + g) * SH + c] = __float2bfloat16_rn(fmaxf(acc[nt][0] + b0, 0.f));
      S.H1b[(r0 + g) * SH + c + 1] = __float2bfloat16_rn(fmaxf(acc[nt][1] + b1, 0.f));
      S.H1b[(r0 + g + 8) * SH + c] = __float2bfloat16_rn(fmaxf(acc[nt][2] + b0, 0.f));
      S.H1b[(r0 + g + 8) * SH + c + 1] = __float2bfloat16_rn(fmaxf(acc[nt][3] + b1, 0.f));
    }
  }
  __syncwarp();
  // ---- layer 2: H2 = relu(H1 W2^T + b2)
  {
    float acc[8][4] = {};
    warp_mma<8, NH>(S.H1b, SH, r0, S.W2b, SH, acc);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int c = nt * 8 + 2 * t;
      const float b0 = params[O_B2 + c], b1 = params[O_B2 + c + 1];
      S.H2b[(r0 + g) * SH + c] = __float2bfloat16_rn(fmaxf(acc[nt][0] + b0, 0.f));
      S.H2b[(r0 + g) * SH + c + 1] = __float2bfloat16_rn(fmaxf(acc[nt][1] + b1, 0.f));
      S.H2b[(r0 + g + 8) * SH + c] = __float2bfloat16_rn(fmaxf(acc[nt][2] + b0, 0.f));
      S.H2b[(r0 + g + 8) * SH + c + 1] = __float2bfloat16_rn(fmaxf(acc[nt][3] + b1, 0.f));
    }
  }
  __syncwarp();
  // ---- layer 3: O = sigmoid(H2 W3^T + b3) (8 padded output columns, 3 used)
  {
    float acc[1][4] = {};
    warp_mma<1, NH>(S.H2b, SH, r0, S.W3b, SH, acc);
    const int c = 2 * t;
    const float zz[4] = {acc[0][0], acc[0][1], acc[0][2], acc[0][3]};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int row = r0 + g + (q >= 2 ? 8 : 0), col = c + (q & 1);
      if (col < NOUT) {
        const float z = zz[q] + params[O_B3 + col];
        S.O[row * 4 + col] = 1.f / (1.f + __expf(-z));
      }
    }
  }
  __syncthreads();

  if (mode == 0) {
    for (int e = tid; e < kRows * NOUT; e += kThreads) {
      const int r = e / NOUT, j = e % NOUT;
      if (base + r < n) out[(base + r) * NOUT + j] = S.O[r * 4 + j];
    }
    continue;
  }

  // ---- backward (FP32 CUDA cores)
  float lsum = 0.f;
  for (int e = tid; e < kRows * NOUT; e += kThreads) {
    const int r = e / NOUT, j = e % NOUT;
    const float o = S.O[r * 4 + j], m = S.M[r * 4 + j], d = o - S.Y[r * 4 + j];
    lsum += m * d * d;
    S.dZ3[r * 4 + j] = 2.f * m * d * inv_norm * o * (1.f - o);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) S.red[warp] = lsum;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) s += S.red[w];
    atomicAdd(loss, s * inv_norm);
  }
  // dW3, db3
  if (tid < NOUT * NH) {
    const int j = tid / NH, k = tid % NH;
    float s = 0.f;
    for (int r = 0; r < kRows; ++r) s += S.dZ3[r * 4 + j] * __bfloat162float(S.H2b[r * SH + k]);
    atomicAdd(&grads[O_W3 + j * NH + k], s);
  } else if (tid < NOUT * NH + NOUT) {
    const int j = tid - NOUT * NH;
    float s = 0.f;
    for (int r = 0; r < kRows; ++r) s += S.dZ3[r * 4 + j];
    atomicAdd(&grads[O_B3 + j], s);
  }
  // dZ2 = (dZ3 W3) * [H2 > 0]
  for (int e = tid; e < kRows * NH; e += kThreads) {
    const int r = e / NH, k = e % NH;
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < NOUT; ++j) s += S.dZ3[r * 4 + j] * S.W3f[j * NH + k];
    S.dZ2[r * SD + k] = __bfloat162float(S.H2b[r * SH + k]) > 0.f ? s : 0.f;
  }
  __syncthreads();
  // dW2, db2
  for (int e = tid; e < NH * NH; e += kThreads) {
    const int m = e / NH, k = e % NH;
    float s = 0.f;
    for (int r = 0; r < kRows; ++r) s += S.dZ2[r * SD + m] * __bfloat162float(S.H1b[r * SH + k]);
    atomicAdd(&grads[O_W2 + e], s);
  }
  if (tid < NH) {
    float s = 0.f;
    for (int r = 0; r < kRows; ++r) s += S.dZ2[r * SD + tid];
    atomicAdd(&grads[O_B2 + tid], s);
  }
  // dZ1 = (dZ2 W2) * [H1 > 0]
  for (int e = tid; e < kRows * NH; e += kThreads) {
    const int r = e / NH, k = e % NH;
    float s = 0.f;
    for (int m = 0; m < NH; ++m) s += S.dZ2[r * SD + m] * S.W2f[m * NH + k];
    S.dZ1[r * SD + k] = __bfloat162float(S.H1b[r * SH + k]) > 0.f ? s : 0.f;
  }
  __syncthreads();
  // dW1, db1
  for (int e = tid; e < NH * NF; e += kThreads) {
    const int m = e / NF, k = e % NF;
    float s = 0.f;
    for (int r = 0; r < kRows; ++r) s += S.dZ1[r * SD + m] * __bfloat162float(S.Xb[r * SX + k]);
    atomicAdd(&grads[O_W1 + e], s);
  }
  if (tid < NH) {
    float s = 0.f;
    for (int r = 0; r < kRows; ++r) s += S.dZ1[r * SD + tid];
    atomicAdd(&grads[O_B1 + tid], s);
  }
  }  // tiles
}

// Inference alone: the forward pass of k_mlp (same BF16 roundings, same MMA sequence, same
// epilogues, so the same outputs) with each warp working through its own tiles of 16 samples.
// Without the backward buffers a block needs 44 KB of shared memory instead of k_mlp's, so
// more blocks share an SM, and no block-wide barrier stands between a warp's tiles.
constexpr int kWarpRows = 16;
struct MlpInferSmem {
  __nv_bfloat16 W1b[NH * SX];
  __nv_bfloat16 W2b[NH * SH];
  __nv_bfloat16 W3b[8 * SH];
  __nv_bfloat16 Xb[kThreads / 32][kWarpRows * SX];
  __nv_bfloat16 Hb[kThreads / 32][kWarpRows * SH];  // layer-1 output, then layer 2's in place
};

__global__ void __launch_bounds__(kThreads)
k_mlp_infer(const float* __restrict__ params, int n, const float* __restrict__ feats,
            float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpInferSmem& S = *reinterpret_cast<MlpInferSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  for (int e = tid; e < NH * NF; e += kThreads)
    S.W1b[(e / NF) * SX + e % NF] = __float2bfloat16_rn(params[O_W1 + e]);
  for (int e = tid; e < NH * NH; e += kThreads)
    S.W2b[(e / NH) * SH + e % NH] = __float2bfloat16_rn(params[O_W2 + e]);
  for (int e = tid; e < 8 * NH; e += kThreads) {
    const int j = e / NH, k = e % NH;
    S.W3b[j * SH + k] = __float2bfloat16_rn(j < NOUT ? params[O_W3 + j * NH + k] : 0.f);
  }
  __syncthreads();
  __nv_bfloat16* X = S.Xb[warp];
  __nv_bfloat16* H = S.Hb[warp];
  const long long tiles = ((long long)n + kWarpRows - 1) / kWarpRows;
  for (long long tile = (long long)blockIdx.x * (kThreads / 32) + warp; tile < tiles;
       tile += (long long)gridDim.x * (kThreads / 32)) {
    const long long base = tile * kWarpRows;
    __syncwarp();                                  // the previous tile's reads are done
    for (int e = lane; e < kWarpRows * NF; e += 32) {
      const int r = e / NF, k = e % NF;
      const long long i = base + r;
      X[r * SX + k] = __float2bfloat16_rn(i < n ? feats[i * NF + k] : 0.f);
    }
    __syncwarp();
    {
      float acc[8][4] = {};
      warp_mma<8, NF>(X, SX, 0, S.W1b, SX, acc);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int c = nt * 8 + 2 * t;
        const float b0 = params[O_B1 + c], b1 = params[O_B1 + c + 1];
        H[g * SH + c] = __float2bfloat16_rn(fmaxf(acc[nt][0] + b0, 0.f));
        H[g * SH + c + 1] = __float2bfloat16_rn(fmaxf(acc[nt][1] + b1, 0.f));
        H[(g + 8) * SH + c] = __float2bfloat16_rn(fmaxf(acc[nt][2] + b0, 0.f));
        H[(g + 8) * SH + c + 1] = __float2bfloat16_rn(fmaxf(acc[nt][3] + b1, 0.f));
      }
    }
    __syncwarp();
    {
      float acc[8][4] = {};
      warp_mma<8, NH>(H, SH, 0, S.W2b, SH, acc);
      __syncwarp();                                // layer 1's values are all read
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int c = nt * 8 + 2 * t;
        const float b0 = params[O_B2 + c], b1 = params[O_B2 + c + 1];
        H[g * SH + c] = __float2bfloat16_rn(fmaxf(acc[nt][0] + b0, 0.f));
        H[g * SH + c + 1] = __float2bfloat16_rn(fmaxf(acc[nt][1] + b1, 0.f));
        H[(g + 8) * SH + c] = __float2bfloat16_rn(fmaxf(acc[nt][2] + b0, 0.f));
        H[(g + 8) * SH + c + 1] = __float2bfloat16_rn(fmaxf(acc[nt][3] + b1, 0.f));
      }
    }
    __syncwarp();
    {
      float acc[1][4] = {};
      warp_mma<1, NH>(H, SH, 0, S.W3b, SH, acc);
      const int c = 2 * t;
      const float zz[4] = {acc[0][0], acc[0][1], acc[0][2], acc[0][3]};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = g + (q >= 2 ? 8 : 0), col = c + (q & 1);
        const long long i = base + row;
        if (col < NOUT && i < n) {
          const float z = zz[q] + params[O_B3 + col];
          out[i * NOUT + col] = 1.f / (1.f + __expf(-z));
        }
      }
    }
  }
}

__global__ void k_adam(int np, float* __restrict__ p, const float* __restrict__ gr,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    const float gg = gr[i];
    const float mi = b1 * m[i] + (1.f - b1) * gg;
    const float vi = b2 * v[i] + (1.f - b2) * gg * gg;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// Features of every regional node of a level (layout described at the top of the file).
template <int KIND>
__global__ void __launch_bounds__(kTile)
k_features(Grid G, const double* __restrict__ coef, const uint8_t* __restrict__ mult,
           const int* __restrict__ gid, const int* __restrict__ cgrp, const int* __restrict__ gptr,
           const int* __restrict__ gslot, float* __restrict__ feats) {
  using St = Sten<KIND>;
  RMG_FOR_NODES(G)
    int x[3];
    decode(li, R, x[0], x[1], x[2]);
    const int stride[3] = {1, R.nx, R.nx * R.ny};
    float* f = feats + (size_t)n * NF;
    const double dn = comp_coupling<KIND>(coef, G.n_r, n, St::CENTER, mult, gid, cgrp, gptr, gslot);
    const double dref = dn > 0.0 ? dn : 1.0;
    const double inv_ref = 1.0 / dref;            // one FP64 division per node, not 21
    const int len[3] = {R.nx, R.ny, R.nz};
    for (int a = 0; a < 3; ++a) {
      int rem = a < St::DIM ? x[a] % 3 : 0;
      if (rem && x[a] - rem + 3 > len[a] - 1) rem = 0;   // no right coarse node in the region
      const int slot = sten_slot<KIND>(a == 0, a == 1, a == 2);
      if (!rem || slot < 0) {
        for (int q = 0; q < 9; ++q) f[9 * a + q] = 0.f;
        continue;
      }
      const int p0 = n - rem * stride[a];
      // ratios in FP64, logarithms in FP32 (the features are FP32 network inputs)
      for (int e = 0; e < 3; ++e) {
        const double k = -comp_coupling<KIND>(coef, G.n_r, p0 + e * stride[a], slot, mult, gid,
                                              cgrp, gptr, gslot);
        const float v = log10f(fmaxf((float)(k * inv_ref), 1e-12f));
        f[9 * a + e] = fminf(v, 2.f);
      }
      for (int i = 0; i < 4; ++i) {
        const double d = comp_coupling<KIND>(coef, G.n_r, p0 + i * stride[a], St::CENTER, mult,
                                             gid, cgrp, gptr, gslot);
        const float v = log10f(fmaxf((float)(d * inv_ref), 1e-12f));
        f[9 * a + 3 + i] = fminf(v, 12.f);
      }
      f[9 * a + 7] = (float)(rem / 3.0);
      f[9 * a + 8] = 1.f;
    }
    for (int q = 27; q < NF; ++q) f[q] = 0.f;
  RMG_END_FOR_NODES
}

// Predicted weights -> per-axis interpolation weights (0 along inactive axes).
__global__ void k_weights_from_out(int n_r, const float* __restrict__ feats,
                                   const float* __restrict__ out, float* __restrict__ wr) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < n_r; n += gridDim.x * blockDim.x)
    for (int a = 0; a < 3; ++a)
      wr[(size_t)a * n_r + n] = feats[(size_t)n * NF + 9 * a + 8] > 0.5f ? out[n * 3 + a] : 0.f;
}

size_t mlp_smem() { return sizeof(MlpSmem); }

}  // namespace
}  // namespace rmg

using namespace rmg;

struct rmg_mlp {
  rmg_ctx* ctx = nullptr;
  DBuf<float> p, g, m, v, loss;
  int steps_done = 0;
};

namespace {
template <class F>
rmg_status mlp_guard(rmg_ctx* ctx, F&& f) {
  if (!ctx) return RMG_ERR_ARG;
  try {
    RMG_CUDA(cudaSetDevice(ctx->c.device));
    f();
    ctx->c.last_error.clear();
    return RMG_OK;
  } catch (const Error& e) {
    ctx->c.last_error = e.what();
    return e.status;
  } catch (const std::exception& e) {
    ctx->c.last_error = e.what();
    return RMG_ERR_CUDA;
  }
}

void mlp_launch(rmg_mlp* net, int n, const float* feats, const float* labels, const float* mask,
                int mode, int sample, int rows, unsigned long long seed, float inv_norm,
                float* out, float* loss) {
  Ctx& c = net->ctx->c;
  if (mode == 0 && !sample) {                    // inference over samples 0 .. n-1
    const int smem = (int)sizeof(MlpInferSmem);
    RMG_CUDA(cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smem));
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_infer, kThreads, smem) !=
        cudaSuccess) {
      cudaGetLastError();
      per_sm = 1;
    }
    const long long warps = ((long long)n + kWarpRows - 1) / kWarpRows;
    const long long want = (warps + kThreads / 32 - 1) / (kThreads / 32);
    const int blocks = (int)std::max<long long>(
        1, std::min<long long>(want, (long long)c.nsm * std::max(1, per_sm)));
    k_mlp_infer<<<blocks, kThreads, smem, c.stream>>>(net->p.get(), n, feats, out);
    RMG_LAUNCHED();
    return;
  }
  const int smem = (int)mlp_smem();
  RMG_CUDA(cudaFuncSetAttribute(k_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const long long tiles = (rows + kRows - 1) / kRows;
  const int blocks = (int)std::min<long long>(tiles, (long long)c.nsm * 2);
  k_mlp<<<blocks, kThreads, smem, c.stream>>>(net->p.get(), n, tiles, feats, labels, mask, mode,
                                             sample, seed, inv_norm, out, net->g.get(), loss);
  RMG_LAUNCHED();
}
}  // namespace

extern "C" {

int rmg_mlp_num_params(void) { return NPARAMS; }

rmg_status rmg_mlp_create(rmg_ctx* ctx, const float* init_params, rmg_mlp** out) {
  if (!out) return RMG_ERR_ARG;
  *out = nullptr;
  rmg_mlp* net = new (std::nothrow) rmg_mlp();
  if (!net) return RMG_ERR_NOMEM;
  net->ctx = ctx;
  rmg_status st = mlp_guard(ctx, [&] {
    RMG_REQUIRE(init_params, RMG_ERR_ARG, "init_params is NULL");
    net->p.alloc(NPARAMS); net->g.alloc(NPARAMS); net->m.alloc(NPARAMS); net->v.alloc(NPARAMS);
    RMG_CUDA(cudaMemcpy(net->p.get(), init_params, NPARAMS * sizeof(float), cudaMemcpyHostToDevice));
    RMG_CUDA(cudaMemset(net->m.get(), 0, NPARAMS * sizeof(float)));
    RMG_CUDA(cudaMemset(net->v.get(), 0, NPARAMS * sizeof(float)));
  });
  if (st != RMG_OK) {
    delete net;
    return st;
  }
  *out = net;
  return RMG_OK;
}

void rmg_mlp_destroy(rmg_mlp* net) { delete net; }

rmg_status rmg_mlp_get_params(rmg_mlp* net, float* params) {
  if (!net || !params) return RMG_ERR_ARG;
  return mlp_guard(net->ctx, [&] {
    RMG_CUDA(cudaStreamSynchronize(net->ctx->c.stream));
    RMG_CUDA(cudaMemcpy(params, net->p.get(), NPARAMS * sizeof(float), cudaMemcpyDeviceToHost));
  });
}

rmg_status rmg_mlp_forward(rmg_mlp* net, int n, const float* feats, float* out) {
  if (!net) return RMG_ERR_ARG;
  return mlp_guard(net->ctx, [&] {
    RMG_REQUIRE(n > 0 && feats && out, RMG_ERR_ARG, "bad arguments");
    mlp_launch(net, n, feats, nullptr, nullptr, 0, 0, n, 0, 0.f, out, nullptr);
  });
}

rmg_status rmg_mlp_gradient(rmg_mlp* net, int n, const float* feats, const float* labels,
                            const float* mask, float* grad, float* loss) {
  if (!net) return RMG_ERR_ARG;
  return mlp_guard(net->ctx, [&] {
    RMG_REQUIRE(n > 0 && feats && labels && mask && grad && loss, RMG_ERR_ARG, "bad arguments");
    Ctx& c = net->ctx->c;
    net->loss.ensure(1);
    RMG_CUDA(cudaMemsetAsync(net->g.get(), 0, NPARAMS * sizeof(float), c.stream));
    RMG_CUDA(cudaMemsetAsync(net->loss.get(), 0, sizeof(float), c.stream));
    mlp_launch(net, n, feats, labels, mask, 1, 0, n, 0, 1.f / (3.f * n), nullptr, net->loss.get());
    RMG_CUDA(cudaStreamSynchronize(c.stream));
    RMG_CUDA(cudaMemcpy(grad, net->g.get(), NPARAMS * sizeof(float), cudaMemcpyDeviceToHost));
    RMG_CUDA(cudaMemcpy(loss, net->loss.get(), sizeof(float), cudaMemcpyDeviceToHost));
  });
}

rmg_status rmg_mlp_train(rmg_mlp* net, int n, const float* feats, const float* labels,
                         const float* mask, int steps, int batch, float lr,
                         unsigned long long seed, float* loss_history) {
  if (!net) return RMG_ERR_ARG;
  return mlp_guard(net->ctx, [&] {
    RMG_REQUIRE(n > 0 && feats && labels && mask && steps > 0, RMG_ERR_ARG, "bad arguments");
    RMG_REQUIRE(batch >= kRows && batch % kRows == 0, RMG_ERR_ARG, "batch must be a multiple of 128");
    Ctx& c = net->ctx->c;
    net->loss.ensure((size_t)steps);
    RMG_CUDA(cudaMemsetAsync(net->loss.get(), 0, sizeof(float) * steps, c.stream));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int s = 0; s < steps; ++s) {
      RMG_CUDA(cudaMemsetAsync(net->g.get(), 0, NPARAMS * sizeof(float), c.stream));
      mlp_launch(net, n, feats, labels, mask, 1, 1, batch,
                 seed * 0x100000001B3ull + (unsigned long long)(net->steps_done + s) * batch,
                 1.f / (3.f * batch), nullptr, net->loss.get() + s);
      const int t = net->steps_done + s + 1;
      const float c1 = 1.f / (1.f - powf(b1, (float)t)), c2 = 1.f / (1.f - powf(b2, (float)t));
      k_adam<<<(NPARAMS + 255) / 256, 256, 0, c.stream>>>(NPARAMS, net->p.get(), net->g.get(),
                                                         net->m.get(), net->v.get(), lr, b1, b2,
                                                         eps, c1, c2);
      RMG_LAUNCHED();
    }
    net->steps_done += steps;
    RMG_CUDA(cudaStreamSynchronize(c.stream));
    if (loss_history)
      RMG_CUDA(cudaMemcpy(loss_history, net->loss.get(), sizeof(float) * steps,
                          cudaMemcpyDeviceToHost));
  });
}

rmg_status rmg_hier_mlp_features(rmg_hier* hh, int level, float* feats) {
  if (!hh) return RMG_ERR_ARG;
  return mlp_guard(hh->h.layout->ctx, [&] {
    Hier& h = hh->h;
    RMG_REQUIRE(level >= 0 && level < h.levels() && feats, RMG_ERR_ARG, "bad arguments");
    Level& L = *h.lv[level];
    const Grid G = L.grid();
    const int gb = persistent_grid(*h.c, G.ntiles);
#define RMG_FEAT(K)                                                                            \
  k_features<K><<<gb, kTile, 0, h.c->stream>>>(G, L.coef.get(), L.mult.get(), L.gid.get(),     \
                                               L.cgrp.get(), L.gptr.get(), L.gslot.get(), feats)
    switch (L.kind) {
      case 5: RMG_FEAT(5); break;
      case 7: RMG_FEAT(7); break;
      case 9: RMG_FEAT(9); break;
      default: RMG_FEAT(27); break;
    }
#undef RMG_FEAT
    RMG_LAUNCHED();
  });
}

rmg_status rmg_hier_mlp_weights(rmg_hier* hh, int level, rmg_mlp* net, float* wr) {
  if (!hh || !net) return RMG_ERR_ARG;
  Hier& h = hh->h;
  const int n_r = (level >= 0 && level < h.levels()) ? h.lv[level]->n_r : 0;
  rmg_status st = mlp_guard(h.layout->ctx, [&] {
    RMG_REQUIRE(n_r > 0 && wr, RMG_ERR_ARG, "bad arguments");
    h.mlp_feats.ensure((size_t)h.lv[0]->n_r * NF);       // sized for the finest level, kept
    h.mlp_out.ensure((size_t)h.lv[0]->n_r * 3);
  });
  if (st != RMG_OK) return st;
  st = rmg_hier_mlp_features(hh, level, h.mlp_feats.get());
  if (st != RMG_OK) return st;
  return mlp_guard(h.layout->ctx, [&] {
    mlp_launch(net, n_r, h.mlp_feats.get(), nullptr, nullptr, 0, 0, n_r, 0, 0.f,
               h.mlp_out.get(), nullptr);
    k_weights_from_out<<<persistent_grid(*h.c, (n_r + 255) / 256), 256, 0, h.c->stream>>>(
        n_r, h.mlp_feats.get(), h.mlp_out.get(), wr);
    RMG_LAUNCHED();
  });
}

}  // extern "C"
