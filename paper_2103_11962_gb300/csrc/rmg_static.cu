// A regional operator apply that allocates no device memory.
//
// Some callers cannot call cudaMalloc when they need this operation: applications that hand
// all device memory to their own pool allocator, or real-time loops that cannot afford the
// device-wide synchronisation an allocation or a free can cause. rmg_regional_apply_static serves them: it
// takes plain arrays (no context, layout or hierarchy handle) and keeps its scratch in one
// fixed, file-scope device array that every GPU which loads the library holds until the
// process exits.
//
// Scratch layout (kStaticBytes in total):
//   [0, kTableBytes)            region table: offsets and dims of at most kStaticMaxRegions
//   [kTableBytes, kStaticBytes) composite accumulator: at most kStaticMaxComposite doubles
// Every call overwrites the table and zeroes the accumulator before use. Calls that overlap
// on the GPU (other streams, other host threads) share the array and race.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "rmg_kernels.cuh"

namespace rmg {
namespace {

constexpr int kStaticMaxRegions = 4096;
constexpr long long kStaticMaxComposite = 1LL << 22;                // 4,194,304 nodes
constexpr size_t kTableBytes = 192 * 1024;                          // region table + dims
constexpr size_t kStaticBytes = kTableBytes + sizeof(double) * (size_t)kStaticMaxComposite;
static_assert(sizeof(RegionDev) * kStaticMaxRegions + 3 * sizeof(int) * kStaticMaxRegions <=
                  kTableBytes, "region table does not fit");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Host-side address of g_static_scratch per device, taken once with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void* g_static_ptr[kMaxDevices] = {};

// Region dims (3 ints per region, copied after the table) -> RegionDev entries with offsets.
__global__ void k_static_table(int nreg, const int* __restrict__ dims, RegionDev* __restrict__ tab) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int off = 0;
  for (int r = 0; r < nreg; ++r) {
    tab[r] = make_region(dims[3 * r], dims[3 * r + 1], dims[3 * r + 2], off);
    off += dims[3 * r] * dims[3 * r + 1] * dims[3 * r + 2];
  }
}

__global__ void k_static_zero(long long n, double* __restrict__ acc) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    acc[k] = 0.0;
}

// Region stencil row of every regional node, summed into the composite accumulator: the
// sum over co-located copies (Psi [[A]] u) without precomputed interface groups.
template <int KIND>
__global__ void __launch_bounds__(256)
k_static_scatter(const RegionDev* __restrict__ tab, int nreg, int n_r,
                 const double* __restrict__ coef, const int64_t* __restrict__ gid,
                 long long ncomp, const double* __restrict__ u, double* __restrict__ acc) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < n_r; n += gridDim.x * blockDim.x) {
    const RegionDev R = tab[region_of(tab, nreg, n)];
    int i, j, l;
    decode(n - R.off, R, i, j, l);
    const double au = stencil_row<KIND, double, double, double>(coef, u, n, n_r, i, j, l, R);
    const int64_t g = gid[n];
    if (g >= 0 && g < ncomp) atomicAdd(&acc[g], au);
  }
}

// y = Psi^T acc; nodes with a gid outside [0, n_composite) receive NaN.
__global__ void k_static_gather(int n_r, const int64_t* __restrict__ gid, long long ncomp,
                                const double* __restrict__ acc, double* __restrict__ y) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < n_r; n += gridDim.x * blockDim.x) {
    const int64_t g = gid[n];
    y[n] = (g >= 0 && g < ncomp) ? acc[g] : __longlong_as_double(0x7ff8000000000000LL);
  }
}

rmg_status static_fail(char* msg, int msg_len, rmg_status st, const char* text) {
  if (msg && msg_len > 0) {
    std::strncpy(msg, text, (size_t)msg_len - 1);
    msg[msg_len - 1] = '\0';
  }
  return st;
}

}  // namespace
}  // namespace rmg

using namespace rmg;

extern "C" rmg_status rmg_regional_apply_static(int dim, int nregions, const int32_t* region_dims,
                                                int stencil, const double* coeffs,
                                                const int64_t* region_gids, int64_t n_composite,
                                                const double* u, double* y, void* cuda_stream,
                                                char* msg, int msg_len) {
  if (msg && msg_len > 0) msg[0] = '\0';
  if (!region_dims || !coeffs || !region_gids || !u || !y)
    return static_fail(msg, msg_len, RMG_ERR_ARG, "null pointer argument");
  if (!((dim == 2 && (stencil == 5 || stencil == 9)) || (dim == 3 && (stencil == 7 || stencil == 27))))
    return static_fail(msg, msg_len, RMG_ERR_ARG, "stencil must be 5/9 in 2D and 7/27 in 3D");
  if (nregions < 1 || nregions > kStaticMaxRegions)
    return static_fail(msg, msg_len, RMG_ERR_ARG,
                       "nregions must be in [1, 4096] (the static scratch holds 4096 regions)");
  if (n_composite < 1 || n_composite > kStaticMaxComposite)
    return static_fail(msg, msg_len, RMG_ERR_ARG,
                       "n_composite must be in [1, 4194304] (the static scratch holds 4194304 "
                       "composite nodes)");
  long long n_r = 0;
  for (int r = 0; r < nregions; ++r) {
    const int nx = region_dims[3 * r], ny = region_dims[3 * r + 1], nz = region_dims[3 * r + 2];
    if (nx < 1 || ny < 1 || nz < 1 || (dim == 2 && nz != 1))
      return static_fail(msg, msg_len, RMG_ERR_ARG, "bad region dims");
    n_r += (long long)nx * ny * nz;
  }
  if (n_r >= (1LL << 31)) return static_fail(msg, msg_len, RMG_ERR_ARG, "too many regional nodes");

  // the work runs on the device of the caller's stream (the current device for the legacy
  // default stream); that device is current for the rest of the call and the caller's device
  // is restored on return
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess)
    return static_fail(msg, msg_len, RMG_ERR_CUDA, "cudaGetDevice failed");
  int dev = prev;
  if (st && cudaStreamGetDevice(st, &dev) != cudaSuccess)
    return static_fail(msg, msg_len, RMG_ERR_CUDA, "cudaStreamGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices)
    return static_fail(msg, msg_len, RMG_ERR_CUDA, "device index out of range");
  if (dev != prev && cudaSetDevice(dev) != cudaSuccess)
    return static_fail(msg, msg_len, RMG_ERR_CUDA, "cudaSetDevice failed");
  struct RestoreDevice {
    int prev, dev;
    ~RestoreDevice() { if (dev != prev) cudaSetDevice(prev); }
  } restore{prev, dev};
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[dev]) {
      // once per device, with that device current: the device address of the scratch array
      cudaError_t e = cudaGetSymbolAddress(&g_static_ptr[dev], g_static_scratch);
      if (e != cudaSuccess) {
        g_static_ptr[dev] = nullptr;
        return static_fail(msg, msg_len, RMG_ERR_CUDA, cudaGetErrorString(e));
      }
    }
    base = g_static_ptr[dev];
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  RegionDev* tab = reinterpret_cast<RegionDev*>(b);
  int* dims_dev = reinterpret_cast<int*>(b + sizeof(RegionDev) * kStaticMaxRegions);
  double* acc = reinterpret_cast<double*>(b + kTableBytes);

  cudaError_t e = cudaMemcpyAsync(dims_dev, region_dims, sizeof(int) * 3 * (size_t)nregions,
                                  cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return static_fail(msg, msg_len, RMG_ERR_CUDA, cudaGetErrorString(e));
  k_static_table<<<1, 32, 0, st>>>(nregions, dims_dev, tab);
  const int nb = (int)std::min<long long>((n_r + 255) / 256, 152 * 8);
  const int zb = (int)std::min<long long>((n_composite + 255) / 256, 152 * 8);
  k_static_zero<<<zb, 256, 0, st>>>(n_composite, acc);
  switch (stencil) {
    case 5: k_static_scatter<5><<<nb, 256, 0, st>>>(tab, nregions, (int)n_r, coeffs, region_gids, n_composite, u, acc); break;
    case 7: k_static_scatter<7><<<nb, 256, 0, st>>>(tab, nregions, (int)n_r, coeffs, region_gids, n_composite, u, acc); break;
    case 9: k_static_scatter<9><<<nb, 256, 0, st>>>(tab, nregions, (int)n_r, coeffs, region_gids, n_composite, u, acc); break;
    default: k_static_scatter<27><<<nb, 256, 0, st>>>(tab, nregions, (int)n_r, coeffs, region_gids, n_composite, u, acc); break;
  }
  k_static_gather<<<nb, 256, 0, st>>>((int)n_r, region_gids, n_composite, acc, y);
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(msg, msg_len, RMG_ERR_CUDA, cudaGetErrorString(e));
  g_launches += 4;
  return RMG_OK;
}
