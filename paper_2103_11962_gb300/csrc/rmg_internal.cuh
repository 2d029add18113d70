// Internal declarations of the region multigrid library (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "rmg.h"

namespace rmg {

// ------------------------------------------------------------------------------ errors
struct Error : std::runtime_error {
  rmg_status status;
  Error(rmg_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define RMG_CUDA(x)                                                                        \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess)                                                                 \
      throw ::rmg::Error(e_ == cudaErrorMemoryAllocation ? RMG_ERR_NOMEM : RMG_ERR_CUDA,   \
                         std::string(#x) + ": " + cudaGetErrorString(e_));                 \
  } while (0)
// Kernel launches issued by the library (graph replays add the kernels of the graph).
extern unsigned long long g_launches;
extern bool g_capturing;
#define RMG_LAUNCHED()                                  \
  do {                                                  \
    RMG_CUDA(cudaGetLastError());                       \
    if (!::rmg::g_capturing) ++::rmg::g_launches;        \
  } while (0)
#define RMG_REQUIRE(cond, st, msg)                     \
  do {                                                 \
    if (!(cond)) throw ::rmg::Error((st), (msg));      \
  } while (0)

// Device-side error codes written to Ctx::d_err (first error wins).
enum DevErr : int {
  DERR_NONE = 0,
  DERR_GID_RANGE = 1,       // a gid outside [0, n_composite)
  DERR_UNCOVERED = 2,       // a composite node in no region
  DERR_MULT = 3,            // more than 255 copies
  DERR_STENCIL = 4,         // CSR entry outside the declared stencil
  DERR_COARSE_MISMATCH = 5, // co-located nodes disagree on being coarse points
  DERR_NOT_SPD = 6,         // non-positive pivot in the coarse Cholesky
};

// ------------------------------------------------------------------------------ buffers
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  explicit DBuf(size_t count) { alloc(count); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count) {
    release();
    if (count) RMG_CUDA(cudaMalloc(&p, count * sizeof(T)));
    n = count;
  }
  // Keep the allocation when it already has `count` elements (pointers captured in a CUDA
  // graph stay valid); otherwise reallocate.
  void ensure(size_t count) {
    if (n != count || (count && !p)) alloc(count);
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  T* get() const { return p; }
  size_t bytes() const { return n * sizeof(T); }
};

// ------------------------------------------------------------------------------ stencils
// Slot orders (coefficient s of node n couples n to n + offset(s)):
//   7-point : (-z, -y, -x, 0, +x, +y, +z)          5-point : (-y, -x, 0, +x, +y)
//   27-point: s = (dx+1) + 3(dy+1) + 9(dz+1)       9-point : s = (dx+1) + 3(dy+1)
template <int KIND> struct Sten;
template <> struct Sten<7> {
  static constexpr int S = 7, CENTER = 3, DIM = 3;
  __host__ __device__ static constexpr int dx(int s) { return s == 2 ? -1 : (s == 4 ? 1 : 0); }
  __host__ __device__ static constexpr int dy(int s) { return s == 1 ? -1 : (s == 5 ? 1 : 0); }
  __host__ __device__ static constexpr int dz(int s) { return s == 0 ? -1 : (s == 6 ? 1 : 0); }
};
template <> struct Sten<5> {
  static constexpr int S = 5, CENTER = 2, DIM = 2;
  __host__ __device__ static constexpr int dx(int s) { return s == 1 ? -1 : (s == 3 ? 1 : 0); }
  __host__ __device__ static constexpr int dy(int s) { return s == 0 ? -1 : (s == 4 ? 1 : 0); }
  __host__ __device__ static constexpr int dz(int) { return 0; }
};
template <> struct Sten<27> {
  static constexpr int S = 27, CENTER = 13, DIM = 3;
  __host__ __device__ static constexpr int dx(int s) { return s % 3 - 1; }
  __host__ __device__ static constexpr int dy(int s) { return (s / 3) % 3 - 1; }
  __host__ __device__ static constexpr int dz(int s) { return s / 9 - 1; }
};
template <> struct Sten<9> {
  static constexpr int S = 9, CENTER = 4, DIM = 2;
  __host__ __device__ static constexpr int dx(int s) { return s % 3 - 1; }
  __host__ __device__ static constexpr int dy(int s) { return s / 3 - 1; }
  __host__ __device__ static constexpr int dz(int) { return 0; }
};

// Slot of offset (dx, dy, dz) in stencil KIND, or -1.
template <int KIND>
__host__ __device__ inline int sten_slot(int dx, int dy, int dz) {
  for (int s = 0; s < Sten<KIND>::S; ++s)
    if (Sten<KIND>::dx(s) == dx && Sten<KIND>::dy(s) == dy && Sten<KIND>::dz(s) == dz) return s;
  return -1;
}

// Galerkin coarse stencil of a fine stencil: 7 -> 27, 27 -> 27 (3D); 5 -> 9, 9 -> 9 (2D).
inline int coarse_kind(int kind) { return (kind == 5 || kind == 9) ? 9 : 27; }

// ------------------------------------------------------------------------------ geometry
struct RegionDev {
  int nx, ny, nz, pad;
  int off;     // first regional node of the region
  float rnx, rny;   // 1/nx, 1/ny for the division-free index decode (0: exact integer path)
};

// Region descriptor with the reciprocals of decode(): regions of fewer than 2^22 nodes take the
// float path (exact after one correction step), larger ones the integer division.
__host__ __device__ inline RegionDev make_region(int nx, int ny, int nz, int off) {
  const bool fast = (long long)nx * ny * nz < (1LL << 22);
  return RegionDev{nx, ny, nz, 0, off, fast ? 1.0f / (float)nx : 0.0f,
                   fast ? 1.0f / (float)ny : 0.0f};
}

// A tile of one region: in run mode (Grid::lx < 0) up to kTile consecutive nodes from `start`;
// in box mode a tx x ty x tz box of nodes with corner (x0, y0, z0), tx * ty * tz = kTile.
struct Tile {
  int region;
  int start;              // run mode: local start inside the region
  short x0, y0, z0, pad;  // box mode: corner of the box
};

constexpr int kTile = 256;

// Everything a node-parallel kernel needs to locate node (region, i, j, l).
struct Grid {
  const RegionDev* regions;
  const Tile* tiles;
  int ntiles;
  int nreg;
  int n_r;
  int lx = -1, ly = 0;    // box mode: tx = 2^lx, ty = 2^ly, tz = kTile / (tx ty); lx < 0: runs
};

struct Ctx;

// One level of the regional hierarchy.
struct Level {
  int dim = 3;
  int kind = 7;                  // stencil points stored per node (per block)
  int B = 1;                     // dofs per node (3 for elasticity): B x B blocks of stencils
  int nreg = 0;
  std::vector<int> hdims;        // 3 per region
  std::vector<int> hoff;         // nreg + 1
  int n_r = 0;
  int ncomp = 0;                 // composite id space of this level
  std::vector<Tile> htiles;
  DBuf<RegionDev> regions;
  DBuf<Tile> tiles;
  // layout (Psi)
  DBuf<int> gid;                 // composite id per regional node
  DBuf<uint8_t> mask;            // Dirichlet flag per regional node
  DBuf<uint8_t> mult;            // copies of the co-located composite node
  DBuf<int> c2r;                 // composite -> lowest regional slot
  DBuf<int> cgrp;                // composite -> interface group or -1
  int ngroups = 0, nslots = 0;
  DBuf<int> gptr;                // ngroups + 1
  DBuf<int> gslot;               // regional slots of every group, ascending
  DBuf<int> rid;                 // region of every regional node (built for the split)
  DBuf<int> sgrp;                // group of every group slot (nslots)
  DBuf<int4> affine;             // per region {g0, gy, gz, ok}: gid = g0 + i + gy j + gz l
  // operator
  DBuf<double> coef;             // kind * n_r, slot-major
  DBuf<double> dinv;             // 1 / (Psi^T Psi diag([[A]]))
  // single precision copies for the mixed-precision cycle
  DBuf<float> coef32;
  DBuf<__nv_bfloat16> coef16;
  DBuf<float> dinv32;

  Grid grid() const { return Grid{regions.get(), tiles.get(), (int)htiles.size(), nreg, n_r, -1, 0}; }
};

// Device-resident scalars of the solver (no host round trip inside a V-cycle or a CG step).
struct Scalars {
  double lam[16];          // power-method estimate per level
  double cheb_c1[16][8];   // Chebyshev d <- c1 d + c2 D^-1 r, per level and step
  double cheb_c2[16][8];
  float cheb_c1f[16][8];   // the same coefficients rounded to FP32 for the FP32 cycle
  float cheb_c2f[16][8];
  double pw_norm, pw_inv;  // power method scratch (norm and its reciprocal)
  double pw_num, pw_den;
  double rz, pq, alpha, beta, rr, bb, rz_new;
  int half_asym;           // level-0 FP32 stencil not bitwise symmetric (full planes in use)
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int nsm = 152;
  std::string last_error;
  DBuf<int> d_err;                // device error flag
  DBuf<double> partials;          // block partial sums for reductions
  int max_partials = 0;
  void check_device_error(const char* where);
};

int persistent_grid(const Ctx& c, int work_items, int per_sm = 8);

// ------------------------------------------------------------------------------ scans
// Exclusive prefix sum of n ints; returns the total (synchronises).
int exclusive_scan(Ctx& c, const int* in, int* out, int n);

}  // namespace rmg

// Opaque handles of the C ABI.
struct rmg_ctx {
  rmg::Ctx c;
};

struct rmg_layout {
  rmg_ctx* ctx = nullptr;
  rmg::Level L0;
  bool has_operator = false;
  rmg::DBuf<double> ybuf;         // interface partials for rmg_regional_apply
  rmg::DBuf<double> tmp;          // composite temp
  rmg::DBuf<double> apbuf;        // Galerkin-product scratch (rows of [[A]][[P]]), all hierarchies
  // device copies of a host composite CSR (rmg_operator_from_host_csr)
  rmg::DBuf<int64_t> csr_rowptr, csr_col;
  rmg::DBuf<double> csr_val;
};
