// The regional multigrid hierarchy and its solve phase.
#pragma once

#include <memory>

#include "rmg_internal.cuh"

namespace rmg {

// Work vectors of one level in the cycle's arithmetic type VT.
template <typename VT>
struct LevelVecs {
  DBuf<VT> u, u2, b, r, y, d;
  void alloc(int n) {
    u.alloc(n); u2.alloc(n); b.alloc(n); r.alloc(n); y.alloc(n); d.alloc(n);
  }
};

// Stencil-sweep tile shapes (index 0: runs of kTile consecutive nodes; 1..8: boxes
// 2^lx x 2^ly x kTile / 2^(lx + ly); 9: 32 x 8 columns through all z-planes of a region,
// staged in shared memory (k_stencil_half27_staged), marked lx = -3), in the order
// rmg_options.tile_shape numbers them.
struct TileShape { int lx, ly; };
constexpr TileShape kTileShapes[] = {{-1, 0}, {5, 3}, {6, 2}, {7, 1}, {4, 4},
                                     {5, 2}, {4, 3}, {4, 2}, {3, 3}, {-3, 0}};
constexpr int kStagedShape = 9;
constexpr int kNumTileShapes = (int)(sizeof(kTileShapes) / sizeof(kTileShapes[0]));
static_assert(kNumTileShapes == RMG_NUM_TILE_SHAPES, "tile shape table and header disagree");

struct Hier {
  rmg_layout* layout = nullptr;
  Ctx* c = nullptr;
  rmg_options o{};
  std::vector<std::unique_ptr<Level>> own;   // levels 1..L-1
  std::vector<Level*> lv;                    // all levels; lv[0] is the layout's level
  std::vector<LevelVecs<double>> v64;
  std::vector<LevelVecs<float>> v32;
  DBuf<Scalars> sc;
  Scalars hsc{};                             // host copy after setup
  // coarsest composite level
  int nc = 0;
  DBuf<int> cidx, cu2slot;
  DBuf<long long> cu2gid;
  DBuf<double> Mfac, X, Ainv, xc, rc;
  DBuf<double> Linv, Dblk, Tinv;             // L^-1, inverted 32 x 32 diagonal blocks, scratch
  // mixed-precision coarse solve: FP32 inverse of S Abar S (S = diag(Abar)^-1/2) and
  // coarse_refine FP64 refinement steps per solve; coarse_refine = 0: the FP64 inverse Ainv
  DBuf<double> cscale, cres, cnorm;
  DBuf<float> M32, Ainv32, Linv32, Tinv32, Dblk32, cw32;
  DBuf<int> cerr;
  int coarse_refine = 0;
  int graph_refine = -1;                     // coarse_refine the graph was captured with
  double coarse_rho = 0.0;                   // measured contraction of one refinement step
  // graph of one V-cycle
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t graph_stream = nullptr;
  int launches = 0;
  // stored transfer weights per level (to the next coarser level; linear 3:1 when not
  // stored): pw[l][a * n_r + n] = weight of the right coarse neighbour along axis a (FP32;
  // the entries of P are the FP32 products wz (wy wx) in every precision)
  std::vector<char> stored;
  std::vector<DBuf<float>> pw;
  std::vector<char> graph_stored;            // stored-transfer flags the graph was captured with
  // stencil-sweep tiles per level (autotuned shape; see kTileShapes): shape index and grid
  std::vector<int> shape;
  std::vector<DBuf<Tile>> stiles;
  std::vector<Grid> sgrid;
  bool tuned = false;
  bool dense_ok = true;                      // coarsest level within the dense solver
  int kind0 = 0;                             // level-0 stencil and buffer seen by the graph
  const double* coef0 = nullptr;
  // probe: CUDA events around one level-0 smoother stencil launch of every V-cycle
  cudaEvent_t probe_ev[2] = {nullptr, nullptr};
  bool probe_pending = false;
  double probe_ms = 0.0;
  long long probe_count = 0;
  // learned-prolongator inference scratch (features and network outputs)
  DBuf<float> mlp_feats, mlp_out;
  // per-region energies (tile ranges, tile partials, region sums) and accepted regions
  DBuf<int> energy_tiles;
  DBuf<double> energy_part, energy_out;
  DBuf<uint8_t> accept;
  // PCG work vectors (regional, FP64)
  DBuf<double> x, r, z, p, q, zold, tmp;
  DBuf<float> zold32;                        // previous FP32 cycle output (flexible CG)
  double* pinned = nullptr;                  // host-mapped residual read-back
  // FP32 cycle, scalar operator: level 0 also as half planes (k_level0_fp32), read by the sweeps
  // while the device flag Scalars::half_asym is 0
  bool half_on = false;
  DBuf<float> half32;

  ~Hier();
  int levels() const { return (int)lv.size(); }
  // tuned stencil-sweep grid of level l, or null (the level's run tiles) before tuning
  const Grid* sweep(int l) const {
    return l < (int)shape.size() && shape[l] >= 0 ? &sgrid[l] : nullptr;
  }
  bool mixed() const { return o.precision != RMG_PREC_FP64; }
  // half planes of level l for the FP32 sweeps, or null
  const float* half(int l) const { return (l == 0 && half_on) ? half32.get() : nullptr; }
  const int* half_flag() const;
};

void hier_build(Hier& h);          // symbolic: coarse layouts, buffers
void hier_numeric(Hier& h);        // numeric: diagonals, RAP, lambda, coarse factor, graph
void tile_shape(const Hier& h, int level, int* tx, int* ty, int* tz);
void galerkin_level(Hier& h, int level);   // one Galerkin product, level -> level + 1
// Largest dense coarse system (unknowns) the coarse solver factors.
constexpr long long kMaxDense = 16384;
void probe_collect(Hier& h);       // read the probe events of the last V-cycle
void vcycle(Hier& h);              // lv[0] rhs in v64[0].b (or v32[0].b) -> result in .u
void vcycle_apply(Hier& h, const double* r, double* z, int regional);
void set_transfer_weights(Hier& h, int level, const float* wr);
void opdep_weights(Hier& h, int level, float* wr);
void constant_weights(Hier& h, int level, float* wr);
double convergence_factor(Hier& h, int iters, unsigned long long seed);
void region_energies(Hier& h, int iters, unsigned long long seed, double* e0, double* eK);
void blend_weights(Hier& h, int level, const uint8_t* accept_host, const float* learned,
                   float* out);
int region_colours(Hier& h, int* colours);
void pcg_solve(Hier& h, const double* b, double* x, double rtol, int maxit, double* history,
               rmg_solve_info* info);

}  // namespace rmg

struct rmg_hier {
  rmg::Hier h;
};
