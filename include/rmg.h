/*
 * rmg.h - C ABI of a single-GPU region multigrid library (GB300, sm_103a).
 *
 * Method: "Non-invasive multigrid for semi-structured grids" (arXiv 2103.11962).
 * A composite matrix A on a mesh tiled by structured box regions is split into region
 * matrices (Sec. 4); interface nodes are duplicated in every region that contains them
 * (Sec. 3.1, the boolean map Psi). A regional V-cycle (Sec. 3.3 and the regional mgCycle
 * figure of Sec. 3.6) then runs region-locally: smoothing (Sec. 3.4), 3:1 structured
 * restriction and interpolation (Sec. 3.2, Sec. 3.3), Galerkin coarse operators computed per
 * region (eq. "RegionalGalerkinProduct", Theorem 1), and a dense direct solve of the
 * composite coarsest operator (Sec. 3.5). The only coupling between regions is the interface
 * summation Psi^T Psi. The V-cycle preconditions a conjugate-gradient solve.
 *
 * Conventions for every entry point:
 *  - Arrays named "device" are caller-owned CUDA device pointers on the context's device.
 *    "host" arrays are read during the call only. const pointers are never written.
 *  - All work is queued on the context's stream. Calls return once the work is queued,
 *    except where a function says it synchronises.
 *  - No C++ exception crosses the ABI. Every function returns an rmg_status. The message of
 *    the last failure is available from rmg_last_error().
 *  - Objects created by rmg_*_create / rmg_setup are owned by the caller and released with
 *    the matching destroy function. The library allocates its internal buffers with
 *    cudaMalloc on the context's device.
 *  - Vectors are FP64. A "regional" vector has one entry per regional node; regions are
 *    concatenated in region order and nodes inside a region are ordered x fastest. A
 *    "composite" vector has one entry per composite node (index = global id, gid).
 *  - A regional vector is "consistent" when all copies of an interface node hold the same
 *    value (it is Psi^T of a composite vector).
 */
#ifndef RMG_H
#define RMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rmg_ctx rmg_ctx;
typedef struct rmg_layout rmg_layout;
typedef struct rmg_hier rmg_hier;

typedef enum {
  RMG_OK = 0,
  RMG_ERR_ARG = 1,           /* invalid argument (null pointer, bad size, bad option)      */
  RMG_ERR_LAYOUT = 2,        /* region map does not conform (bad gids, sizes not 3k+1 ...) */
  RMG_ERR_CUDA = 3,          /* a CUDA runtime call failed                                 */
  RMG_ERR_NOMEM = 4,         /* device allocation failed                                   */
  RMG_ERR_SINGULAR = 5,      /* coarsest operator not positive definite                    */
  RMG_ERR_NOT_CONVERGED = 6, /* solver reached maxit above the tolerance                   */
  RMG_ERR_TIMEOUT = 7,       /* a device-side wait ran out (no kernel here waits today)    */
  RMG_ERR_STATE = 8          /* call out of order (e.g. setup before an operator is set)   */
} rmg_status;

/* Smoothers (Sec. 3.4): damped Jacobi, Chebyshev (Algorithm 2), and the region Gauss-Seidel of
 * Algorithm 1 in multicolour order: every sweep recomputes the regional residual (with the
 * interface sum) and then visits the colour classes of every region (2 colours for 5/7-point
 * stencils, the parities of i, j, l for 9/27-point ones; ascending colours before the coarse
 * correction, descending after it), each node taking delta = omega r / d~ from its residual
 * corrected by the region's own already-updated neighbours. Copies of interface nodes are
 * updated by their own regions and need not agree (as the paper notes); rmg_pcg_solve uses
 * the flexible CG form with it. Scalar operators only (RMG_ERR_ARG for B > 1). */
typedef enum {
  RMG_SMOOTHER_JACOBI = 0,
  RMG_SMOOTHER_CHEBYSHEV = 1,
  RMG_SMOOTHER_GS = 2
} rmg_smoother;

/* Arithmetic of the V-cycle. The outer CG always runs in FP64. */
typedef enum {
  RMG_PREC_FP64 = 0,            /* plain method, FP64 throughout                              */
  RMG_PREC_FP32 = 1,            /* V-cycle vectors and coefficients in FP32                   */
  RMG_PREC_FP32_BF16COEF = 2    /* FP32 vectors, stencil coefficients stored as BF16          */
} rmg_precision;

typedef struct {
  int levels;            /* hierarchy levels including the finest (>= 1)                   */
  int smoother;          /* rmg_smoother                                                   */
  int nu1, nu2;          /* pre/post: Jacobi sweeps, or Chebyshev polynomial applications */
  double omega;          /* Jacobi damping (Sec. 3.4)                                      */
  int cheb_degree;       /* Chebyshev: updates of u per application (Algorithm 2)          */
  double eig_ratio;      /* Chebyshev interval [lambda/eig_ratio, boost*lambda] (Sec. 3.4) */
  double boost;
  int power_iters;       /* power-method steps for lambda_max(D^-1 A), in [1, 100]        */
  int power_seed_base;   /* start vector of level l: SplitMix64 stream seed_base + l        */
  int precision;         /* rmg_precision                                                  */
  int use_graph;         /* capture the V-cycle in a CUDA graph (1) or launch eagerly (0)  */
  int tile_shape;        /* stencil-sweep tiles: -1 autotune (default), else a shape index  */
  int symmetric_storage; /* FP32 cycle, scalar operator: half planes of level 0 (1, default),
                            or the full planes only (0); see rmg_hier_coef_planes           */
} rmg_options;

/* Tile shapes of the stencil sweeps (rmg_options.tile_shape, rmg_hier_tile_shape). Every
 * launch covers all regions of a level with blocks of 256 threads, each block one tile of one
 * region. Shape 0: runs of 256 consecutive regional nodes. Shapes 1..8: boxes tx x ty x tz of
 * (32,8,1), (64,4,1), (128,2,1), (16,16,1), (32,4,2), (16,8,2), (16,4,4), (8,8,4); in 2D only
 * the tz = 1 boxes apply. Shape 9: 32 x 8 tiles of a region's x-y planes, each block stepping
 * through all z-planes with the tile (and a one-node ring) of u and of the coefficient planes
 * copied into shared memory ahead of use; it applies to the half-plane sweeps of a 3D 27-point
 * level 0 in the FP32 cycle (rmg_hier_tile_shape reports 32 x 8 x 0). With -1 the first
 * numeric setup times every applicable shape on every smoothed level (the residual sweep in
 * the hierarchy's precision, CUDA events) and keeps the fastest; the choice does not change any
 * result (each node computes the same row). */
#define RMG_NUM_TILE_SHAPES 10

typedef struct {
  int iterations;        /* products with A (0 when the initial residual already passes)  */
  double relres;         /* final ||b - A x|| / ||b|| (recurrence residual, FP64)           */
  double true_relres;    /* recomputed from x at the end                                   */
  double seconds;        /* wall time of the solve (host clock, synchronised)              */
  int vcycles;           /* preconditioner applications                                    */
} rmg_solve_info;

/* Defaults: 4 levels, Jacobi, nu1 = nu2 = 2, omega 0.67, degree 3, eig_ratio 20, boost 1.1,
 * 10 power iterations, seed base 10, FP64, graph on, tile shapes autotuned, symmetric storage
 * on. */
void rmg_options_default(rmg_options* opts);

/* Create a context on CUDA device `device` that queues work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). */
rmg_status rmg_create(rmg_ctx** out, int device, void* cuda_stream);
void rmg_destroy(rmg_ctx* ctx);
/* Message of the most recent failure on this context ("" if none). Valid until next call. */
const char* rmg_last_error(rmg_ctx* ctx);
/* Change the stream used by later calls (the captured V-cycle graph replays on it too). */
rmg_status rmg_set_stream(rmg_ctx* ctx, void* cuda_stream);

/*
 * Region layout (Sec. 3.1 and Sec. 4: the application supplies, per region, the number of
 * grid points per dimension and, per regional node, the composite node it is co-located
 * with; the library builds Psi implicitly: multiplicities Psi Psi^T and the interface groups
 * used for Psi^T Psi).
 *   dim             2 or 3 (2D regions have nz = 1)
 *   nregions        number of regions m
 *   region_dims     host, int32[3*m]: nx, ny, nz of every region (nodes per axis)
 *   region_gids     device, int64[n_r], n_r = sum nx*ny*nz: composite id in [0, n_composite)
 *                   of every regional node, regions concatenated, nodes x fastest
 *   n_composite     number of composite nodes; every one must appear in some region
 *   dirichlet       device, uint8[n_composite] or NULL: 1 marks a masked (Dirichlet) node
 * Errors: RMG_ERR_ARG for bad sizes, RMG_ERR_LAYOUT when a gid is out of range, a composite
 * node is in no region, or a node is shared by more than 255 regional copies.
 * Synchronises the stream (it reads back the interface-group count).
 */
rmg_status rmg_layout_create(rmg_ctx* ctx, int dim, int nregions, const int32_t* region_dims,
                             const int64_t* region_gids, int64_t n_composite,
                             const uint8_t* dirichlet, rmg_layout** out);
void rmg_layout_destroy(rmg_layout* layout);

/* Sizes of a layout: regional nodes, composite nodes, shared composite nodes (interface
 * groups) and regional slots in those groups. Any pointer may be NULL. */
rmg_status rmg_layout_sizes(rmg_layout* layout, int64_t* n_regional, int64_t* n_composite,
                            int64_t* n_groups, int64_t* n_group_slots);

/*
 * Non-invasive operator construction (Sec. 4). The composite matrix, fully assembled, in
 * CSR form on the device (row = composite id, entries of a row in any order). Every region
 * k receives A_ij / q_ij for the off-diagonals it contains (q_ij = number of regions that
 * contain both i and j) and a diagonal chosen so the region matrix reproduces A applied to
 * the constant vector, divided by the multiplicity (row sum zero for interior rows).
 *   stencil         5 or 9 (dim 2), 7 or 27 (dim 3): the neighbourhood every region row
 *                   may use; an entry outside it fails with RMG_ERR_LAYOUT
 *   rowptr, col     device int64 [n_composite + 1], [nnz]; val device double [nnz]
 * Replaces any operator set before. Synchronises the stream (error flag read-back).
 */
rmg_status rmg_operator_from_csr(rmg_layout* layout, int stencil, const int64_t* rowptr,
                                 const int64_t* col, const double* val);

/* Block operators with dofs_per_node = 3 (3D linear elasticity: 3x3 blocks per stencil
 * offset, 81 coefficients per dof row with a 27-point stencil). The composite CSR numbers
 * dofs node-major (row/column g * 3 + c). Every 3x3 block (c, c') is split by the rule of
 * rmg_operator_from_csr applied to the scalar matrix A[c::3, c'::3]; for the translations
 * (the rigid-body nullspace used by the paper's draft appendix rule) this keeps
 * sum_k A^(k) = A block by block. Transfers are the scalar 3:1 interpolation on every
 * component, so the coarse operators are again 3x3-block 27-point (9-point in 2D) stencils.
 * Regional vectors of such a layout are component-major: entry c * n_r + n; composite
 * vectors are node-major (g * 3 + c). The stencil must be 27 (3D) or 9 (2D). */
rmg_status rmg_operator_from_block_csr(rmg_layout* layout, int stencil, int dofs_per_node,
                                       const int64_t* rowptr, const int64_t* col,
                                       const double* val);

/* The same split as rmg_operator_from_csr (dofs_per_node = 1) or rmg_operator_from_block_csr
 * (dofs_per_node = 3), from a composite CSR in HOST memory, the form in which an application
 * usually holds its assembled matrix (Sec. 4: the application supplies the composite operator
 * and the region map, and the library dis-assembles it). rowptr is host int64[n_rows + 1] with
 * n_rows = n_composite * dofs_per_node and rowptr[0] = 0; col (host int64) and val (host
 * double) have rowptr[n_rows] entries. The arrays are copied to device buffers that the layout
 * owns (allocated on the first call, reallocated only when nnz changes, freed with the layout),
 * on the context's stream: page-locked host arrays that the driver maps into the device's
 * address space (cudaPointerGetAttributes reports a device pointer) and that are 8-byte
 * aligned are read by a copy kernel over the host link; any other host memory is copied with
 * cudaMemcpyAsync. The host arrays may be reused once the call returns. Errors: RMG_ERR_ARG for
 * null pointers, dofs_per_node other than 1 or 3, or a rowptr that does not start at 0; otherwise
 * those of the device-CSR calls. Synchronises the stream. */
rmg_status rmg_operator_from_host_csr(rmg_layout* layout, int stencil, int dofs_per_node,
                                      const int64_t* rowptr, const int64_t* col,
                                      const double* val);

/* Set already-split region matrices directly: coeffs is device double[stencil * n_r],
 * slot-major (coefficient s of regional node n at s * n_r + n). Slot order: 7-point
 * (-z,-y,-x,0,+x,+y,+z); 5-point (-y,-x,0,+x,+y); 9/27-point: (dx+1) + 3(dy+1) [+ 9(dz+1)]. */
rmg_status rmg_operator_from_region_stencils(rmg_layout* layout, int stencil,
                                             const double* coeffs);

/* Regional operator apply, the eq. "regional residual" with b = 0:
 * y = Psi^T Psi [[A]] u. u and y are device regional vectors (u consistent); y is
 * consistent on return. */
rmg_status rmg_regional_apply(rmg_layout* layout, const double* u, double* y);

/* Psi^T: regional r from composite c (device vectors). */
rmg_status rmg_comp_to_reg(rmg_layout* layout, const double* c, double* r);
/* Psi (average = 0: sum of copies) or (Psi Psi^T)^-1 Psi (average = 1: mean of copies). */
rmg_status rmg_reg_to_comp(rmg_layout* layout, const double* r, double* c, int average);

/*
 * Hierarchy setup (the regional mgSetup figure of Sec. 3.6): per level the composite
 * diagonal D~ = Psi^T Psi diag([[A]]) (Sec. 3.2), 3:1 linear interpolation per region
 * (Sec. 3.2, coarse nodes at local multiples of 3), the regional Galerkin product
 * [[Abar]] = [[R]] [[A]] [[P]] (eq. RegionalGalerkinProduct), Chebyshev bounds from the
 * power method (Sec. 3.4), and on the coarsest level the composite operator
 * Abar = Psibar [[Abar]] Psibar^T and its dense Cholesky factor (Sec. 3.5). Every region
 * dimension must allow levels-1 coarsenings by 3 (n - 1 divisible by 3 each time) and
 * co-located nodes must agree on being coarse points, else RMG_ERR_LAYOUT. The layout must
 * outlive the hierarchy. Synchronises the stream.
 */
rmg_status rmg_setup(rmg_layout* layout, const rmg_options* opts, rmg_hier** out);
/* Recompute all numeric setup from the layout's current operator, reusing every buffer and
 * the captured graph (for a new operator on the same mesh). Synchronises the stream. */
rmg_status rmg_setup_numeric(rmg_hier* hier);
void rmg_hier_destroy(rmg_hier* hier);

/*
 * Interpolation with stored per-node weights (the general transfers of Table 4 "Generic": the
 * sparsity of 3:1 linear interpolation, coefficients of the caller's choice). wr is device
 * float[3 * n_r(level)], axis-major: wr[a * n_r + n] is the weight regional fine node n takes
 * from its right coarse neighbour along axis a (1 - wr from the left one); it is ignored along
 * axes where n sits on a coarse index. Co-located copies must carry identical weights and
 * interface nodes may only use interface coarse nodes (Lemma 2); weights computed from
 * composite data satisfy both. The entries of P are the FP32 products wz (wy wx) of the
 * per-axis weights (1 - w for the left neighbour, also in FP32), in every precision of the
 * cycle and in the Galerkin products. wr = NULL restores linear interpolation. Call
 * rmg_setup_numeric afterwards (it rebuilds the Galerkin products and, if the kind of
 * transfer changed, re-captures the V-cycle graph). Levels 0 .. levels-2.
 */
rmg_status rmg_hier_set_transfer_weights(rmg_hier* hier, int level, const float* wr);
/* Operator-dependent weights of a level (device float[3 * n_r], layout as above, computed in
 * FP64 and rounded): along each
 * axis the fine nodes between two coarse nodes are weighted by the series resistances
 * 1/(-A_ij) of the three composite couplings on that line (the 1D A-harmonic extension,
 * linear for constant coefficients; linear where a coupling is not negative). */
rmg_status rmg_hier_opdep_weights(rmg_hier* hier, int level, float* wr);
/* Piecewise-constant 3:1 transfer weights of a level (the "Const" transfers of Table 4 and of
 * the hybrid experiments, Sec. 6.4): every fine node takes weight 1 from its nearest coarse
 * node along each axis; layout as above. Pass to rmg_hier_set_transfer_weights. */
rmg_status rmg_hier_constant_weights(rmg_hier* hier, int level, float* wr);

/*
 * Learned prolongator (no counterpart in the paper, which keeps linear interpolation and
 * notes that matrix-dependent transfers must match at co-located nodes, Sec. 3.2).
 * A small MLP maps 27 features of a fine node's local composite operator (padded to 32) to
 * the three per-axis interpolation weights of rmg_hier_set_transfer_weights:
 *   32 -> 64 (ReLU) -> 64 (ReLU) -> 3 (sigmoid); forward on BF16 tensor cores with FP32
 *   accumulation, backward in FP32, Adam on FP32 master weights.
 * Parameters (float[rmg_mlp_num_params()], host): W1[64][32], b1[64], W2[64][64], b2[64],
 * W3[3][64], b3[3]. Features: float[n][32] row-major (device). Labels and loss mask:
 * float[n][3] (device); the loss is sum mask (out - label)^2 / (3 n).
 */
typedef struct rmg_mlp rmg_mlp;
int rmg_mlp_num_params(void);
rmg_status rmg_mlp_create(rmg_ctx* ctx, const float* init_params, rmg_mlp** out);
void rmg_mlp_destroy(rmg_mlp* mlp);
/* Copies the current FP32 parameters to host memory (synchronises). */
rmg_status rmg_mlp_get_params(rmg_mlp* mlp, float* params);
/* out (device float[n][3]) = network(feats). */
rmg_status rmg_mlp_forward(rmg_mlp* mlp, int n, const float* feats, float* out);
/* Loss and gradient over all n samples in order (host outputs; synchronises). */
rmg_status rmg_mlp_gradient(rmg_mlp* mlp, int n, const float* feats, const float* labels,
                            const float* mask, float* grad, float* loss);
/* steps Adam steps (learning rate lr) on batches of `batch` samples (a multiple of 128)
 * drawn with replacement by a counter-based hash of (seed, step, row); loss_history: host
 * float[steps] or NULL. Synchronises at the end. */
rmg_status rmg_mlp_train(rmg_mlp* mlp, int n, const float* feats, const float* labels,
                         const float* mask, int steps, int batch, float lr,
                         unsigned long long seed, float* loss_history);
/* Features of every regional node of a hierarchy level (device float[n_r][32]). */
rmg_status rmg_hier_mlp_features(rmg_hier* hier, int level, float* feats);
/* Network inference on a level: per-axis weights (device float[3 * n_r]) for
 * rmg_hier_set_transfer_weights (zero along axes where a node sits on a coarse index).
 * Uses scratch kept by the hierarchy (allocated on the first call). */
rmg_status rmg_hier_mlp_weights(rmg_hier* hier, int level, rmg_mlp* mlp, float* wr);

/* Measured convergence of the V-cycle as a stationary solver: from a SplitMix64 random
 * error e (stream `seed`, zero at masked nodes), iterate e <- e - M^-1 A e `iters` times and
 * return (||e_iters||_A / ||e_0||_A)^(1/iters). Used to label training operators and to
 * accept or reject learned interpolation. Synchronises once per cycle. Uses the PCG work
 * vectors of the hierarchy. */
rmg_status rmg_hier_convergence_factor(rmg_hier* hier, int iters, unsigned long long seed,
                                       double* factor);

/* Per-region error energies of the V-cycle as a stationary solver, for accepting learned
 * interpolation region by region (no counterpart in the paper). From a SplitMix64 random error
 * e (stream `seed`, zero at masked nodes) the cycle runs `iters` times, e <- e - M^-1 A e. For
 * every region k, e0[k] and eK[k] (host double[nregions]) receive E_k(e) = e_k^T A^(k) e_k
 * before and after: the region matrix of the split (Sec. 4) applied to the region's copy of e,
 * without the interface sum. By Lemma 1 the E_k add up to e^T A e, and for M-matrix operators
 * (non-positive couplings, row sums zero or positive) every A^(k) is positive semi-definite,
 * so (eK[k] / e0[k])^(1 / (2 iters)) is the region's share of the A-norm reduction. Scalar
 * operators only. Uses the PCG work vectors; synchronises. */
rmg_status rmg_hier_region_energies(rmg_hier* hier, int iters, unsigned long long seed,
                                    double* e0, double* eK);
/* Stored transfer weights (device float[3 * n_r(level)], the layout of
 * rmg_hier_set_transfer_weights) that take `learned` (same layout) at every node all of whose
 * regions accept (accept: host uint8[nregions(level)], nonzero = accept) and linear
 * interpolation (rem / 3, rounded to FP32) elsewhere, zero along axes where the node sits on a
 * coarse index. The copies of an interface node lie in the same regions, so they receive
 * identical weights, as Lemma 2 requires. Synchronises. */
rmg_status rmg_hier_blend_weights(rmg_hier* hier, int level, const uint8_t* accept,
                                  const float* learned, float* out);

/* A colouring of the regions (host int colours[nregions], *ncolours = number of colours) in
 * which regions that share a composite node get different colours (greedy, region order). A
 * transfer changed only in the regions of one colour, blended with rmg_hier_blend_weights,
 * leaves every interface node and every other region's rows unchanged, so its effect can be
 * measured region by region without neighbours interfering. Synchronises. */
rmg_status rmg_hier_region_colours(rmg_hier* hier, int* colours, int* ncolours);

/* One regional V-cycle with zero initial guess, z = M^-1 r: the regional mgCycle of the
 * figure in Sec. 3.6 with the operations of Sec. 3.3 (smoothing with the regional residual,
 * restriction w = Psibar^T Psibar [[R]] [[Psi Psi^T]]^-1 r, recursion, coarse solve of the
 * composite coarsest operator, Sec. 3.5, region-local prolongation, post-smoothing). r and z
 * are device vectors, composite (layout_flag = 0) or regional and consistent
 * (layout_flag = 1). A composite r is copied into every regional copy; the regional output is
 * returned as the mean over the copies (the composite value). Errors: RMG_ERR_STATE when the
 * coarsest level exceeds the dense solver (RMG_MAX_DENSE). Returns once queued. */
rmg_status rmg_vcycle_apply(rmg_hier* hier, const double* r, double* z, int layout_flag);

/*
 * Preconditioned conjugate gradients in FP64 with one V-cycle as preconditioner (Sec. 6.2
 * notes that the region multigrid is normally used as a Krylov preconditioner; the paper's
 * runs use it as a stand-alone solver). b and x are device composite vectors (x: in =
 * initial guess, out = solution). Entries at masked nodes of b are taken as zero. The plain
 * method (RMG_PREC_FP64) runs textbook PCG; the FP32 and BF16 cycles and the region
 * Gauss-Seidel cycle run inside flexible CG (beta = r.(z - z_old) / r_old.z_old). Every inner
 * product, update and the stopping test are FP64; the FP32 cycle receives the residual scaled
 * by a power of two near 1/||b|| (exact, and the cycle is linear), so the result does not
 * depend on the scale of b. When the recurrence residual passes ||r||_2 / ||b||_2 <= rtol the
 * true residual b - A x is recomputed in FP64; the solve stops only if that one passes too,
 * and otherwise restarts from the true residual. It returns RMG_ERR_NOT_CONVERGED (x still
 * written) after maxit iterations. history: host double[maxit + 1] or NULL, receives the
 * relative residual per iteration. Synchronises the stream once per iteration (the
 * convergence test).
 */
rmg_status rmg_pcg_solve(rmg_hier* hier, const double* b, double* x, double rtol, int maxit,
                         double* history, rmg_solve_info* info);

/*
 * Regional operator apply that allocates no device memory: y = Psi^T Psi [[A]] u, the same
 * result as rmg_regional_apply, for callers that cannot call cudaMalloc at that point
 * (applications whose own pool allocator owns all device memory, loops that cannot afford
 * the device-wide synchronisation an allocation or a free can cause). The
 * paper has no counterpart: it is a deployment variant of the interface summation.
 * No handle is needed; every argument is a plain array:
 *   dim, nregions, region_dims (host int32[3*m]), region_gids (device int64[n_r]),
 *   n_composite  as for rmg_layout_create (no Dirichlet mask: masked rows are already
 *                identity rows of the split operator)
 *   stencil, coeffs  already-split region stencils, device double[stencil * n_r], slot-major
 *                (the layout of rmg_operator_from_region_stencils / rmg_hier_level_export)
 *   u, y         device regional vectors (u consistent); y is consistent on return
 *   cuda_stream  stream for the work (NULL = legacy default stream)
 *   msg, msg_len optional caller buffer that receives the error text
 * Scratch: one file-scope device array of about 32 MiB held by every GPU that loads the
 * library until the process exits, with room for at most 4096 regions and 4,194,304
 * composite nodes; larger inputs fail with RMG_ERR_ARG before any work is queued. Each call
 * rewrites the region table and zeroes the accumulator it keeps there; calls that overlap
 * on the GPU (other streams or host threads) share the array and race. The work runs on the
 * device that cuda_stream belongs to (the current device for the legacy default stream): the
 * call makes that device current for its duration and restores the caller's device before
 * it returns. The first call for a device takes the device address of that device's copy of
 * the array (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture. The summation order over the
 * copies of an interface node is not fixed (atomic adds), so results can differ from
 * rmg_regional_apply in the last bits. Regional nodes whose gid is outside
 * [0, n_composite) receive NaN. Returns once the work is queued.
 */
rmg_status rmg_regional_apply_static(int dim, int nregions, const int32_t* region_dims,
                                     int stencil, const double* coeffs,
                                     const int64_t* region_gids, int64_t n_composite,
                                     const double* u, double* y, void* cuda_stream, char* msg,
                                     int msg_len);

/* ---- introspection (tests and benchmarks) ------------------------------------------- */
/* Levels, and per level: regions, regional nodes, composite id space, stencil points. */
rmg_status rmg_hier_level_sizes(rmg_hier* hier, int level, int64_t* n_regional,
                                int64_t* n_composite, int* stencil);
/* Dofs per node of the hierarchy's operator (1, or 3 for block operators). */
rmg_status rmg_hier_dofs_per_node(rmg_hier* hier, int* dofs);
/* Copy level data to caller device buffers (any may be NULL):
 *   coeffs  double[B * B * stencil * n_r] region stencils (slot-major, see above; block
 *           (c, c') of a B-dof operator at offset (c * B + c') * stencil * n_r), FP64 copy
 *   dinv    double[B * n_r] inverse composite diagonal in regional layout (component-major)
 *   gids    int64[n_r] composite id of every regional node on that level */
rmg_status rmg_hier_level_export(rmg_hier* hier, int level, double* coeffs, double* dinv,
                                 int64_t* gids);
/* Chebyshev lambda~ estimate of a level (host). */
rmg_status rmg_hier_lambda(rmg_hier* hier, int level, double* lam);
/* Recompute the Galerkin product [[Abar]] = [[R]] [[A]] [[P]] of level -> level + 1 alone
 * (eq. RegionalGalerkinProduct; the level's current transfer: linear, or the stored weights of
 * rmg_hier_set_transfer_weights), exactly as rmg_setup_numeric computes it, on the context's
 * stream. For timing the triple product (Table 4) or refreshing one coarse operator; the
 * diagonals, lambda and the coarse factor are not refreshed. RMG_ERR_ARG for a level outside
 * 0 .. levels-2.
 *
 * A hierarchy whose coarsest level has more than 16384 unknowns (RMG_MAX_DENSE) is built
 * without the dense coarse solver: setup, this call and the introspection calls work, while
 * cycles and solves fail with RMG_ERR_STATE. */
#define RMG_MAX_DENSE 16384
rmg_status rmg_hier_galerkin(rmg_hier* hier, int level);

/* Tile shape the stencil sweeps of a level use (see RMG_NUM_TILE_SHAPES): the box extents, or
 * 0, 0, 0 for runs of 256 nodes (also for the coarsest level, which is not smoothed). Host
 * ints; fails with RMG_ERR_ARG for a level outside the hierarchy. */
rmg_status rmg_hier_tile_shape(rmg_hier* hier, int level, int* tx, int* ty, int* tz);
/* Stencil coefficients per regional node that the cycle's sweeps read on a level, as of the
 * last rmg_setup_numeric: B * B * S for an S-point stencil, or (S + 1) / 2 where the half form
 * is in use. The half form (FP32 cycle, scalar operator, level 0, symmetric_storage 1) rests
 * on the symmetry of the regional operator, a(n, n+e) = a(n+e, n) inside every region (Sec. 4
 * splits a symmetric composite matrix into symmetric region matrices): it keeps the centre and
 * the (S - 1) / 2 slots after it, and reads a coefficient of the other half at the neighbour
 * that owns its mirror. Each setup compares every mirrored pair of the FP32 coefficients bit
 * for bit; the half form is used only when all agree, so that the sweeps compute exactly the
 * rows of the full form and no result changes. Host int; RMG_ERR_ARG for a level outside the
 * hierarchy, RMG_ERR_STATE before the first numeric setup. */
rmg_status rmg_hier_coef_planes(rmg_hier* hier, int level, int* planes);
/* Coarsest composite matrix restricted to unmasked nodes (dense, row-major, host double
 * [(B*nc)^2], dof cu * B + c) and the composite ids of those nodes (host int64[nc]). Pass NULL
 * to query nc (the number of unmasked composite nodes). */
rmg_status rmg_hier_coarse_matrix(rmg_hier* hier, int64_t* nc, double* dense, int64_t* ids);
/* Kernels launched by this library in this process so far (a graph replay counts the
 * kernels of the graph). Kernels recorded into a graph during capture are not counted. */
unsigned long long rmg_launch_count(void);
/* Live timing of the dominant kernel: every V-cycle records CUDA events around one
 * level-0 smoother stencil launch (the first post-smoothing Chebyshev recurrence step, or the
 * first post-smoothing Jacobi sweep). rmg_pcg_solve reads them after each of its
 * per-iteration synchronisations. Returns the accumulated milliseconds and the number of
 * timed launches since the last reset (reset = 1 clears the totals after reading). */
rmg_status rmg_hier_probe(rmg_hier* hier, int reset, double* total_ms, long long* count);
/* Kernel launches queued by one V-cycle (0 when eager mode has not run yet). */
rmg_status rmg_hier_vcycle_launches(rmg_hier* hier, int* launches);

#ifdef __cplusplus
}
#endif
#endif /* RMG_H */
