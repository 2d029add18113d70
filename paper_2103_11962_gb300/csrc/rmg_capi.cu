// extern "C" entry points: argument checks, exception -> status translation.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>

#include "rmg_hier.cuh"
#include "rmg_layout.cuh"

using namespace rmg;

namespace {

rmg_status fail(rmg_ctx* ctx, rmg_status st, const char* msg) {
  if (ctx) ctx->c.last_error = msg;
  return st;
}

template <class F>
rmg_status guarded(rmg_ctx* ctx, F&& f) {
  if (!ctx) return RMG_ERR_ARG;
  try {
    RMG_CUDA(cudaSetDevice(ctx->c.device));
    f();
    ctx->c.last_error.clear();
    return RMG_OK;
  } catch (const Error& e) {
    return fail(ctx, e.status, e.what());
  } catch (const std::bad_alloc&) {
    return fail(ctx, RMG_ERR_NOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(ctx, RMG_ERR_CUDA, e.what());
  }
}

// Copy of `bytes` bytes (a multiple of 8, both ends 8-byte aligned) from page-locked host memory
// that the device can address (src: its device pointer) into device memory, read by the SMs
// over the host link: 16-byte loads when both ends allow them, else 8-byte ones.
__global__ void k_copy_from_host(const void* __restrict__ src, void* __restrict__ dst,
                                 size_t bytes) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((((uintptr_t)src | (uintptr_t)dst) & 15) == 0) {
    const int4* s = static_cast<const int4*>(src);
    int4* d = static_cast<int4*>(dst);
    const size_t n16 = bytes / 16;
    for (size_t k = t0; k < n16; k += stride) d[k] = s[k];
    if (t0 == 0 && (bytes & 15))
      reinterpret_cast<int64_t*>(dst)[bytes / 8 - 1] =
          reinterpret_cast<const int64_t*>(src)[bytes / 8 - 1];
  } else {
    const int64_t* s = static_cast<const int64_t*>(src);
    int64_t* d = static_cast<int64_t*>(dst);
    for (size_t k = t0; k < bytes / 8; k += stride) d[k] = s[k];
  }
}

// Host-to-device copy of an array of 8-byte elements on stream st. Page-locked host memory
// that the driver reports as mapped into the device's address space (cudaPointerGetAttributes:
// a host allocation with a device pointer) is read by a kernel, which draws more of the host
// link's bandwidth than a copy-engine transfer; any other host memory goes by cudaMemcpyAsync.
void copy_host_array(void* dst, const void* src, size_t bytes, cudaStream_t st, int nsm) {
  if (!bytes) return;
  cudaPointerAttributes a{};
  const bool mapped = cudaPointerGetAttributes(&a, src) == cudaSuccess &&
                      a.type == cudaMemoryTypeHost && a.devicePointer != nullptr;
  if (!mapped || (((uintptr_t)src | (uintptr_t)dst) & 7)) {
    cudaGetLastError();                          // unregistered memory: not an error
    RMG_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    return;
  }
  const size_t blocks = std::min<size_t>((bytes / 16 + 255) / 256, (size_t)nsm * 8);
  k_copy_from_host<<<(unsigned)std::max<size_t>(blocks, 1), 256, 0, st>>>(a.devicePointer, dst,
                                                                          bytes);
  RMG_LAUNCHED();
}

}  // namespace

extern "C" {

void rmg_options_default(rmg_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->levels = 4;
  o->smoother = RMG_SMOOTHER_JACOBI;
  o->nu1 = 2;
  o->nu2 = 2;
  o->omega = 0.67;
  o->cheb_degree = 3;
  o->eig_ratio = 20.0;
  o->boost = 1.1;
  o->power_iters = 10;
  o->power_seed_base = 10;
  o->precision = RMG_PREC_FP64;
  o->use_graph = 1;
  o->tile_shape = -1;
  o->symmetric_storage = 1;
}

rmg_status rmg_create(rmg_ctx** out, int device, void* stream) {
  if (!out) return RMG_ERR_ARG;
  *out = nullptr;
  rmg_ctx* ctx = new (std::nothrow) rmg_ctx();
  if (!ctx) return RMG_ERR_NOMEM;
  ctx->c.device = device;
  ctx->c.stream = (cudaStream_t)stream;
  rmg_status st = guarded(ctx, [&] {
    int ndev = 0;
    RMG_CUDA(cudaGetDeviceCount(&ndev));
    RMG_REQUIRE(device >= 0 && device < ndev, RMG_ERR_ARG, "no such CUDA device");
    RMG_CUDA(cudaDeviceGetAttribute(&ctx->c.nsm, cudaDevAttrMultiProcessorCount, device));
    ctx->c.d_err.alloc(1);
    RMG_CUDA(cudaMemset(ctx->c.d_err.get(), 0, sizeof(int)));
    ctx->c.max_partials = ctx->c.nsm * 8;
    ctx->c.partials.alloc(2 * ctx->c.max_partials);   // room for two fused reductions
  });
  if (st != RMG_OK) {
    delete ctx;
    return st;
  }
  *out = ctx;
  return RMG_OK;
}

void rmg_destroy(rmg_ctx* ctx) { delete ctx; }

const char* rmg_last_error(rmg_ctx* ctx) { return ctx ? ctx->c.last_error.c_str() : "null context"; }

rmg_status rmg_set_stream(rmg_ctx* ctx, void* stream) {
  if (!ctx) return RMG_ERR_ARG;
  ctx->c.stream = (cudaStream_t)stream;
  return RMG_OK;
}

rmg_status rmg_layout_create(rmg_ctx* ctx, int dim, int nregions, const int32_t* region_dims,
                             const int64_t* region_gids, int64_t n_composite,
                             const uint8_t* dirichlet, rmg_layout** out) {
  if (!out) return fail(ctx, RMG_ERR_ARG, "out is NULL");
  *out = nullptr;
  rmg_layout* lay = new (std::nothrow) rmg_layout();
  if (!lay) return RMG_ERR_NOMEM;
  lay->ctx = ctx;
  rmg_status st = guarded(ctx, [&] {
    layout_create(ctx->c, lay->L0, dim, nregions, region_dims, region_gids, n_composite, dirichlet);
    lay->ybuf.alloc(lay->L0.n_r);
  });
  if (st != RMG_OK) {
    delete lay;
    return st;
  }
  *out = lay;
  return RMG_OK;
}

void rmg_layout_destroy(rmg_layout* lay) { delete lay; }

rmg_status rmg_layout_sizes(rmg_layout* lay, int64_t* n_regional, int64_t* n_composite,
                            int64_t* n_groups, int64_t* n_group_slots) {
  if (!lay) return RMG_ERR_ARG;
  if (n_regional) *n_regional = lay->L0.n_r;
  if (n_composite) *n_composite = lay->L0.ncomp;
  if (n_groups) *n_groups = lay->L0.ngroups;
  if (n_group_slots) *n_group_slots = lay->L0.nslots;
  return RMG_OK;
}

rmg_status rmg_operator_from_csr(rmg_layout* lay, int stencil, const int64_t* rowptr,
                                 const int64_t* col, const double* val) {
  if (!lay) return RMG_ERR_ARG;
  return guarded(lay->ctx, [&] {
    split_from_csr(lay->ctx->c, lay->L0, stencil, 1, rowptr, col, val);
    lay->has_operator = true;
  });
}

rmg_status rmg_operator_from_block_csr(rmg_layout* lay, int stencil, int dofs_per_node,
                                       const int64_t* rowptr, const int64_t* col,
                                       const double* val) {
  if (!lay) return RMG_ERR_ARG;
  return guarded(lay->ctx, [&] {
    split_from_csr(lay->ctx->c, lay->L0, stencil, dofs_per_node, rowptr, col, val);
    lay->ybuf.ensure((size_t)dofs_per_node * lay->L0.n_r);
    lay->has_operator = true;
  });
}

rmg_status rmg_operator_from_host_csr(rmg_layout* lay, int stencil, int dofs_per_node,
                                      const int64_t* rowptr, const int64_t* col,
                                      const double* val) {
  if (!lay) return RMG_ERR_ARG;
  return guarded(lay->ctx, [&] {
    RMG_REQUIRE(rowptr && col && val, RMG_ERR_ARG, "null CSR array");
    RMG_REQUIRE(dofs_per_node == 1 || dofs_per_node == 3, RMG_ERR_ARG,
                "dofs_per_node must be 1 or 3");
    const size_t nrows = (size_t)lay->L0.ncomp * (size_t)dofs_per_node;
    RMG_REQUIRE(rowptr[0] == 0 && rowptr[nrows] >= 0, RMG_ERR_ARG,
                "rowptr must start at 0 and end at nnz >= 0");
    const size_t nnz = (size_t)rowptr[nrows];
    cudaStream_t st = lay->ctx->c.stream;
    lay->csr_rowptr.ensure(nrows + 1);
    lay->csr_col.ensure(std::max<size_t>(nnz, 1));
    lay->csr_val.ensure(std::max<size_t>(nnz, 1));
    const int nsm = lay->ctx->c.nsm;
    copy_host_array(lay->csr_rowptr.get(), rowptr, (nrows + 1) * sizeof(int64_t), st, nsm);
    copy_host_array(lay->csr_col.get(), col, nnz * sizeof(int64_t), st, nsm);
    copy_host_array(lay->csr_val.get(), val, nnz * sizeof(double), st, nsm);
    split_from_csr(lay->ctx->c, lay->L0, stencil, dofs_per_node, lay->csr_rowptr.get(),
                   lay->csr_col.get(), lay->csr_val.get());
    lay->ybuf.ensure((size_t)dofs_per_node * lay->L0.n_r);
    lay->has_operator = true;
  });
}

rmg_status rmg_operator_from_region_stencils(rmg_layout* lay, int stencil, const double* coeffs) {
  if (!lay) return RMG_ERR_ARG;
  return guarded(lay->ctx, [&] {
    Level& L = lay->L0;
    RMG_REQUIRE(coeffs, RMG_ERR_ARG, "coeffs is NULL");
    RMG_REQUIRE((L.dim == 2 && (stencil == 5 || stencil == 9)) ||
                    (L.dim == 3 && (stencil == 7 || stencil == 27)),
                RMG_ERR_ARG, "stencil must be 5/9 in 2D and 7/27 in 3D");
    L.kind = stencil;
    L.coef.ensure((size_t)stencil * L.n_r);
    RMG_CUDA(cudaMemcpyAsync(L.coef.get(), coeffs, L.coef.bytes(), cudaMemcpyDeviceToDevice,
                             lay->ctx->c.stream));
    lay->has_operator = true;
  });
}

rmg_status rmg_regional_apply(rmg_layout* lay, const double* u, double* y) {
  if (!lay) return RMG_ERR_ARG;
  return guarded(lay->ctx, [&] {
    RMG_REQUIRE(lay->has_operator, RMG_ERR_STATE, "no operator set on the layout");
    RMG_REQUIRE(u && y, RMG_ERR_ARG, "null vector");
    regional_apply(lay->ctx->c, lay->L0, u, y, lay->ybuf.get());
  });
}

rmg_status rmg_comp_to_reg(rmg_layout* lay, const double* c, double* r) {
  if (!lay) return RMG_ERR_ARG;
  return guarded(lay->ctx, [&] {
    RMG_REQUIRE(c && r, RMG_ERR_ARG, "null vector");
    comp_to_reg(lay->ctx->c, lay->L0, c, r, false);
  });
}

rmg_status rmg_reg_to_comp(rmg_layout* lay, const double* r, double* c, int average) {
  if (!lay) return RMG_ERR_ARG;
  return guarded(lay->ctx, [&] {
    RMG_REQUIRE(c && r, RMG_ERR_ARG, "null vector");
    reg_to_comp(lay->ctx->c, lay->L0, r, c, average ? 1 : 0);
  });
}

rmg_status rmg_setup(rmg_layout* lay, const rmg_options* opts, rmg_hier** out) {
  if (!lay || !out) return RMG_ERR_ARG;
  *out = nullptr;
  rmg_hier* hh = new (std::nothrow) rmg_hier();
  if (!hh) return RMG_ERR_NOMEM;
  rmg_status st = guarded(lay->ctx, [&] {
    Hier& h = hh->h;
    h.layout = lay;
    h.c = &lay->ctx->c;
    if (opts) h.o = *opts; else rmg_options_default(&h.o);
    hier_build(h);
    hier_numeric(h);
  });
  if (st != RMG_OK) {
    delete hh;
    return st;
  }
  *out = hh;
  return RMG_OK;
}

rmg_status rmg_setup_numeric(rmg_hier* hh) {
  if (!hh) return RMG_ERR_ARG;
  return guarded(hh->h.layout->ctx, [&] { hier_numeric(hh->h); });
}

void rmg_hier_destroy(rmg_hier* hh) { delete hh; }

rmg_status rmg_vcycle_apply(rmg_hier* hh, const double* r, double* z, int layout_flag) {
  if (!hh) return RMG_ERR_ARG;
  return guarded(hh->h.layout->ctx, [&] {
    RMG_REQUIRE(r && z, RMG_ERR_ARG, "null vector");
    vcycle_apply(hh->h, r, z, layout_flag);
  });
}

rmg_status rmg_pcg_solve(rmg_hier* hh, const double* b, double* x, double rtol, int maxit,
                         double* history, rmg_solve_info* info) {
  if (!hh) return RMG_ERR_ARG;
  return guarded(hh->h.layout->ctx, [&] {
    RMG_REQUIRE(b && x, RMG_ERR_ARG, "null vector");
    RMG_REQUIRE(maxit >= 0 && rtol >= 0, RMG_ERR_ARG, "bad rtol/maxit");
    pcg_solve(hh->h, b, x, rtol, maxit, history, info);
  });
}

rmg_status rmg_hier_level_sizes(rmg_hier* hh, int level, int64_t* n_regional, int64_t* n_composite,
                                int* stencil) {
  if (!hh) return RMG_ERR_ARG;
  Hier& h = hh->h;
  if (level < 0 || level >= h.levels()) return fail(h.layout->ctx, RMG_ERR_ARG, "bad level");
  if (n_regional) *n_regional = h.lv[level]->n_r;
  if (n_composite) *n_composite = h.lv[level]->ncomp;
  if (stencil) *stencil = h.lv[level]->kind;
  return RMG_OK;
}

rmg_status rmg_hier_dofs_per_node(rmg_hier* hh, int* dofs) {
  if (!hh || !dofs) return RMG_ERR_ARG;
  *dofs = hh->h.lv[0]->B;
  return RMG_OK;
}

namespace {
__global__ void k_int_to_i64(int n, const int* a, int64_t* b) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) b[k] = a[k];
}
}  // namespace

rmg_status rmg_hier_level_export(rmg_hier* hh, int level, double* coeffs, double* dinv,
                                 int64_t* gids) {
  if (!hh) return RMG_ERR_ARG;
  return guarded(hh->h.layout->ctx, [&] {
    Hier& h = hh->h;
    RMG_REQUIRE(level >= 0 && level < h.levels(), RMG_ERR_ARG, "bad level");
    Level& L = *h.lv[level];
    cudaStream_t st = h.c->stream;
    // coefficients: B*B*stencil*n_r (block (c,c') at offset (c*B+c')*stencil*n_r); dinv: B*n_r
    if (coeffs)
      RMG_CUDA(cudaMemcpyAsync(coeffs, L.coef.get(), L.coef.bytes(), cudaMemcpyDeviceToDevice, st));
    if (dinv)
      RMG_CUDA(cudaMemcpyAsync(dinv, L.dinv.get(), L.dinv.bytes(), cudaMemcpyDeviceToDevice, st));
    if (gids) {
      k_int_to_i64<<<persistent_grid(*h.c, (L.n_r + 255) / 256), 256, 0, st>>>(L.n_r, L.gid.get(), gids);
      RMG_LAUNCHED();
    }
  });
}

rmg_status rmg_hier_set_transfer_weights(rmg_hier* hh, int level, const float* wr) {
  if (!hh) return RMG_ERR_ARG;
  return guarded(hh->h.layout->ctx, [&] { set_transfer_weights(hh->h, level, wr); });
}

rmg_status rmg_hier_opdep_weights(rmg_hier* hh, int level, float* wr) {
  if (!hh) return RMG_ERR_ARG;
  return guarded(hh->h.layout->ctx, [&] {
    RMG_REQUIRE(wr, RMG_ERR_ARG, "wr is NULL");
    opdep_weights(hh->h, level, wr);
  });
}

rmg_status rmg_hier_convergence_factor(rmg_hier* hh, int iters, unsigned long long seed,
                                       double* factor) {
  if (!hh || !factor) return RMG_ERR_ARG;
  return guarded(hh->h.layout->ctx, [&] {
    RMG_REQUIRE(iters > 0, RMG_ERR_ARG, "iters must be positive");
    *factor = convergence_factor(hh->h, iters, seed);
  });
}

rmg_status rmg_hier_region_energies(rmg_hier* hh, int iters, unsigned long long seed,
                                    double* e0, double* eK) {
  if (!hh) return RMG_ERR_ARG;
  return guarded(hh->h.layout->ctx, [&] {
    RMG_REQUIRE(iters > 0 && e0 && eK, RMG_ERR_ARG, "bad arguments");
    region_energies(hh->h, iters, seed, e0, eK);
  });
}

rmg_status rmg_hier_blend_weights(rmg_hier* hh, int level, const uint8_t* accept,
                                  const float* learned, float* out) {
  if (!hh) return RMG_ERR_ARG;
  return guarded(hh->h.layout->ctx, [&] {
    RMG_REQUIRE(accept && learned && out, RMG_ERR_ARG, "bad arguments");
    blend_weights(hh->h, level, accept, learned, out);
  });
}

rmg_status rmg_hier_region_colours(rmg_hier* hh, int* colours, int* ncolours) {
  if (!hh) return RMG_ERR_ARG;
  return guarded(hh->h.layout->ctx, [&] {
    RMG_REQUIRE(colours && ncolours, RMG_ERR_ARG, "bad arguments");
    *ncolours = region_colours(hh->h, colours);
  });
}

rmg_status rmg_hier_galerkin(rmg_hier* hh, int level) {
  if (!hh) return RMG_ERR_ARG;
  return guarded(hh->h.layout->ctx, [&] { galerkin_level(hh->h, level); });
}

rmg_status rmg_hier_constant_weights(rmg_hier* hh, int level, float* wr) {
  if (!hh) return RMG_ERR_ARG;
  return guarded(hh->h.layout->ctx, [&] {
    RMG_REQUIRE(wr, RMG_ERR_ARG, "wr is NULL");
    constant_weights(hh->h, level, wr);
  });
}

rmg_status rmg_hier_lambda(rmg_hier* hh, int level, double* lam) {
  if (!hh || !lam) return RMG_ERR_ARG;
  Hier& h = hh->h;
  if (level < 0 || level >= h.levels() || level >= 16) return fail(h.layout->ctx, RMG_ERR_ARG, "bad level");
  *lam = h.hsc.lam[level];
  return RMG_OK;
}

rmg_status rmg_hier_tile_shape(rmg_hier* hh, int level, int* tx, int* ty, int* tz) {
  if (!hh || !tx || !ty || !tz) return RMG_ERR_ARG;
  Hier& h = hh->h;
  if (level < 0 || level >= h.levels()) return fail(h.layout->ctx, RMG_ERR_ARG, "bad level");
  if (h.shape[level] < 0) { *tx = *ty = *tz = 0; return RMG_OK; }
  tile_shape(h, level, tx, ty, tz);
  return RMG_OK;
}

rmg_status rmg_hier_coef_planes(rmg_hier* hh, int level, int* planes) {
  if (!hh || !planes) return RMG_ERR_ARG;
  Hier& h = hh->h;
  if (level < 0 || level >= h.levels()) return fail(h.layout->ctx, RMG_ERR_ARG, "bad level");
  if (h.kind0 == 0) return fail(h.layout->ctx, RMG_ERR_STATE, "no numeric setup yet");
  const Level& L = *h.lv[level];
  *planes = (h.half(level) && h.hsc.half_asym == 0) ? (L.kind + 1) / 2 : L.B * L.B * L.kind;
  return RMG_OK;
}

rmg_status rmg_hier_coarse_matrix(rmg_hier* hh, int64_t* nc, double* dense, int64_t* ids) {
  if (!hh || !nc) return RMG_ERR_ARG;
  return guarded(hh->h.layout->ctx, [&] {
    Hier& h = hh->h;
    *nc = h.nc;
    const size_t nd = (size_t)h.nc * h.lv[h.levels() - 1]->B;
    if (dense && h.nc)
      RMG_CUDA(cudaMemcpy(dense, h.X.get(), nd * nd * sizeof(double), cudaMemcpyDeviceToHost));
    if (ids && h.nc)
      RMG_CUDA(cudaMemcpy(ids, h.cu2gid.get(), (size_t)h.nc * sizeof(long long),
                          cudaMemcpyDeviceToHost));
  });
}

unsigned long long rmg_launch_count(void) { return g_launches; }

rmg_status rmg_hier_probe(rmg_hier* hh, int reset, double* total_ms, long long* count) {
  if (!hh) return RMG_ERR_ARG;
  Hier& h = hh->h;
  if (total_ms) *total_ms = h.probe_ms;
  if (count) *count = h.probe_count;
  if (reset) {
    h.probe_ms = 0.0;
    h.probe_count = 0;
  }
  return RMG_OK;
}

rmg_status rmg_hier_vcycle_launches(rmg_hier* hh, int* launches) {
  if (!hh || !launches) return RMG_ERR_ARG;
  *launches = hh->h.launches;
  return RMG_OK;
}

}  // extern "C"
