"""Thin Python binding of the C ABI in include/rmg.h (ctypes; argument marshalling only).

Every computation runs in the CUDA library librmg.so. Device arrays are torch tensors whose
data pointers are handed to the library; the library queues its kernels on the torch stream
current when the context is created (or set later with ``Context.set_stream``).

There is no CPU fallback: if librmg.so is missing or cannot be loaded, importing the
library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librmg.so")

RMG_OK = 0
STATUS = {0: "RMG_OK", 1: "RMG_ERR_ARG", 2: "RMG_ERR_LAYOUT", 3: "RMG_ERR_CUDA",
          4: "RMG_ERR_NOMEM", 5: "RMG_ERR_SINGULAR", 6: "RMG_ERR_NOT_CONVERGED",
          7: "RMG_ERR_TIMEOUT", 8: "RMG_ERR_STATE"}
JACOBI, CHEBYSHEV, GAUSS_SEIDEL = 0, 1, 2
FP64, FP32, FP32_BF16COEF = 0, 1, 2


class RmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("smoother", ctypes.c_int), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("omega", ctypes.c_double), ("cheb_degree", ctypes.c_int),
                ("eig_ratio", ctypes.c_double), ("boost", ctypes.c_double),
                ("power_iters", ctypes.c_int), ("power_seed_base", ctypes.c_int),
                ("precision", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("tile_shape", ctypes.c_int), ("symmetric_storage", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("relres", ctypes.c_double),
                ("true_relres", ctypes.c_double), ("seconds", ctypes.c_double),
                ("vcycles", ctypes.c_int)]


_lib = None
P = ctypes.c_void_p
I64P = ctypes.POINTER(ctypes.c_int64)


def lib():
    """Load librmg.so (raises when it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with "
                          "`python -m paper_2103_11962_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "rmg_options_default": (None, [ctypes.POINTER(Options)]),
        "rmg_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, P]),
        "rmg_destroy": (None, [P]),
        "rmg_last_error": (ctypes.c_char_p, [P]),
        "rmg_set_stream": (ctypes.c_int, [P, P]),
        "rmg_layout_create": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int64,
                                             P, ctypes.POINTER(P)]),
        "rmg_layout_destroy": (None, [P]),
        "rmg_layout_sizes": (ctypes.c_int, [P, I64P, I64P, I64P, I64P]),
        "rmg_operator_from_csr": (ctypes.c_int, [P, ctypes.c_int, P, P, P]),
        "rmg_operator_from_region_stencils": (ctypes.c_int, [P, ctypes.c_int, P]),
        "rmg_operator_from_block_csr": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, P, P, P]),
        "rmg_operator_from_host_csr": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, P, P, P]),
        "rmg_hier_dofs_per_node": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int)]),
        "rmg_regional_apply": (ctypes.c_int, [P, P, P]),
        "rmg_comp_to_reg": (ctypes.c_int, [P, P, P]),
        "rmg_reg_to_comp": (ctypes.c_int, [P, P, P, ctypes.c_int]),
        "rmg_setup": (ctypes.c_int, [P, ctypes.POINTER(Options), ctypes.POINTER(P)]),
        "rmg_setup_numeric": (ctypes.c_int, [P]),
        "rmg_hier_destroy": (None, [P]),
        "rmg_vcycle_apply": (ctypes.c_int, [P, P, P, ctypes.c_int]),
        "rmg_pcg_solve": (ctypes.c_int, [P, P, P, ctypes.c_double, ctypes.c_int, P,
                                         ctypes.POINTER(SolveInfo)]),
        "rmg_hier_level_sizes": (ctypes.c_int, [P, ctypes.c_int, I64P, I64P,
                                                ctypes.POINTER(ctypes.c_int)]),
        "rmg_hier_level_export": (ctypes.c_int, [P, ctypes.c_int, P, P, P]),
        "rmg_hier_lambda": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "rmg_hier_galerkin": (ctypes.c_int, [P, ctypes.c_int]),
        "rmg_hier_tile_shape": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int)]),
        "rmg_hier_coef_planes": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "rmg_hier_coarse_matrix": (ctypes.c_int, [P, I64P, P, P]),
        "rmg_hier_vcycle_launches": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int)]),
        "rmg_launch_count": (ctypes.c_ulonglong, []),
        "rmg_hier_set_transfer_weights": (ctypes.c_int, [P, ctypes.c_int, P]),
        "rmg_hier_opdep_weights": (ctypes.c_int, [P, ctypes.c_int, P]),
        "rmg_hier_constant_weights": (ctypes.c_int, [P, ctypes.c_int, P]),
        "rmg_hier_convergence_factor": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_ulonglong,
                                                       ctypes.POINTER(ctypes.c_double)]),
        "rmg_hier_region_energies": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_ulonglong, P, P]),
        "rmg_hier_blend_weights": (ctypes.c_int, [P, ctypes.c_int, P, P, P]),
        "rmg_hier_region_colours": (ctypes.c_int, [P, P, ctypes.POINTER(ctypes.c_int)]),
        "rmg_mlp_num_params": (ctypes.c_int, []),
        "rmg_mlp_create": (ctypes.c_int, [P, P, ctypes.POINTER(P)]),
        "rmg_mlp_destroy": (None, [P]),
        "rmg_mlp_get_params": (ctypes.c_int, [P, P]),
        "rmg_mlp_forward": (ctypes.c_int, [P, ctypes.c_int, P, P]),
        "rmg_mlp_gradient": (ctypes.c_int, [P, ctypes.c_int, P, P, P, P, P]),
        "rmg_mlp_train": (ctypes.c_int, [P, ctypes.c_int, P, P, P, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_float, ctypes.c_ulonglong, P]),
        "rmg_hier_mlp_features": (ctypes.c_int, [P, ctypes.c_int, P]),
        "rmg_hier_mlp_weights": (ctypes.c_int, [P, ctypes.c_int, P, P]),
        "rmg_regional_apply_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, ctypes.c_int,
                                                     P, P, ctypes.c_int64, P, P, P,
                                                     ctypes.c_char_p, ctypes.c_int]),
        "rmg_hier_probe": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_longlong)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names of the C ABI functions this binding expects."""
    return ["rmg_options_default", "rmg_create", "rmg_destroy", "rmg_last_error",
            "rmg_set_stream", "rmg_layout_create", "rmg_layout_destroy", "rmg_layout_sizes",
            "rmg_operator_from_csr", "rmg_operator_from_region_stencils", "rmg_regional_apply",
            "rmg_comp_to_reg", "rmg_reg_to_comp", "rmg_setup", "rmg_setup_numeric",
            "rmg_hier_destroy", "rmg_vcycle_apply", "rmg_pcg_solve", "rmg_hier_level_sizes",
            "rmg_hier_level_export", "rmg_hier_lambda", "rmg_hier_coarse_matrix",
            "rmg_hier_vcycle_launches", "rmg_launch_count", "rmg_hier_probe",
            "rmg_regional_apply_static", "rmg_hier_set_transfer_weights",
            "rmg_operator_from_block_csr", "rmg_operator_from_host_csr",
            "rmg_hier_dofs_per_node",
            "rmg_hier_opdep_weights", "rmg_hier_constant_weights", "rmg_hier_convergence_factor",
            "rmg_hier_region_energies", "rmg_hier_blend_weights", "rmg_hier_region_colours",
            "rmg_hier_tile_shape", "rmg_hier_coef_planes", "rmg_hier_galerkin",
            "rmg_mlp_num_params", "rmg_mlp_create",
            "rmg_mlp_destroy", "rmg_mlp_get_params", "rmg_mlp_forward", "rmg_mlp_gradient",
            "rmg_mlp_train", "rmg_hier_mlp_features", "rmg_hier_mlp_weights"]


def regional_apply_static(dim, region_dims, stencil, coeffs, region_gids, n_composite, u, y,
                          stream=None):
    """y = Psi^T Psi [[A]] u through the entry point that allocates no device memory.

    For callers that cannot allocate device memory when they apply the operator; the
    scratch lives in a fixed device array inside librmg.so (see include/rmg.h)."""
    rd = np.ascontiguousarray(np.asarray(region_dims, dtype=np.int32).reshape(-1))
    buf = ctypes.create_string_buffer(512)
    st = lib().rmg_regional_apply_static(int(dim), rd.size // 3, rd.ctypes.data_as(P),
                                         int(stencil), _ptr(coeffs), _ptr(region_gids),
                                         int(n_composite), _ptr(u), _ptr(y),
                                         ctypes.c_void_p(stream or 0), buf, 512)
    if st != RMG_OK:
        raise RmgError(st, buf.value.decode())


def launch_count() -> int:
    """Kernels launched by librmg.so so far in this process."""
    return int(lib().rmg_launch_count())


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a, dtype):
    """Address of a contiguous host array (CPU torch tensor or numpy array) of `dtype`."""
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags.c_contiguous:
            raise TypeError(f"host array must be C-contiguous {np.dtype(dtype).name}")
        return ctypes.c_void_p(a.ctypes.data)
    if a.device.type != "cpu" or not a.is_contiguous() or a.element_size() != np.dtype(dtype).itemsize:
        raise TypeError("host tensor must be a contiguous CPU tensor of the right type")
    return ctypes.c_void_p(a.data_ptr())


def default_options(**kw) -> Options:
    o = Options()
    lib().rmg_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Context:
    def __init__(self, device=0, stream=None):
        import torch
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        h = P()
        st = lib().rmg_create(ctypes.byref(h), device, ctypes.c_void_p(stream))
        if st != RMG_OK:
            raise RmgError(st, "rmg_create failed")
        self.h = h

    def check(self, st):
        if st != RMG_OK:
            raise RmgError(st, lib().rmg_last_error(self.h).decode())

    def set_stream(self, stream):
        self.check(lib().rmg_set_stream(self.h, ctypes.c_void_p(stream)))

    def close(self):
        if self.h:
            lib().rmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Layout:
    """Region layout: region dims (host), regional->composite ids and Dirichlet mask (device)."""

    def __init__(self, ctx: Context, dim, region_dims, region_gids, n_composite, dirichlet=None):
        self.ctx = ctx
        rd = np.ascontiguousarray(np.asarray(region_dims, dtype=np.int32).reshape(-1))
        self._rd = rd
        self.nregions = rd.size // 3
        self._keep = (region_gids, dirichlet)
        h = P()
        ctx.check(lib().rmg_layout_create(
            ctx.h, dim, rd.size // 3, rd.ctypes.data_as(P), _ptr(region_gids), int(n_composite),
            _ptr(dirichlet), ctypes.byref(h)))
        self.h = h

    def sizes(self):
        a, b, c, d = (ctypes.c_int64() for _ in range(4))
        self.ctx.check(lib().rmg_layout_sizes(self.h, ctypes.byref(a), ctypes.byref(b),
                                              ctypes.byref(c), ctypes.byref(d)))
        return dict(n_regional=a.value, n_composite=b.value, n_groups=c.value,
                    n_group_slots=d.value)

    def operator_from_csr(self, stencil, rowptr, col, val):
        self._csr = (rowptr, col, val)
        self.ctx.check(lib().rmg_operator_from_csr(self.h, stencil, _ptr(rowptr), _ptr(col),
                                                   _ptr(val)))
        self._csr = None

    def operator_from_block_csr(self, stencil, dofs_per_node, rowptr, col, val):
        self.ctx.check(lib().rmg_operator_from_block_csr(self.h, stencil, dofs_per_node,
                                                         _ptr(rowptr), _ptr(col), _ptr(val)))

    def operator_from_host_csr(self, stencil, dofs_per_node, rowptr, col, val):
        """Split a composite CSR held in host memory (CPU torch tensors or numpy arrays of
        int64 / int64 / float64; page-locked tensors give DMA copies)."""
        self.ctx.check(lib().rmg_operator_from_host_csr(self.h, stencil, dofs_per_node,
                                                        _host_ptr(rowptr, np.int64),
                                                        _host_ptr(col, np.int64),
                                                        _host_ptr(val, np.float64)))

    def operator_from_region_stencils(self, stencil, coeffs):
        self.ctx.check(lib().rmg_operator_from_region_stencils(self.h, stencil, _ptr(coeffs)))

    def regional_apply(self, u, y):
        self.ctx.check(lib().rmg_regional_apply(self.h, _ptr(u), _ptr(y)))

    def comp_to_reg(self, c, r):
        self.ctx.check(lib().rmg_comp_to_reg(self.h, _ptr(c), _ptr(r)))

    def reg_to_comp(self, r, c, average=True):
        self.ctx.check(lib().rmg_reg_to_comp(self.h, _ptr(r), _ptr(c), 1 if average else 0))

    def close(self):
        if getattr(self, "h", None):
            lib().rmg_layout_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hierarchy:
    def __init__(self, layout: Layout, options: Options = None):
        self.layout = layout
        self.ctx = layout.ctx
        self.options = options if options is not None else default_options()
        h = P()
        self.ctx.check(lib().rmg_setup(layout.h, ctypes.byref(self.options), ctypes.byref(h)))
        self.h = h

    def setup_numeric(self):
        self.ctx.check(lib().rmg_setup_numeric(self.h))

    def vcycle(self, r, z, regional=False):
        self.ctx.check(lib().rmg_vcycle_apply(self.h, _ptr(r), _ptr(z), 1 if regional else 0))

    def pcg(self, b, x, rtol=1e-10, maxit=200, history=True):
        info = SolveInfo()
        hist = np.zeros(maxit + 1) if history else None
        st = lib().rmg_pcg_solve(self.h, _ptr(b), _ptr(x), float(rtol), int(maxit),
                                 hist.ctypes.data_as(P) if hist is not None else None,
                                 ctypes.byref(info))
        if st not in (RMG_OK, 6):
            self.ctx.check(st)
        out = dict(iterations=info.iterations, relres=info.relres,
                   true_relres=info.true_relres, seconds=info.seconds, vcycles=info.vcycles,
                   converged=(st == RMG_OK))
        if hist is not None:
            out["history"] = hist[:info.iterations + 1].copy()
        return out

    def level_sizes(self, level):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        s = ctypes.c_int()
        self.ctx.check(lib().rmg_hier_level_sizes(self.h, level, ctypes.byref(a), ctypes.byref(b),
                                                  ctypes.byref(s)))
        return a.value, b.value, s.value

    def dofs_per_node(self):
        v = ctypes.c_int()
        self.ctx.check(lib().rmg_hier_dofs_per_node(self.h, ctypes.byref(v)))
        return v.value

    def level_export(self, level, coeffs=None, dinv=None, gids=None):
        self.ctx.check(lib().rmg_hier_level_export(self.h, level, _ptr(coeffs), _ptr(dinv),
                                                   _ptr(gids)))

    def galerkin(self, level):
        """Recompute the Galerkin product of level -> level + 1 alone (asynchronous)."""
        self.ctx.check(lib().rmg_hier_galerkin(self.h, level))

    def tile_shape(self, level):
        """(tx, ty, tz) of the level's stencil-sweep tiles; (0, 0, 0) for runs of 256 nodes."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self.ctx.check(lib().rmg_hier_tile_shape(self.h, level, ctypes.byref(a), ctypes.byref(b),
                                                 ctypes.byref(c)))
        return a.value, b.value, c.value

    def coef_planes(self, level):
        """Stencil coefficients per node the cycle's sweeps read on a level (half form: fewer)."""
        v = ctypes.c_int()
        self.ctx.check(lib().rmg_hier_coef_planes(self.h, level, ctypes.byref(v)))
        return v.value

    def lam(self, level):
        v = ctypes.c_double()
        self.ctx.check(lib().rmg_hier_lambda(self.h, level, ctypes.byref(v)))
        return v.value

    def coarse_matrix(self):
        nc = ctypes.c_int64()
        self.ctx.check(lib().rmg_hier_coarse_matrix(self.h, ctypes.byref(nc), None, None))
        n = nc.value
        B = self.dofs_per_node()
        dense = np.zeros((n * B, n * B))
        ids = np.zeros(n, dtype=np.int64)
        if n:
            self.ctx.check(lib().rmg_hier_coarse_matrix(self.h, ctypes.byref(nc),
                                                        dense.ctypes.data_as(P),
                                                        ids.ctypes.data_as(P)))
        return dense, ids

    def set_transfer_weights(self, level, wr):
        """Stored per-node interpolation weights for level -> level+1 (None = linear)."""
        self.ctx.check(lib().rmg_hier_set_transfer_weights(self.h, level, _ptr(wr)))

    def constant_weights(self, level, wr):
        """Piecewise-constant (nearest coarse node) weights of a level into wr (3 * n_r)."""
        self.ctx.check(lib().rmg_hier_constant_weights(self.h, level, _ptr(wr)))

    def opdep_weights(self, level, wr):
        """Operator-dependent (series-resistance) weights of a level into wr (3 * n_r)."""
        self.ctx.check(lib().rmg_hier_opdep_weights(self.h, level, _ptr(wr)))

    def convergence_factor(self, iters=6, seed=7):
        """Mean A-norm error reduction per V-cycle, measured as a stationary solver."""
        v = ctypes.c_double()
        self.ctx.check(lib().rmg_hier_convergence_factor(self.h, int(iters), int(seed),
                                                         ctypes.byref(v)))
        return v.value

    def region_energies(self, iters=6, seed=7):
        """(e0, eK): per-region energies e_k^T A^(k) e_k of the error before and after `iters`
        V-cycles as a stationary solver (numpy arrays, one entry per region)."""
        nreg = self.layout.nregions
        e0 = np.zeros(nreg)
        eK = np.zeros(nreg)
        self.ctx.check(lib().rmg_hier_region_energies(self.h, int(iters), int(seed),
                                                      e0.ctypes.data_as(P), eK.ctypes.data_as(P)))
        return e0, eK

    def blend_weights(self, level, accept, learned, out):
        """Learned weights at nodes whose regions all accept, linear weights elsewhere."""
        acc = np.ascontiguousarray(np.asarray(accept, dtype=np.uint8))
        self.ctx.check(lib().rmg_hier_blend_weights(self.h, level, acc.ctypes.data_as(P),
                                                    _ptr(learned), _ptr(out)))

    def region_colours(self):
        """(colours, ncolours): a colouring of the regions in which touching regions differ."""
        col = np.zeros(self.layout.nregions, dtype=np.int32)
        nc = ctypes.c_int()
        self.ctx.check(lib().rmg_hier_region_colours(self.h, col.ctypes.data_as(P),
                                                     ctypes.byref(nc)))
        return col, nc.value

    def mlp_features(self, level, feats):
        self.ctx.check(lib().rmg_hier_mlp_features(self.h, level, _ptr(feats)))

    def mlp_weights(self, level, mlp, wr):
        self.ctx.check(lib().rmg_hier_mlp_weights(self.h, level, mlp.h, _ptr(wr)))

    def probe(self, reset=True):
        """(total ms, launches) of the timed level-0 smoother kernel since the last reset."""
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        self.ctx.check(lib().rmg_hier_probe(self.h, 1 if reset else 0, ctypes.byref(ms),
                                            ctypes.byref(n)))
        return ms.value, n.value

    def vcycle_launches(self):
        v = ctypes.c_int()
        self.ctx.check(lib().rmg_hier_vcycle_launches(self.h, ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "h", None):
            lib().rmg_hier_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The learned prolongator's network (parameters live on the device)."""

    def __init__(self, ctx: Context, init_params):
        self.ctx = ctx
        p = np.ascontiguousarray(np.asarray(init_params, dtype=np.float32))
        if p.size != lib().rmg_mlp_num_params():
            raise ValueError("wrong parameter count")
        h = P()
        ctx.check(lib().rmg_mlp_create(ctx.h, p.ctypes.data_as(P), ctypes.byref(h)))
        self.h = h

    @staticmethod
    def num_params():
        return int(lib().rmg_mlp_num_params())

    def params(self):
        out = np.zeros(self.num_params(), dtype=np.float32)
        self.ctx.check(lib().rmg_mlp_get_params(self.h, out.ctypes.data_as(P)))
        return out

    def forward(self, feats, out):
        self.ctx.check(lib().rmg_mlp_forward(self.h, int(feats.shape[0]), _ptr(feats), _ptr(out)))

    def gradient(self, feats, labels, mask):
        g = np.zeros(self.num_params(), dtype=np.float32)
        loss = ctypes.c_float()
        self.ctx.check(lib().rmg_mlp_gradient(self.h, int(feats.shape[0]), _ptr(feats),
                                              _ptr(labels), _ptr(mask), g.ctypes.data_as(P),
                                              ctypes.byref(loss)))
        return float(loss.value), g

    def train(self, feats, labels, mask, steps, batch=16384, lr=1e-3, seed=0):
        hist = np.zeros(steps, dtype=np.float32)
        self.ctx.check(lib().rmg_mlp_train(self.h, int(feats.shape[0]), _ptr(feats), _ptr(labels),
                                           _ptr(mask), int(steps), int(batch), float(lr),
                                           int(seed), hist.ctypes.data_as(P)))
        return hist

    def close(self):
        if getattr(self, "h", None):
            lib().rmg_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
