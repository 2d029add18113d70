"""Benchmark: region multigrid preconditioned CG to a 1e-10 relative residual.

One step = one linear system solved from device-resident inputs through the C ABI:
non-invasive split of the composite CSR matrix into region stencils, numeric hierarchy setup
(diagonals, regional Galerkin products, Chebyshev power method, coarsest Cholesky and inverse)
and PCG with one regional V-cycle per iteration. The mesh (region layout, interface groups)
and the hierarchy's buffers and CUDA graph are built once before timing.

Headline: the largest single-GPU workload, the 3D Q1 Laplacian on 8x8x8 regions of 55^3 nodes
(80M unknowns), with the V-cycle in FP32 inside FP64 flexible CG. The plain FP64 method and the
BF16-coefficient cycle are measured beside it on the same system, all to the same 1e-10 relative
FP64 residual. Every other workload (2D Poisson, 3D diffusion with uneven regions, high-contrast
diffusion, elasticity) is measured in the same invocation as a sub-record in all three
precisions (``configs``).

Metric: V-cycle DOF/s = unknowns x V-cycles of the step / step time (whole step, setup
included), and the time to the 1e-10 relative residual.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
       [--workload NAME] [--configs all|none|NAME,...] [--precision fp32|fp64|bf16]
       [--no-mixed] [--no-e2e] [--no-cpu] [--no-learned] [--json-out FILE]
Under torchrun every rank solves its own copy of the system (independent problems, no
collective on the data path; weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "V-cycle DOF/s & time to 1e-10 rel. residual, mixed/learned vs plain FP64"
UNIT = "DOF*V-cycles/s"
RTOL = 1e-10
HEADLINE = "c3_q1laplace3d"
SUBRECORDS = ("c1_poisson2d", "c2_diffusion3d", "c4_highcontrast3d", "c5_elasticity_full")


# Per-node algorithmic bytes and FP64 flops of the timed kernel, the fine-level Chebyshev
# recurrence sweep (k_stencil_half, k_stencil or k_bstencil with EpiCheb): its coefficient
# streams, u, b, D~^-1, d read; d and u_out written; 1-byte multiplicity read.
def sweep_bytes(prec, planes, B=1):
    """Algorithmic bytes per regional node of the Chebyshev recurrence sweep: the stencil
    coefficients the sweep reads per node (`planes`: B*B*S, or (S+1)/2 for the half form of a
    symmetric FP32 stencil, as rmg_hier_coef_planes reports), u, b, D~^-1 and d read and d,
    u_out written for each of the B components, and the 1-byte multiplicity."""
    cb = {"fp64": 8, "fp32": 4, "bf16": 2}[prec]
    vb = 8 if prec == "fp64" else 4
    return planes * cb + B * 6 * vb + 1


def sweep_flops(stencil, B=1):
    """FP64 flops per regional node of the same sweep (2 per stored coefficient + 6 per dof)."""
    return 2 * B * B * stencil + 6 * B


CHEB = dict(levels=4, smoother="chebyshev", nu1=1, nu2=1, degree=3)
WORKLOADS = {
    "c3_q1laplace3d": dict(CHEB, l2="inputs larger than L2",
                           desc="3D Q1 Laplacian (27-point), 8x8x8 regions of 55^3 nodes (433^3 "
                                "composite, 80M unknowns, 2.2G nonzeros; CSR assembled on the "
                                "device by the workload generator), rhs U[-1,1] seed 2"),
    "c2_diffusion3d": dict(CHEB, l2="inputs larger than L2",
                           desc="3D 7-point variable-coefficient diffusion, 8x8x4 regions with "
                                "per-axis node counts from {28,55,82} (seed 1), log-normal "
                                "per-element kappa (sigma 1), Chebyshev degree 3, 4 levels"),
    "c4_highcontrast3d": dict(CHEB, l2="inputs larger than L2",
                              desc="3D 7-point diffusion, 7x7x7 regions with per-axis node "
                                   "counts from {28,55,82} (seed 3), kappa constant per region, "
                                   "log-uniform in [1e-3, 1e3]"),
    "c5_elasticity_full": dict(CHEB, power_iters=30, l2="inputs larger than L2",
                               desc="3D linear elasticity, 8x8x8 regions with per-axis node "
                                    "counts from {28,55} (seed 95, the first seed from 4 on "
                                    "giving 60M +- 15% dofs: 271x271x244 nodes, 53.6M unknowns, "
                                    "4.4G nonzeros; CSR assembled on the device), E log-normal "
                                    "(sigma 0.5), nu 0.3, x=0 clamped, uniform body load; 30 "
                                    "power steps"),
    "c1_poisson2d": dict(levels=4, smoother="jacobi", nu1=2, nu2=2, omega=0.67,
                         l2="L2 flushed between timed steps (inputs fit in L2)",
                         desc="2D Poisson 5-point, 2x2 regions of 82x82, Jacobi 0.67, nu 2/2, "
                              "4 levels"),
    # reduced sizes for profiling and for the oracle comparisons
    "c3_q1laplace3d_slice": dict(CHEB, l2="inputs larger than L2",
                                 desc="3D Q1 Laplacian (27-point), 4x4x4 regions of 55^3 nodes "
                                      "(the 4x4x4-region slice of the 8x8x8 configuration)"),
    "c3_quarter": dict(CHEB, l2="inputs larger than L2",
                       desc="3D Q1 Laplacian (27-point), 4x4x2 regions of 55^3 nodes "
                            "(profiling size)"),
    "c2_quarter": dict(CHEB, l2="inputs larger than L2",
                       desc="C2-shaped 3D 7-point diffusion on 4x4x2 regions (profiling size)"),
    "offset_heldout": dict(CHEB, l2="inputs larger than L2",
                           desc="3D 7-point diffusion, 4x4x4 regions with per-axis node counts "
                                "from {28,55} (seed 77), kappa log-uniform in [1e-3, 1e3] on "
                                "8x8x8 boxes whose faces lie off the coarse-grid planes (held "
                                "out from the learned prolongator's training family)"),
    "c5_elasticity": dict(CHEB, power_iters=30, l2="inputs larger than L2",
                          desc="3D linear elasticity, Q1 hexahedra, 3 dofs per node, 3x3x3 "
                               "regions of 28^3 nodes (the paper's 82^3 elasticity mesh), E "
                               "log-normal (sigma 0.5), nu 0.3, x=0 clamped, uniform body load"),
}


def workload_config(name):
    """The `config` object of a workload: the same in the native and the reference arm."""
    cfg = WORKLOADS[name]
    return {"workload": name, "desc": cfg["desc"], "smoother": cfg["smoother"],
            "levels": cfg["levels"], "rtol": RTOL, "l2": cfg["l2"]}


def make_problem(name, dev):
    import workloads as W
    from workloads import device as WD
    if name == "c3_q1laplace3d":
        return WD.q1_laplace3d(region_grid=(8, 8, 8), n=55, seed=2, device=dev)
    if name == "c3_q1laplace3d_slice":
        return WD.q1_laplace3d(region_grid=(4, 4, 4), n=55, seed=2, device=dev)
    if name == "c3_quarter":
        return WD.q1_laplace3d(region_grid=(4, 4, 2), n=55, seed=2, device=dev)
    if name == "c2_diffusion3d":
        return WD.diffusion3d_7pt(region_grid=(8, 8, 4), choices=(28, 55, 82), seed=1, device=dev)
    if name == "c2_quarter":
        return WD.diffusion3d_7pt(region_grid=(4, 4, 2), choices=(28, 55, 82), seed=1, device=dev)
    if name == "c4_highcontrast3d":
        return WD.highcontrast3d_7pt(region_grid=(7, 7, 7), choices=(28, 55, 82), seed=3,
                                     device=dev)
    if name == "c5_elasticity_full":
        return WD.elasticity3d(region_grid=(8, 8, 8), choices=(28, 55), seed=95, device=dev)
    if name == "c5_elasticity":
        return W.elasticity3d(region_grid=(3, 3, 3), choices=(28,), seed=4)
    if name == "offset_heldout":
        return W.highcontrast3d_offset(region_grid=(4, 4, 4), choices=(28, 55), seed=77, blocks=8)
    return W.config(name)


def training_family(family):
    """Seeded small operators the learned prolongator is trained on: 2x2x2 regions of 10^3
    nodes of the workload's PDE family (seeds 1000 + s for the high-contrast family, as the
    C4 configuration prescribes)."""
    import workloads as W
    if family == "c4":
        return lambda s: W.highcontrast3d_7pt(region_grid=(2, 2, 2), choices=(10,), seed=1000 + s)
    if family == "offset":
        return lambda s: W.highcontrast3d_offset(region_grid=(2, 2, 2), choices=(10,),
                                                 seed=5000 + s)
    return lambda s: W.diffusion3d_7pt(region_grid=(2, 2, 2), choices=(10, 19, 28), seed=2000 + s)


def kernel_source_hash():
    """First 16 hex digits of the sha256 of the sources that define the timed sweeps."""
    import hashlib
    h = hashlib.sha256()
    for f in ("rmg_internal.cuh", "rmg_kernels.cuh", "rmg_launch.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2103_11962_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, prec):
    """DRAM bytes per regional node of the timed sweep measured by ncu
    (profiles/sweep_dram_bytes.json), or None when that capture predates the current kernel
    sources or does not cover this kernel and precision."""
    path = os.path.join(ROOT, "profiles", "sweep_dram_bytes.json")
    if not os.path.exists(path):
        return None, None
    d = json.load(open(path))
    if d.get("kernel_source_sha256_16") != kernel_source_hash():
        return None, None
    e = d.get("kernels", {}).get(f"{kernel} {prec}")
    if not e:
        return None, None
    return float(e["dram_bytes_per_node"]), e.get("capture", "")


def device_problem(p, dev):
    """Device arrays of a problem: uploaded from the host generator, or already on the device
    (the workloads assembled there)."""
    from paper_2103_11962_gb300 import DeviceProblem, upload
    if hasattr(p, "rowptr"):
        import numpy as np
        import torch
        return DeviceProblem(dim=p.dim, stencil=p.stencil, n=p.n_nodes,
                             region_dims=np.asarray(p.region_dims, dtype=np.int32),
                             rowptr=p.rowptr, col=p.col, val=p.val, b=p.b,
                             gids=torch.from_numpy(p.region_gids).to(dev),
                             dirichlet=torch.from_numpy(p.dirichlet).to(dev))
    return upload(p, dev)


L2_BYTES = 129 * 1000 ** 2       # L2 of one GB300


def input_bytes(dp):
    """Bytes of one step's inputs: the composite CSR and the right-hand side."""
    return sum(int(t.numel()) * t.element_size() for t in (dp.rowptr, dp.col, dp.val, dp.b))


def l2_flush_buffer(dp, dev):
    """A buffer of twice the L2 size when a step's inputs fit in L2, else None. Writing it
    between timed steps evicts what the previous step left in L2."""
    import torch
    if input_bytes(dp) > L2_BYTES:
        return None
    return torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (every rank solves its own system; the job ends with the last
    one). Identity without a process group."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_value(units_per_rank, world, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (ms / 1e3)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    out = {"hbm_gbs": 6800.0, "src": "fallback"}
    if os.path.exists(p):
        d = json.load(open(p))
        out = {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured",
               "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0))}
    # FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x max SM clock (measured 1.196 TFLOP/s
    # with dependent-free FMA chains at 1995 MHz on this part).
    out["fp64_tflops"] = 152 * 2 * 2 * out.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    return out


def host_info():
    """nproc and the CPU model of the host (lscpu, else /proc/cpuinfo)."""
    info = {"nproc": os.cpu_count()}
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    info["cpu_model"] = model
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable"):
                info["mem_available_gb"] = round(int(ln.split()[1]) / 1e6, 1)
    except Exception:
        pass
    return info


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2])); power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------ oracle legs
# The CPU oracle (plain FP64 region multigrid, numpy/scipy) on a bounded sample of a workload:
# split, hierarchy and PCG to 1e-10, timed inside the process (imports excluded).
ORACLE_SAMPLES = {
    "c3": ("W.q1_laplace3d(region_grid=(2, 2, 2), n=55, seed=2)", "cheb",
           "C3-shaped 2x2x2-region Q1 sample (regions of 55^3 nodes, as in the workload; "
           "109^3 composite nodes, seed 2)"),
    "c3_small": ("W.q1_laplace3d(region_grid=(2, 2, 2), n=28, seed=2)", "cheb",
                 "C3-shaped 2x2x2-region Q1 sample (regions of 28^3 nodes; 55^3 composite "
                 "nodes, seed 2)"),
    "c2": ("W.diffusion3d_7pt(region_grid=(2, 2, 2), choices=(28, 55, 82), seed=1)", "cheb",
           "C2-shaped 2x2x2-region instance (slabs from {28,55,82}, seed 1, log-normal kappa)"),
    "c4": ("W.highcontrast3d_7pt(region_grid=(2, 2, 2), choices=(28, 55, 82), seed=3)", "cheb",
           "C4-shaped 2x2x2-region high-contrast instance (slabs from {28,55,82}, seed 3)"),
    "c5": ("W.elasticity3d(region_grid=(2, 2, 2), choices=(10, 19), seed=4)", "block",
           "C5-shaped 2x2x2-region elasticity instance (slabs from {10,19}, seed 4)"),
    "c1": ("W.config('c1_poisson2d')", "jacobi", "full C1 workload"),
}


def oracle_sample_key(workload, small=False):
    k = workload[:2]
    if k == "c3" and small:
        return "c3_small"
    return k if k in ORACLE_SAMPLES else "c2"


def oracle_sample_cmd(key, save_x=None):
    """Command that runs the CPU oracle pipeline on sample `key` and prints a JSON summary;
    with save_x, the solution is written there (numpy .npy)."""
    expr, kind, sample = ORACLE_SAMPLES[key]
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
import workloads as W
from oracle import cycle, hierarchy, krylov
p = {expr}
kind = {kind!r}
t0 = time.perf_counter()
if kind == 'block':
    levels = hierarchy.build_block(p, 4)
    perm = hierarchy.node_major_to_component_major(p.n_nodes, p.dofs_per_node)
    A, b = levels[0].A, p.b[perm]
    o = cycle.Options(smoother='chebyshev', nu1=1, nu2=1, degree=3, power_iters=30)
else:
    levels = hierarchy.build(p, 4)
    A, b = p.A, p.b
    if kind == 'jacobi':
        o = cycle.Options(smoother='jacobi', nu1=2, nu2=2, omega=0.67)
    else:
        o = cycle.Options(smoother='chebyshev', nu1=1, nu2=1, degree=3)
mg = cycle.RegionalMG(levels, o)
counts = {{}}
x, it, hist = krylov.pcg(A, b, krylov.regional_preconditioner(mg), rtol={RTOL}, counts=counts)
t1 = time.perf_counter()
if {save_x!r}:
    np.save({save_x!r}, x)
print(json.dumps(dict(seconds=t1 - t0, iterations=it, vcycles=counts['vcycles'],
                      unknowns=p.n_unknowns, n_regional=p.n_regional_nodes,
                      sample={sample!r})))
"""
    return [sys.executable, "-c", code]


def _oracle_env():
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    return env


def run_oracle_sample(key, save_x=None):
    """One single-threaded oracle process on sample `key`."""
    res = subprocess.run(oracle_sample_cmd(key, save_x), capture_output=True, text=True,
                         env=_oracle_env(), timeout=900)
    if res.returncode != 0:
        raise RuntimeError(res.stderr[-2000:])
    d = json.loads(res.stdout.strip().splitlines()[-1])
    d["value"] = d["unknowns"] * d["vcycles"] / d["seconds"]
    return d


def run_oracle_parallel(key, procs):
    """`procs` single-threaded oracle processes on independent copies of sample `key`, started
    together: the multi-core throughput of the oracle on the host. Each copy's time is
    measured inside its process; the batch takes as long as its slowest copy."""
    ps = [subprocess.Popen(oracle_sample_cmd(key), stdout=subprocess.PIPE,
                           stderr=subprocess.PIPE, text=True, env=_oracle_env())
          for _ in range(procs)]
    outs = []
    for pr in ps:
        o, e = pr.communicate(timeout=1800)
        if pr.returncode != 0:
            raise RuntimeError(e[-2000:])
        outs.append(json.loads(o.strip().splitlines()[-1]))
    worst = max(d["seconds"] for d in outs)
    units = sum(d["unknowns"] * d["vcycles"] for d in outs)
    return dict(value=units / worst, seconds=worst, procs=procs, sample=outs[0]["sample"],
                iterations=outs[0]["iterations"], unknowns=outs[0]["unknowns"])


def oracle_procs(info):
    """Oracle processes for the multi-core leg: the host's cores, at most 16, bounded by
    memory (about 3 GB per C3-sample copy)."""
    n = max(1, min(16, info.get("nproc") or 1))
    mem = info.get("mem_available_gb")
    if mem:
        n = max(1, min(n, int(mem // 4)))
    return n


# ------------------------------------------------------------------------------ native leg
class Bench:
    """Device, stream and timing helpers of the native arm."""

    def __init__(self, args, rank, world, local_rank, dist):
        import torch
        from paper_2103_11962_gb300 import rmg
        self.args, self.rank, self.world, self.dist = args, rank, world, dist
        self.torch, self.rmg = torch, rmg
        self.dev = f"cuda:{local_rank}"
        self.local_rank = local_rank
        self.stream = torch.cuda.current_stream(local_rank)
        self.ctx = rmg.Context(local_rank, self.stream.cuda_stream)

    def options(self, name, prec):
        rmg = self.rmg
        cfg = WORKLOADS[name]
        o = rmg.default_options(levels=cfg["levels"], precision={"fp64": rmg.FP64,
                                                                "fp32": rmg.FP32,
                                                                "bf16": rmg.FP32_BF16COEF}[prec])
        sm = self.args.smoother or cfg["smoother"]
        if sm == "chebyshev":
            o.smoother, o.nu1, o.nu2, o.cheb_degree = (rmg.CHEBYSHEV, cfg["nu1"], cfg["nu2"],
                                                        cfg.get("degree", 3))
        elif sm == "gs":
            o.smoother, o.nu1, o.nu2, o.omega = rmg.GAUSS_SEIDEL, 1, 1, 1.0
        else:
            o.smoother, o.nu1, o.nu2, o.omega = (rmg.JACOBI, cfg["nu1"], cfg["nu2"],
                                                 cfg.get("omega", 0.67))
        o.power_iters = cfg.get("power_iters", 10)
        o.tile_shape = self.args.tile_shape
        return o

    def timed(self, step, K, W_, flush):
        """W_ untimed steps, then K steps bracketed by a barrier and synchronisations, timed with
        CUDA events on the library's stream (with an L2 flush between steps when the inputs
        fit in L2). Returns (ms over ranks, step results, library launches)."""
        torch, rmg, stream = self.torch, self.rmg, self.stream
        for _ in range(W_):
            step()
        if self.dist:
            self.dist.barrier()
        torch.cuda.synchronize()
        l0 = rmg.launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if flush is None:
            ev0.record(stream)
            infos = [step() for _ in range(K)]
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
        else:
            infos, ms = [], 0.0
            for _ in range(K):
                flush.fill_(1)
                ev0.record(stream)
                infos.append(step())
                ev1.record(stream)
                torch.cuda.synchronize()
                ms += ev0.elapsed_time(ev1)
        launches = rmg.launch_count() - l0
        return max_over_ranks(ms, self.dist, self.dev), infos, launches


class Workload:
    """A workload's problem, device arrays and layout, and its per-precision measurements."""

    def __init__(self, B, name):
        self.B, self.name = B, name
        self.cfg = WORKLOADS[name]
        t = time.perf_counter()
        self.p = make_problem(name, B.dev)
        self.dp = device_problem(self.p, B.dev)
        B.torch.cuda.synchronize()
        self.gen_s = time.perf_counter() - t
        t = time.perf_counter()
        p, dp = self.p, self.dp
        self.lay = B.rmg.Layout(B.ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
        self.layout_ms = (time.perf_counter() - t) * 1e3
        self.x = B.torch.zeros(p.n, dtype=B.torch.float64, device=B.dev)
        self.flush = l2_flush_buffer(dp, B.dev)
        self.set_operator()

    def set_operator(self):
        p, dp = self.p, self.dp
        if p.dofs_per_node > 1:
            self.lay.operator_from_block_csr(p.stencil, p.dofs_per_node, dp.rowptr, dp.col, dp.val)
        else:
            self.lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)

    def hierarchy(self, prec):
        return self.B.rmg.Hierarchy(self.lay, self.B.options(self.name, prec))

    def step(self, h):
        self.set_operator()
        h.setup_numeric()
        self.x.zero_()
        return h.pcg(self.dp.b, self.x, rtol=RTOL, maxit=500, history=False)

    def measure(self, h, prec, K, W_, breakdown=False):
        """Time K steps of hierarchy h; the record of one precision."""
        p = self.p
        h.probe(reset=True)
        ms, infos, launches = self.B.timed(lambda: self.step(h), K, W_, self.flush)
        probe_ms, probe_n = h.probe(reset=True)
        info = infos[-1]
        rec = dict(ms_per_step=ms / K, pcg_iterations=info["iterations"],
                   vcycles_per_step=info["vcycles"], true_relres=info["true_relres"],
                   converged=all(i["converged"] for i in infos),
                   value=job_value(p.n_unknowns * info["vcycles"] * K, self.B.world, ms),
                   gpu_launches=int(launches))
        rec["roofline"] = self.roofline(h, prec, probe_ms, probe_n)
        if breakdown:
            rec["breakdown"] = self.breakdown(h)
        return rec

    def roofline(self, h, prec, probe_ms, probe_n):
        """Roofline of the dominant kernel, the fine-level Chebyshev (or Jacobi) sweep timed
        live by CUDA events recorded around one level-0 launch per V-cycle."""
        p = self.p
        kern_ms = probe_ms / max(1, probe_n)
        if not kern_ms > 0:
            return None
        pk = peaks()
        n_r0 = p.n_regional_nodes
        Bd = p.dofs_per_node
        planes0 = h.coef_planes(0)
        bytes_launch = sweep_bytes(prec, planes0, Bd) * n_r0
        flops_launch = sweep_flops(p.stencil, Bd) * n_r0
        gbs = bytes_launch / (kern_ms / 1e3) / 1e9
        tfl = flops_launch / (kern_ms / 1e3) / 1e12
        hbm_frac = gbs / pk["hbm_gbs"]
        kname = (f"k_bstencil<{p.stencil},{Bd}>" if Bd > 1 else
                 f"k_stencil_half<{p.stencil}>" if planes0 < p.stencil else
                 f"k_stencil<{p.stencil}>")
        epi = "EpiJacobi" if self.cfg["smoother"] == "jacobi" else "EpiCheb"
        r = dict(bound="hbm", achieved=round(gbs, 1), peak=pk["hbm_gbs"], unit="GB/s",
                 frac=round(hbm_frac, 4), peak_src=pk["src"] + " (MEASURED_PEAKS.json hbm_gbs)",
                 achieved_is="algorithmic bytes per launch / CUDA-event duration of the launch")
        if prec == "fp64" and tfl / pk["fp64_tflops"] > hbm_frac:
            r = dict(bound="alu", achieved=round(tfl, 4), peak=round(pk["fp64_tflops"], 4),
                     unit="TFLOP/s (FP64)", frac=round(tfl / pk["fp64_tflops"], 4),
                     peak_src="derived: 152 SM x 2 DFMA/clk x 2 flop x max SM clock",
                     hbm=dict(achieved=round(gbs, 1), peak=pk["hbm_gbs"], unit="GB/s",
                              frac=round(hbm_frac, 4)))
        tpn, cap = profiled_traffic(f"{kname} {epi}", prec)
        r.update(kernel=f"{kname[:-1]}, {epi}> level 0 ({prec}, {planes0} coefficients per node)",
                 ms_per_launch=round(kern_ms, 4), launches_timed=probe_n,
                 bytes_per_launch=bytes_launch, flops_per_launch=flops_launch,
                 bytes_per_node=sweep_bytes(prec, planes0, Bd), regional_nodes=n_r0,
                 traffic=(round(tpn * n_r0) if tpn else None),
                 traffic_src=(f"ncu dram__bytes_read.sum + dram__bytes_write.sum per node ({cap}) "
                              "x regional nodes" if tpn else None))
        if tpn:
            r["dram_gbs"] = round(tpn * n_r0 / (kern_ms / 1e3) / 1e9, 1)
            r["dram_frac"] = round(r["dram_gbs"] / pk["hbm_gbs"], 4)
        return r

    def breakdown(self, h):
        """Per-phase times of one step and the V-cycle alone (outside the timed region)."""
        torch, stream = self.B.torch, self.B.stream
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream); self.set_operator()
        e[1].record(stream); h.setup_numeric()
        e[2].record(stream); self.x.zero_()
        h.pcg(self.dp.b, self.x, rtol=RTOL, maxit=500, history=False)
        e[3].record(stream); torch.cuda.synchronize()
        out = dict(split_ms=e[0].elapsed_time(e[1]), setup_ms=e[1].elapsed_time(e[2]),
                   solve_ms=e[2].elapsed_time(e[3]), layout_ms_once=self.layout_ms,
                   generate_s_once=self.gen_s, vcycle_launches=h.vcycle_launches(),
                   tile_shapes=[list(h.tile_shape(l)) for l in range(self.cfg["levels"])])
        r = self.dp.b.clone()
        z = torch.empty_like(r)
        for _ in range(3):
            h.vcycle(r, z)
        torch.cuda.synchronize()
        e[0].record(stream)
        nrep = 20
        for _ in range(nrep):
            h.vcycle(r, z)
        e[1].record(stream); torch.cuda.synchronize()
        vc_ms = e[0].elapsed_time(e[1]) / nrep
        out["vcycle_ms"] = vc_ms
        out["vcycle_dof_per_s"] = self.p.n_unknowns / (vc_ms / 1e3)
        return out

    def problem_info(self):
        p = self.p
        return {"global_dims": list(p.global_dims), "regions": int(p.nregions),
                "unknowns": p.n_unknowns, "regional_nodes": p.n_regional_nodes,
                "composite_nnz": int(p.nnz if hasattr(p, "nnz") else p.A.nnz),
                "dofs_per_node": p.dofs_per_node,
                "l2_flush": self.flush is not None}

    def close(self):
        self.lay.close()
        del self.dp, self.p, self.x
        self.B.torch.cuda.empty_cache()


def precisions_of(args):
    return [args.precision] + ([] if args.no_mixed else
                               [q for q in ("fp64", "fp32", "bf16") if q != args.precision])


def measure_all(B, wl, precs, K, W_, headline_breakdown=True):
    """Every precision of a workload; the first one is the headline. Returns the records."""
    recs = {}
    for i, prec in enumerate(precs):
        h = wl.hierarchy(prec)
        recs[prec] = wl.measure(h, prec, K, W_, breakdown=(i == 0 and headline_breakdown))
        h.close()
    fp64 = recs.get("fp64", {}).get("ms_per_step")
    for r in recs.values():
        r["speedup_vs_fp64"] = fp64 / r["ms_per_step"] if fp64 else None
    return recs


def e2e_leg(B, wl, prec, K, W_):
    """The same step end to end through the C ABI with host buffers: the composite CSR goes in
    through rmg_operator_from_host_csr from page-locked host memory (its H2D copies inside the
    call), b is copied from page-locked memory, and the solution is read back to the host, all
    inside the timed region."""
    torch = B.torch
    p, dp = wl.p, wl.dp
    need_gb = input_bytes(dp) / 1e9
    info = host_info()
    if info.get("mem_available_gb") and info["mem_available_gb"] < 2.5 * need_gb + 16:
        return {"value": None, "unit": UNIT,
                "skipped": f"host memory: {info['mem_available_gb']} GB available, the pinned "
                           f"inputs need {need_gb:.1f} GB"}
    hp = {}
    for k in ("rowptr", "col", "val", "b"):
        t = getattr(dp, k)
        hp[k] = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
        hp[k].copy_(t)
    hx = torch.empty(p.n, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in hp.values())
    d2h = hx.numel() * hx.element_size()
    # the device CSR is not used by this leg: free it for the layout's own copy
    b_dev = dp.b
    dp.rowptr = dp.col = dp.val = None
    torch.cuda.empty_cache()
    h = wl.hierarchy(prec)

    def step():
        wl.lay.operator_from_host_csr(p.stencil, p.dofs_per_node, hp["rowptr"], hp["col"],
                                      hp["val"])
        b_dev.copy_(hp["b"], non_blocking=True)
        h.setup_numeric()
        wl.x.zero_()
        res = h.pcg(b_dev, wl.x, rtol=RTOL, maxit=500, history=False)
        hx.copy_(wl.x, non_blocking=True)
        return res

    ms, infos, _ = B.timed(step, K, W_, None)
    h.close()
    ncyc = infos[-1]["vcycles"]
    return {"value": job_value(p.n_unknowns * ncyc * K, B.world, ms), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": ms / K, "api": "rmg_operator_from_host_csr + rmg_setup_numeric + "
                                          "rmg_pcg_solve, host buffers page-locked"}


def learned_leg(B, wl, family, n_train, K, W_, prec="fp32"):
    """The learned prolongator on a workload: train on n_train seeded operators of `family`
    (labelled by the plain method's two-grid error reduction, outside the timed region), then
    time steps with three level-0 transfers: plain (linear interpolation), learned everywhere
    (the network's weights at every node), and per-region acceptance (learned weights kept
    where a region's energy reduction is no worse than linear, linear elsewhere; the plain
    prolongator if the blend is globally worse). Inside a timed learned step the network
    predicts the weights from the freshly split operator before the numeric setup."""
    import numpy as np
    from paper_2103_11962_gb300 import learned
    torch = B.torch
    t0 = time.perf_counter()
    F, Y, M, factors = learned.training_set(B.ctx, range(n_train), training_family(family),
                                            device=B.dev, batch=50)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    net, hist = learned.train(B.ctx, F, Y, M, steps=8000, batch=16384, lr=2e-3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    out = {"family": family, "train_operators": n_train, "samples": int(F.shape[0]),
           "teacher_better_fraction": float(np.mean(factors[:, 1] < factors[:, 0])),
           "label_s": t1 - t0, "train_s": t2 - t1, "loss_first": float(hist[0]),
           "loss_last": float(hist[-1])}
    del F, Y, M
    p = wl.p
    n_r = p.n_regional_nodes
    h = wl.hierarchy(prec)
    wr = torch.empty(3 * n_r, dtype=torch.float32, device=B.dev)
    mixed = torch.empty_like(wr)

    def run(kind, accept=None):
        def step():
            wl.set_operator()
            if kind == "plain":
                h.set_transfer_weights(0, None)
            elif kind == "teacher":
                h.opdep_weights(0, wr)
                h.set_transfer_weights(0, wr)
            else:
                h.mlp_weights(0, net, wr)
                if kind == "per_region":
                    h.blend_weights(0, accept, wr, mixed)
                    h.set_transfer_weights(0, mixed)
                else:
                    h.set_transfer_weights(0, wr)
            h.setup_numeric()
            wl.x.zero_()
            return h.pcg(wl.dp.b, wl.x, rtol=RTOL, maxit=500, history=False)
        ms, infos, _ = B.timed(step, K, W_, wl.flush)
        i = infos[-1]
        return {"ms_per_step": ms / K, "pcg_iterations": i["iterations"],
                "true_relres": i["true_relres"], "converged": i["converged"],
                "value": job_value(p.n_unknowns * i["vcycles"] * K, B.world, ms)}

    out["plain"] = run("plain")
    out["plain"]["factor"] = h.convergence_factor(6, 7)
    out["teacher"] = run("teacher")
    out["teacher"]["factor"] = h.convergence_factor(6, 7)
    out["learned_all"] = run("learned_all")
    out["learned_all"]["factor"] = h.convergence_factor(6, 7)
    h.mlp_weights(0, net, wr)
    acc = learned.accept_per_region(h, wr, n_r, device=B.dev)
    if acc["accepted"]:
        # the region decisions of the acceptance run, reapplied in every timed step
        out["per_region"] = run("per_region", acc["accept"])
    else:
        out["per_region"] = dict(out["plain"], note="no region kept the learned weights, or the "
                                                    "blend was globally worse: plain prolongator")
    out["per_region"].update(regions=acc["regions"], regions_accepted=acc["regions_accepted"],
                             colour_classes=acc["colours"],
                             factor=acc["factor"], factor_candidate=acc["factor_candidate"],
                             factor_blended=acc["factor_blended"])
    fp = out["plain"]["ms_per_step"]
    for k in ("teacher", "learned_all", "per_region"):
        out[k]["speedup_vs_plain"] = fp / out[k]["ms_per_step"]
    h.close()
    net.close()
    return out


def variant_errors_vs_oracle(B, x_oracle_path, sample_key):
    """||x - x_oracle|| / ||x_oracle|| of every precision on the oracle's sample (the sample the
    CPU baseline solved), and on the 4x4x4-region C3 slice against the stored oracle solution
    at sampled nodes (tests/golden/c3_slice_oracle.txt)."""
    import numpy as np
    import workloads as W
    from paper_2103_11962_gb300 import upload
    torch, rmg = B.torch, B.rmg
    out = {}
    if x_oracle_path and os.path.exists(x_oracle_path):
        x_or = np.load(x_oracle_path)
        p = eval(ORACLE_SAMPLES[sample_key][0], {"W": W})
        dp = upload(p, B.dev)
        lay = rmg.Layout(B.ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
        lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)
        x = torch.zeros(p.n, dtype=torch.float64, device=B.dev)
        rec = {"sample": ORACLE_SAMPLES[sample_key][2], "norm": "2-norm over all unknowns"}
        for prec in ("fp64", "fp32", "bf16"):
            h = rmg.Hierarchy(lay, B.options(HEADLINE, prec))
            x.zero_()
            res = h.pcg(dp.b, x, rtol=RTOL, maxit=500, history=False)
            err = float(np.linalg.norm(x.cpu().numpy() - x_or) / np.linalg.norm(x_or))
            rec[prec] = dict(err_vs_oracle=err, pcg_iterations=res["iterations"],
                             true_relres=res["true_relres"])
            h.close()
        lay.close()
        out["sample_2x2x2"] = rec
    gold = os.path.join(ROOT, "tests", "golden", "c3_slice_oracle.txt")
    if os.path.exists(gold):
        hdr, ids, vals = {}, [], []
        for ln in open(gold):
            if ln.startswith("#"):
                continue
            f = ln.split()
            if f[0].isdigit():
                ids.append(int(f[0])); vals.append(float(f[1]))
            else:
                hdr[f[0]] = f[1:]
        ids, vals = np.asarray(ids), np.asarray(vals)
        norm2, nfree = float(hdr["norm2"][0]), int(hdr["unknowns"][0])
        wl = Workload(B, "c3_q1laplace3d_slice")
        rec = {"sample": "4x4x4-region C3 slice (217^3 composite nodes); oracle solution stored "
                         f"at {ids.size} sampled unknowns with its full 2-norm",
               "norm": "sampled RMS difference / RMS of the oracle solution over all unknowns",
               "oracle_iterations": int(hdr["iterations"][0])}
        for prec in ("fp64", "fp32", "bf16"):
            h = wl.hierarchy(prec)
            res = wl.step(h)
            xs = wl.x[torch.from_numpy(ids).to(B.dev)].cpu().numpy()
            rms_diff = float(np.sqrt(np.mean((xs - vals) ** 2)))
            rec[prec] = dict(err_vs_oracle=rms_diff / (norm2 / np.sqrt(nfree)),
                             max_abs_diff_sampled=float(np.abs(xs - vals).max()),
                             pcg_iterations=res["iterations"], true_relres=res["true_relres"])
            h.close()
        wl.close()
        out["slice_4x4x4"] = rec
    return out


def cpu_baseline_leg(workload, small_sample=False, save_x=None):
    """The oracle as it stands on the host cores: one single-threaded process, then one
    process per core (up to 16) on independent copies of the same bounded sample."""
    info = host_info()
    key = oracle_sample_key(workload, small_sample)
    one = run_oracle_sample(key, save_x)
    procs = oracle_procs(info)
    multi = run_oracle_parallel(key, procs) if procs > 1 else None
    best = multi if multi else dict(value=one["value"], procs=1)
    return {"value": best["value"], "unit": UNIT, "cores": best["procs"], "kind": "oracle",
            "sample": one["sample"] + (f"; {best['procs']} independent copies in parallel "
                                       "single-threaded processes" if multi else ""),
            "nproc": info["nproc"], "cpu_model": info["cpu_model"], "threads_per_process": 1,
            "single_thread": {"value": one["value"], "seconds": one["seconds"],
                              "iterations": one["iterations"], "vcycles": one["vcycles"],
                              "unknowns": one["unknowns"]},
            "multi_core": ({"value": multi["value"], "procs": multi["procs"],
                            "seconds_slowest_copy": multi["seconds"]} if multi else None)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=HEADLINE, choices=list(WORKLOADS))
    ap.add_argument("--configs", default="all",
                    help="sub-records measured after the headline: all, none, or a comma list")
    ap.add_argument("--sub-steps", type=int, default=5)
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--smoother", default=None, choices=["jacobi", "chebyshev", "gs"],
                    help="override the workload's smoother (gs: region Gauss-Seidel, "
                         "Algorithm 1, nu 1/1, omega 1)")
    ap.add_argument("--tile-shape", type=int, default=-1,
                    help="stencil-sweep tile shape (rmg_options.tile_shape; -1 autotunes)")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-oracle-errors", action="store_true")
    ap.add_argument("--train-operators", type=int, default=2000)
    ap.add_argument("--json-out", default=None, help="also write the JSON line to this file")
    ap.add_argument("--rap-table", action="store_true",
                    help="time the Galerkin triple product alone on the single-region 2D "
                         "9-point meshes of the paper's Table 4 (constant, linear and generic "
                         "stored transfers) and print that table as the JSON line")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        reference_arm(args)
        return
    if args.rap_table:
        if rank == 0:
            rap_table(args)
        return

    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B = Bench(args, rank, world, local_rank, dist)
    name = args.workload
    precs = precisions_of(args)

    # ---- headline workload, every precision, clocks sampled over the timed steps
    wl = Workload(B, name)
    clocks = ClockSampler(local_rank)
    clocks.start()
    recs = measure_all(B, wl, precs, args.steps, args.warmup)
    clk = clocks.stop()
    head = recs[args.precision]
    out = {
        "metric": METRIC,
        "value": head["value"],
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32 cycle + f64 CG", "bf16": "f32/bf16 cycle + f64 CG"}[args.precision],
        "data": "synthetic",
        "config": workload_config(name),
        "problem": dict(wl.problem_info(), precision=args.precision,
                        parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
        "time_to_tol_s": head["ms_per_step"] / 1e3,
        "pcg_iterations": head["pcg_iterations"],
        "vcycles_per_step": head["vcycles_per_step"],
        "true_relres": head["true_relres"],
        "breakdown": head.get("breakdown"),
        "gpu_launches": head["gpu_launches"],
        "roofline": head["roofline"],
        "clocks": clk,
        "precisions": {k: v for k, v in recs.items() if k != args.precision},
        "speedup_vs_plain_fp64": head.get("speedup_vs_fp64"),
    }
    if not args.no_e2e:
        try:
            out["e2e"] = e2e_leg(B, wl, args.precision, args.steps, args.warmup)
        except Exception as ex:          # reported, not required
            out["e2e"] = {"value": None, "unit": UNIT, "error": f"{type(ex).__name__}: {ex}"[:300]}
    wl.close()

    # ---- the other workloads as sub-records (all precisions, fewer steps)
    subs = [] if args.configs == "none" else (
        [s for s in SUBRECORDS if s != name] if args.configs == "all" else
        [s for s in args.configs.split(",") if s and s != name])
    if subs:
        out["configs"] = {}
        for sname in subs:
            try:
                swl = Workload(B, sname)
                srecs = measure_all(B, swl, precs, args.sub_steps, max(3, args.warmup))
                out["configs"][sname] = {"config": workload_config(sname),
                                         "problem": swl.problem_info(),
                                         "steps": args.sub_steps, "warmup": max(3, args.warmup),
                                         "precisions": srecs}
                if sname.startswith("c4") and not args.no_learned:
                    try:
                        out["configs"][sname]["learned"] = learned_leg(
                            B, swl, "c4", args.train_operators, args.sub_steps,
                            max(3, args.warmup))
                    except Exception as ex:
                        out["configs"][sname]["learned"] = {"error": f"{type(ex).__name__}: {ex}"[:300]}
                swl.close()
                if sname.startswith("c4") and not args.no_learned:
                    # held out: jumps off the coarse planes, where the teacher beats linear
                    # interpolation (on C4 the jumps sit on coarse planes and it cannot)
                    try:
                        hwl = Workload(B, "offset_heldout")
                        out["configs"][sname]["learned_held_out"] = dict(
                            learned_leg(B, hwl, "offset", args.train_operators // 4,
                                        args.sub_steps, max(3, args.warmup)),
                            config=workload_config("offset_heldout"),
                            problem=hwl.problem_info())
                        hwl.close()
                    except Exception as ex:
                        out["configs"][sname]["learned_held_out"] = {
                            "error": f"{type(ex).__name__}: {ex}"[:300]}
            except Exception as ex:
                out["configs"][sname] = {"error": f"{type(ex).__name__}: {ex}"[:300]}

    # ---- the oracle on the host cores, and every precision's error against it
    if rank == 0 and world == 1 and not args.no_cpu:
        xpath = os.path.join(tempfile.gettempdir(), f"rmg_oracle_x_{os.getpid()}.npy")
        try:
            out["cpu_baseline"] = cpu_baseline_leg(name, save_x=xpath)
        except Exception as ex:  # the baseline is reported, not required
            out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": f"failed: {ex}"[:300]}
        if name.startswith("c3") and not args.no_oracle_errors:
            try:
                out["precision_errors_vs_oracle"] = variant_errors_vs_oracle(
                    B, xpath, oracle_sample_key(name))
            except Exception as ex:
                out["precision_errors_vs_oracle"] = {"error": f"{type(ex).__name__}: {ex}"[:300]}
        if os.path.exists(xpath):
            os.remove(xpath)
    if rank == 0:
        print(json.dumps(out))
        if args.json_out:
            with open(args.json_out, "w") as f:
                f.write(json.dumps(out) + "\n")
    if dist:
        dist.destroy_process_group()


# The paper's Table 4 (serial CPU seconds, Trilinos/MueLu vs its structured kernels), as context.
PAPER_TABLE4 = {(140, 36): dict(muelu_9pt=.0024, const=.0001, muelu_25pt=.0109, generic=.0012,
                                geo=.0009),
                (140, 180): dict(muelu_9pt=.0124, const=.0006, muelu_25pt=.0572, generic=.0061,
                                 geo=.0046),
                (700, 180): dict(muelu_9pt=.0726, const=.0070, muelu_25pt=.2944, generic=.0320,
                                 geo=.0240),
                (700, 900): dict(muelu_9pt=.3702, const=.0356, muelu_25pt=1.4786,
                                 generic=.1606, geo=.1208)}


def rap_table(args):
    """Galerkin triple product [[R]][[A]][[P]] alone (rmg_hier_galerkin, FP64, CUDA events) on
    one region of (3 nx - 2) x (3 ny - 2) nodes with the 2D Q1 9-point operator, for the coarse
    meshes of Table 4: piecewise-constant (Const), linear (Geo, implicit weights) and generic
    stored per-node weights (Generic)."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2103_11962_gb300 import rmg, upload
    dev = "cuda:0"
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream(0)
    ctx = rmg.Context(0, stream.cuda_stream)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    rows = []
    for (cx, cy), paper in PAPER_TABLE4.items():
        p = W.q1_laplace2d_box(3 * cx - 2, 3 * cy - 2, rhs=False)
        dp = upload(p, dev, with_rhs=False)
        lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
        lay.operator_from_csr(9, dp.rowptr, dp.col, dp.val)
        h = rmg.Hierarchy(lay, rmg.default_options(levels=2))
        n_r = p.n_regional_nodes
        wr = torch.empty(3 * n_r, dtype=torch.float32, device=dev)
        row = {"coarse_mesh": f"{cx}x{cy}", "fine_mesh": f"{3 * cx - 2}x{3 * cy - 2}"}
        for kind in ("const", "geo", "generic"):
            if kind == "geo":
                h.set_transfer_weights(0, None)
            elif kind == "const":
                h.constant_weights(0, wr)
                h.set_transfer_weights(0, wr)
            else:
                g = np.random.default_rng(11).uniform(0.05, 0.95, 3 * n_r).astype(np.float32)
                wr.copy_(torch.from_numpy(g))
                h.set_transfer_weights(0, wr)
            h.setup_numeric()
            for _ in range(2):
                h.galerkin(0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            # most of these operators fit in L2: flush it before each timed product
            reps, ms = 10, 0.0
            for _ in range(reps):
                flush.fill_(1)
                e0.record(stream)
                h.galerkin(0)
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
            ms /= reps
            row[f"{kind}_ms"] = round(ms, 4)
            row[f"{kind}_speedup_vs_paper_structured"] = round(paper[kind] * 1e3 / ms, 1)
        row["paper_cpu_serial_s"] = paper
        rows.append(row)
        h.close()
        lay.close()
        del dp
        torch.cuda.empty_cache()
    out = {"metric": "Galerkin triple product time, 2D 9-point operator, one region "
                     "(the meshes of the paper's Table 4)",
           "unit": "ms", "higher_is_better": False, "dtype": "f64", "data": "synthetic",
           "l2": "flushed before each timed product", "rows": rows,
           "note": "Const and Generic run the stored-weight kernels, Geo the implicit linear "
                   "weights; the paper's times are serial CPU (Trilinos/MueLu and its structured "
                   "kernels), context only"}
    print(json.dumps(out))
    if args.json_out:
        with open(args.json_out, "w") as f:
            f.write(json.dumps(out) + "\n")


def reference_arm(args):
    """The CPU oracle as it stands, timed on the host cores: every step runs one process per
    core (up to 16) on independent copies of a bounded sample of the workload, single-threaded
    each; the step's time is its slowest copy."""
    name = args.workload
    info = host_info()
    key = oracle_sample_key(name, small=True)
    procs = oracle_procs(info)
    for _ in range(args.warmup):
        run_oracle_parallel(key, procs)
    t0 = time.perf_counter()
    steps = [run_oracle_parallel(key, procs) for _ in range(args.steps)]
    t1 = time.perf_counter()
    units = sum(s["value"] * s["seconds"] for s in steps)
    value = units / sum(s["seconds"] for s in steps)
    sample = steps[-1]["sample"] + f"; {procs} independent copies in parallel single-threaded " \
                                   "processes per step"
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": (t1 - t0) * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": workload_config(name),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                            "sample": sample, "nproc": info["nproc"],
                            "cpu_model": info["cpu_model"], "threads_per_process": 1},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
