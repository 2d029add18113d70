"""Benchmark: region multigrid preconditioned CG to a 1e-10 relative residual.

One step = one linear system solved from device-resident inputs through the C ABI:
non-invasive split of the composite CSR matrix into region stencils, numeric hierarchy setup
(diagonals, regional Galerkin products, Chebyshev power method, coarsest Cholesky and inverse)
and PCG with one regional V-cycle per iteration. The mesh (region layout, interface groups)
and the hierarchy's buffers and CUDA graph are built once before timing.

The headline path (--precision fp32, the default) runs the V-cycle in FP32 inside FP64 flexible
CG; the plain FP64 method and the BF16-coefficient cycle are measured beside it on the same
system, all to the same 1e-10 relative FP64 residual.

Metric: V-cycle DOF/s = unknowns x V-cycles of the step / step time (whole step, setup
included), and the time to the 1e-10 relative residual.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
       [--workload c2_diffusion3d] [--precision fp32|fp64|bf16] [--no-mixed] [--no-e2e] [--no-cpu]
Under torchrun every rank solves its own copy of the system (independent problems, no
collective on the data path; weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "V-cycle DOF/s & time to 1e-10 rel. residual, mixed/learned vs plain FP64"
RTOL = 1e-10

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

WORKLOADS = {
    "c2_diffusion3d": dict(levels=4, smoother="chebyshev", nu1=1, nu2=1, degree=3,
                           desc="3D 7-point variable-coefficient diffusion, 8x8x4 regions with "
                                "per-axis node counts from {28,55,82} (seed 1), log-normal "
                                "per-element kappa (sigma 1), Chebyshev degree 3, 4 levels"),
    "c2_quarter": dict(levels=4, smoother="chebyshev", nu1=1, nu2=1, degree=3,
                       desc="C2-shaped 3D 7-point diffusion on 4x4x2 regions (profiling size)"),
    "c5_elasticity": dict(levels=4, smoother="chebyshev", nu1=1, nu2=1, degree=3, power_iters=30,
                          desc="3D linear elasticity, Q1 hexahedra, 3 dofs per node (81-coefficient "
                               "block rows), 3x3x3 regions of 28^3 nodes (the paper's 82^3 "
                               "elasticity mesh), E log-normal (sigma 0.5), nu 0.3, x=0 clamped, "
                               "uniform body load; 30 power steps: 10 underestimate "
                               "lambda_max(D^-1 A) by ~25% on this operator"),
    "c5_elasticity_4x4x4": dict(levels=4, smoother="chebyshev", nu1=1, nu2=1, degree=3,
                                power_iters=30,
                                desc="3D linear elasticity as c5_elasticity on 4x4x4 regions of 28^3"),
    "c3_q1laplace3d": dict(levels=4, smoother="chebyshev", nu1=1, nu2=1, degree=3,
                           desc="3D Q1 Laplacian (27-point), 8x8x8 regions of 55^3 nodes (433^3 "
                                "composite, 81M unknowns, 2.2G nonzeros; CSR assembled on the "
                                "device by the workload generator), rhs seed 2"),
    "c5_elasticity_full": dict(levels=4, smoother="chebyshev", nu1=1, nu2=1, degree=3,
                               power_iters=30,
                               desc="3D linear elasticity, 8x8x8 regions with per-axis node counts "
                                    "from {28,55} (seed 95, the first seed from 4 on giving "
                                    "60M +- 15% dofs: 271x271x244 nodes, 53.8M dofs, 4.4G "
                                    "nonzeros; CSR assembled on the device), E log-normal "
                                    "(sigma 0.5), nu 0.3, x=0 clamped, uniform body load"),
    "c3_q1laplace3d_slice": dict(levels=4, smoother="chebyshev", nu1=1, nu2=1, degree=3,
                                 desc="3D Q1 Laplacian (27-point), 4x4x4 regions of 55^3 nodes "
                                      "(the 4x4x4-region slice of the 8x8x8 configuration)"),
    "c4_highcontrast3d": dict(levels=4, smoother="chebyshev", nu1=1, nu2=1, degree=3,
                              desc="3D 7-point diffusion, 7x7x7 regions with per-axis node counts "
                                   "from {28,55,82} (seed 3), kappa constant per region, "
                                   "log-uniform in [1e-3, 1e3]"),
    "c1_poisson2d": dict(levels=4, smoother="jacobi", nu1=2, nu2=2, omega=0.67,
                         desc="2D Poisson 5-point, 2x2 regions of 82x82, Jacobi 0.67, nu 2/2, "
                              "4 levels"),
}


def training_family(workload):
    """Seeded small operators the learned prolongator is trained on (same PDE family)."""
    import workloads as W
    if workload.startswith("c4"):
        return lambda s: W.highcontrast3d_7pt(region_grid=(2, 2, 2), choices=(10,), seed=1000 + s)
    return lambda s: W.diffusion3d_7pt(region_grid=(2, 2, 2), choices=(10, 19, 28), seed=2000 + s)


def profiled_traffic(prec):
    """DRAM bytes per regional node of the timed sweep from the committed ncu summary, or None
    when the kernel sources changed since that capture."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "k_stencil7_cheb_c2quarter.md")
    if not os.path.exists(prof):
        return None
    h = hashlib.sha256()
    for f in ("rmg_internal.cuh", "rmg_kernels.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2103_11962_gb300", "csrc", f), "rb").read())
    text = open(prof).read()
    if f"kernel_source_sha256_16: {h.hexdigest()[:16]}" not in text:
        return None
    key = {"fp64": "fp64", "fp32": "fp32"}.get(prec)
    for line in text.splitlines():
        if key and line.startswith(f"{key}_dram_bytes_per_node:"):
            return float(line.split(":")[1])
    return None


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


# ------------------------------------------------------------------------------ oracle leg
def oracle_sample_cmd(workload, seconds_budget=20.0):
    """Command that runs the CPU oracle pipeline (split, hierarchy, PCG to 1e-10) on a bounded
    sample of the workload and prints a JSON summary. Single-threaded BLAS."""
    code = f"""
import json, os, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
import workloads as W
from oracle import cycle, hierarchy, krylov
w = {workload!r}
cheb = cycle.Options(smoother='chebyshev', nu1=1, nu2=1, degree=3)
block = False
if w in ('c2_diffusion3d', 'c2_quarter'):
    p = W.diffusion3d_7pt(region_grid=(2, 2, 2), choices=(28, 55, 82), seed=1)
    o = cheb
    sample = 'C2-shaped 2x2x2-region instance (slabs from {{28,55,82}}, seed 1, log-normal kappa)'
elif w.startswith('c3'):
    p = W.q1_laplace3d(region_grid=(2, 2, 2), n=28, seed=2)
    o = cheb
    sample = 'C3-shaped 2x2x2-region Q1 instance (28^3 regions, seed 2)'
elif w.startswith('c4'):
    p = W.highcontrast3d_7pt(region_grid=(2, 2, 2), choices=(28, 55, 82), seed=3)
    o = cheb
    sample = 'C4-shaped 2x2x2-region high-contrast instance (slabs from {{28,55,82}}, seed 3)'
elif w.startswith('c5'):
    p = W.elasticity3d(region_grid=(2, 2, 2), choices=(10, 19), seed=4)
    o = cycle.Options(smoother='chebyshev', nu1=1, nu2=1, degree=3, power_iters=30)
    block = True
    sample = 'C5-shaped 2x2x2-region elasticity instance (slabs from {{10,19}}, seed 4)'
else:
    p = W.config('c1_poisson2d')
    o = cycle.Options(smoother='jacobi', nu1=2, nu2=2, omega=0.67)
    sample = 'full C1 workload'
t0 = time.perf_counter()
if block:
    levels = hierarchy.build_block(p, 3)
    perm = hierarchy.node_major_to_component_major(p.n_nodes, p.dofs_per_node)
    A, b = levels[0].A, p.b[perm]
else:
    levels = hierarchy.build(p, 4)
    A, b = p.A, p.b
mg = cycle.RegionalMG(levels, o)
x, it, hist = krylov.pcg(A, b, krylov.regional_preconditioner(mg), rtol={RTOL})
t1 = time.perf_counter()
ncyc = it if hist[-1] <= {RTOL} else it + 1
print(json.dumps(dict(seconds=t1 - t0, iterations=it, vcycles=ncyc, unknowns=p.n_unknowns,
                      n_regional=p.n_regional_nodes, sample=sample)))
"""
    return [sys.executable, "-c", code]


def run_oracle_sample(workload):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    res = subprocess.run(oracle_sample_cmd(workload), capture_output=True, text=True, env=env,
                         timeout=900)
    if res.returncode != 0:
        raise RuntimeError(res.stderr[-2000:])
    d = json.loads(res.stdout.strip().splitlines()[-1])
    d["value"] = d["unknowns"] * d["vcycles"] / d["seconds"]
    return d


# ------------------------------------------------------------------------------ native leg
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="c2_diffusion3d", choices=list(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--smoother", default=None, choices=["jacobi", "chebyshev", "gs"],
                    help="override the workload's smoother (gs: region Gauss-Seidel, "
                         "Algorithm 1, nu 1/1, omega 1)")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--train-operators", type=int, default=40)
    ap.add_argument("--json-out", default=None, help="also write the JSON line to this file")
    ap.add_argument("--rap-table", action="store_true",
                    help="time the Galerkin triple product alone on the single-region 2D "
                         "9-point meshes of the paper's Table 4 (constant, linear and generic "
                         "stored transfers) and print that table as the JSON line")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    cfg = WORKLOADS[args.workload]

    if args.impl == "reference":
        if rank != 0:
            return
        reference_arm(args, cfg)
        return
    if args.rap_table:
        if rank == 0:
            rap_table(args)
        return

    import numpy as np
    import torch

    import workloads as W
    from paper_2103_11962_gb300 import rmg, upload

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = f"cuda:{local_rank}"

    if args.workload == "c2_quarter":
        p = W.diffusion3d_7pt(region_grid=(4, 4, 2), choices=(28, 55, 82), seed=1)
    elif args.workload == "c4_highcontrast3d":
        p = W.config("c4_highcontrast3d")
    elif args.workload == "c5_elasticity":
        p = W.elasticity3d(region_grid=(3, 3, 3), choices=(28,), seed=4)
    elif args.workload == "c5_elasticity_4x4x4":
        p = W.elasticity3d(region_grid=(4, 4, 4), choices=(28,), seed=4)
    elif args.workload == "c3_q1laplace3d_slice":
        p = W.q1_laplace3d(region_grid=(4, 4, 4), n=55, seed=2)
    elif args.workload == "c3_q1laplace3d":
        from workloads import device as WD
        p = WD.q1_laplace3d(region_grid=(8, 8, 8), n=55, seed=2, device=dev)
    elif args.workload == "c5_elasticity_full":
        from workloads import device as WD
        p = WD.elasticity3d(region_grid=(8, 8, 8), choices=(28, 55), seed=95, device=dev)
    else:
        p = W.config(args.workload)
    dp = device_problem(p, dev)
    stream = torch.cuda.current_stream(local_rank)
    ctx = rmg.Context(local_rank, stream.cuda_stream)
    t_lay = time.perf_counter()
    lay = rmg.Layout(ctx, p.dim, p.region_dims, dp.gids, p.n_nodes, dp.dirichlet)
    t_lay = time.perf_counter() - t_lay

    def options(prec):
        o = rmg.default_options(levels=cfg["levels"], precision={"fp64": rmg.FP64,
                                                                "fp32": rmg.FP32,
                                                                "bf16": rmg.FP32_BF16COEF}[prec])
        sm = args.smoother or cfg["smoother"]
        if sm == "chebyshev":
            o.smoother, o.nu1, o.nu2, o.cheb_degree = (rmg.CHEBYSHEV, cfg["nu1"], cfg["nu2"],
                                                        cfg.get("degree", 3))
        elif sm == "gs":
            o.smoother, o.nu1, o.nu2, o.omega = rmg.GAUSS_SEIDEL, 1, 1, 1.0
        else:
            o.smoother, o.nu1, o.nu2, o.omega = (rmg.JACOBI, cfg["nu1"], cfg["nu2"],
                                                 cfg.get("omega", 0.67))
        o.power_iters = cfg.get("power_iters", 10)
        return o

    def set_operator():
        if p.dofs_per_node > 1:
            lay.operator_from_block_csr(p.stencil, p.dofs_per_node, dp.rowptr, dp.col, dp.val)
        else:
            lay.operator_from_csr(p.stencil, dp.rowptr, dp.col, dp.val)

    set_operator()
    hier = rmg.Hierarchy(lay, options(args.precision))
    x = torch.zeros(p.n, dtype=torch.float64, device=dev)
    flush = l2_flush_buffer(dp, dev)

    def step(h):
        set_operator()
        h.setup_numeric()
        x.zero_()
        return h.pcg(dp.b, x, rtol=RTOL, maxit=500, history=False)

    def timed(h, K, W_, e2e=None):
        for _ in range(W_):
            (e2e or step)(h)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        h.probe(reset=True)
        l0 = rmg.launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if flush is None:
            ev0.record(stream)
            infos = [(e2e or step)(h) for _ in range(K)]
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
        else:
            # inputs within L2: the flush write runs between the timed intervals
            infos, ms = [], 0.0
            for _ in range(K):
                flush.fill_(1)
                ev0.record(stream)
                infos.append((e2e or step)(h))
                ev1.record(stream)
                torch.cuda.synchronize()
                ms += ev0.elapsed_time(ev1)
        launches = rmg.launch_count() - l0
        ms = max_over_ranks(ms, dist, dev)
        return ms, infos, launches, h.probe(reset=True)

    clocks = ClockSampler(local_rank)
    clocks.start()
    ms, infos, launches, (probe_ms, probe_n) = timed(hier, args.steps, args.warmup)
    clk = clocks.stop()
    ms_step = ms / args.steps
    info = infos[-1]
    ncyc = info["vcycles"]
    value = job_value(p.n_unknowns * ncyc * args.steps, world, ms)

    # per-phase breakdown of one step (outside the timed region)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream); set_operator()
    e[1].record(stream); hier.setup_numeric()
    e[2].record(stream); x.zero_(); bi = hier.pcg(dp.b, x, rtol=RTOL, maxit=500, history=False)
    e[3].record(stream); torch.cuda.synchronize()
    breakdown = dict(split_ms=e[0].elapsed_time(e[1]), setup_ms=e[1].elapsed_time(e[2]),
                     solve_ms=e[2].elapsed_time(e[3]), layout_ms_once=t_lay * 1e3,
                     vcycle_launches=hier.vcycle_launches(),
                     tile_shapes=[list(hier.tile_shape(l)) for l in range(cfg["levels"])])
    # V-cycle alone (graph replays), for the per-cycle figure
    r = dp.b.clone()
    z = torch.empty_like(r)
    for _ in range(3):
        hier.vcycle(r, z)
    torch.cuda.synchronize()
    e[0].record(stream)
    nrep = 20
    for _ in range(nrep):
        hier.vcycle(r, z)
    e[1].record(stream); torch.cuda.synchronize()
    vc_ms = e[0].elapsed_time(e[1]) / nrep
    breakdown["vcycle_ms"] = vc_ms
    breakdown["vcycle_dof_per_s"] = p.n_unknowns / (vc_ms / 1e3)

    pk = peaks()
    kern_ms = probe_ms / max(1, probe_n)
    n_r0 = p.n_regional_nodes
    prec = args.precision
    Bd = p.dofs_per_node
    planes0 = hier.coef_planes(0)
    bytes_launch = sweep_bytes(prec, planes0, Bd) * n_r0
    flops_launch = sweep_flops(p.stencil, Bd) * n_r0
    roofline = None
    if bytes_launch and kern_ms > 0:
        gbs = bytes_launch / (kern_ms / 1e3) / 1e9
        tfl = flops_launch / (kern_ms / 1e3) / 1e12
        hbm_frac = gbs / pk["hbm_gbs"]
        alu_frac = tfl / pk["fp64_tflops"] if prec == "fp64" else 0.0
        if prec == "fp64" and alu_frac > hbm_frac:
            roofline = dict(bound="alu", achieved=round(tfl, 4), peak=round(pk["fp64_tflops"], 4),
                            unit="TFLOP/s (FP64)", frac=round(alu_frac, 4),
                            hbm=dict(achieved=round(gbs, 1), peak=pk["hbm_gbs"],
                                     unit="GB/s", frac=round(hbm_frac, 4),
                                     peak_src=pk["src"]),
                            peak_src="derived: 152 SM x 2 DFMA/clk x 2 flop x max SM clock")
        else:
            roofline = dict(bound="hbm", achieved=round(gbs, 1), peak=pk["hbm_gbs"], unit="GB/s",
                            frac=round(hbm_frac, 4), peak_src=pk["src"])
        tpn = profiled_traffic(prec)
        tpn = tpn if (p.stencil == 7 and Bd == 1) else None
        kname = ("k_bstencil<{}, {}, EpiCheb>".format(p.stencil, Bd) if Bd > 1 else
                 "k_stencil_half<{}, EpiCheb>".format(p.stencil) if planes0 < p.stencil else
                 "k_stencil<{}, EpiCheb>".format(p.stencil))
        roofline.update(kernel=f"{kname} level 0 ({prec}, {planes0} coefficients per node)",
                        traffic=(round(tpn * n_r0) if tpn else None),
                        traffic_src=("ncu dram__bytes per node (profiles/k_stencil7_cheb_c2quarter.md)"
                                     " x regional nodes" if tpn else None),
                        ms_per_launch=round(kern_ms, 4),
                        launches_timed=probe_n, bytes_per_launch=bytes_launch,
                        flops_per_launch=flops_launch)

    out = {
        "metric": METRIC,
        "value": value,
        "unit": "DOF*V-cycles/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32 cycle + f64 CG", "bf16": "f32/bf16 cycle + f64 CG"}[prec],
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": cfg["desc"],
                   "smoother": args.smoother or cfg["smoother"],
                   "global_dims": list(p.global_dims), "regions": int(p.nregions),
                   "unknowns": p.n_unknowns, "regional_nodes": p.n_regional_nodes,
                   "composite_nnz": int(p.nnz if hasattr(p, "nnz") else p.A.nnz),
                   "levels": cfg["levels"],
                   "precision": prec, "rtol": RTOL,
                   "dofs_per_node": p.dofs_per_node,
                   "l2": ("L2 flushed between timed steps" if flush is not None else
                          "inputs larger than L2 (no flush needed)"),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "time_to_tol_s": ms_step / 1e3,
        "pcg_iterations": info["iterations"],
        "vcycles_per_step": ncyc,
        "true_relres": info["true_relres"],
        "breakdown": breakdown,
        "gpu_launches": int(launches),
        "roofline": roofline,
        "clocks": clk,
    }

    # the other precisions on the same workload (same 1e-10 FP64 residual): the plain FP64
    # method the headline is compared with, and the remaining mixed variant
    fp64_ms = ms_step if prec == "fp64" else None
    if not args.no_mixed:
        others = {}
        for mp in [q for q in ("fp64", "fp32", "bf16") if q != prec]:
            hm = rmg.Hierarchy(lay, options(mp))
            msm, infm, _, (pms, pn) = timed(hm, args.steps, args.warmup)
            im = infm[-1]
            km = pms / max(1, pn)
            bl = sweep_bytes(mp, hm.coef_planes(0), p.dofs_per_node) * n_r0
            tr = profiled_traffic(mp) if (p.stencil == 7 and p.dofs_per_node == 1) else None
            others[mp] = dict(ms_per_step=msm / args.steps,
                              value=p.n_unknowns * im["vcycles"] * args.steps * world / (msm / 1e3),
                              pcg_iterations=im["iterations"], true_relres=im["true_relres"],
                              kernel_ms=km,
                              kernel_hbm_frac=(bl / (km / 1e3) / 1e9 / pk["hbm_gbs"]) if bl and km else None,
                              kernel_traffic=(round(tr * n_r0) if tr else None))
            if mp == "fp64":
                fp64_ms = msm / args.steps
            hm.close()
        for mp, v in others.items():
            v["speedup_vs_fp64"] = fp64_ms / v["ms_per_step"] if fp64_ms else None
        out["precisions"] = others
    out["speedup_vs_plain_fp64"] = fp64_ms / ms_step if fp64_ms else None

    # learned prolongator: trained offline (outside the timed region) on small operators of the
    # same family labelled by the plain method; inside every timed step the network predicts
    # the level-0 weights from the new operator before the numeric setup
    if not args.no_learned and p.stencil == 7 and p.dofs_per_node == 1:
        from paper_2103_11962_gb300 import learned
        t0 = time.perf_counter()
        F, Y, M, factors = learned.training_set(ctx, range(args.train_operators),
                                                training_family(args.workload), device=dev)
        t1 = time.perf_counter()
        net, hist = learned.train(ctx, F, Y, M, steps=1500, batch=16384, lr=2e-3)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        wr = torch.empty(3 * p.n_regional_nodes, dtype=torch.float32, device=dev)

        def lstep(h):
            set_operator()
            h.mlp_weights(0, net, wr)
            h.set_transfer_weights(0, wr)
            h.setup_numeric()
            x.zero_()
            return h.pcg(dp.b, x, rtol=RTOL, maxit=500, history=False)

        lres = {"train_operators": args.train_operators, "samples": int(F.shape[0]),
                "teacher_better_fraction": float(np.mean(factors[:, 1] < factors[:, 0])),
                "label_s": t1 - t0, "train_s": t2 - t1, "loss_first": float(hist[0]),
                "loss_last": float(hist[-1])}
        del F, Y, M
        for tag in [args.precision] + (["fp64"] if args.precision != "fp64" else ["fp32"]):
            hl = hier if tag == args.precision else rmg.Hierarchy(lay, options(tag))
            acc = learned.apply_learned(hl, net, p.n_regional_nodes, device=dev)
            entry = dict(acc)
            if acc["accepted"]:
                msl, infl, _, _ = timed(hl, args.steps, args.warmup, e2e=lstep)
                il = infl[-1]
                entry.update(ms_per_step=msl / args.steps, pcg_iterations=il["iterations"],
                             true_relres=il["true_relres"],
                             value=p.n_unknowns * il["vcycles"] * args.steps * world / (msl / 1e3),
                             speedup_vs_fp64=(fp64_ms / (msl / args.steps)) if fp64_ms else None)
                hl.set_transfer_weights(0, None)
                hl.setup_numeric()
            lres[tag] = entry
            if hl is not hier:
                hl.close()
        out["learned"] = lres
        net.close()

    # end to end through the C ABI with host buffers: H2D of the step's inputs (composite
    # CSR + right-hand side) from pinned memory, the step, D2H of the solution
    if not args.no_e2e:
        hp = {}
        for k in ("rowptr", "col", "val", "b"):
            t = getattr(dp, k)
            hp[k] = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
            hp[k].copy_(t)
        hx = torch.empty(p.n, dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in hp.values())
        d2h = hx.numel() * hx.element_size()

        def e2e_step(h):
            for k, t in hp.items():
                getattr(dp, k).copy_(t, non_blocking=True)
            res = step(h)
            hx.copy_(x, non_blocking=True)
            return res

        mse, infe, _, _ = timed(hier, args.steps, args.warmup, e2e=e2e_step)
        out["e2e"] = {"value": p.n_unknowns * infe[-1]["vcycles"] * args.steps * world / (mse / 1e3),
                      "unit": "DOF*V-cycles/s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h), "ms_per_step": mse / args.steps}

    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            cb = run_oracle_sample(args.workload)
            out["cpu_baseline"] = {"value": cb["value"], "unit": "DOF*V-cycles/s", "cores": 1,
                                   "kind": "oracle", "sample": cb["sample"],
                                   "seconds": cb["seconds"], "iterations": cb["iterations"],
                                   "unknowns": cb["unknowns"]}
        except Exception as ex:  # the baseline is reported, not required
            out["cpu_baseline"] = {"value": None, "unit": "DOF*V-cycles/s", "cores": 1,
                                   "kind": "oracle", "sample": f"failed: {ex}"[:300]}
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


def reference_arm(args, cfg):
    """The CPU oracle as it stands, timed on the host cores (bounded samples per step)."""
    samples = []
    for _ in range(args.warmup):
        run_oracle_sample(args.workload)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        samples.append(run_oracle_sample(args.workload))
    t1 = time.perf_counter()
    units = sum(s["unknowns"] * s["vcycles"] for s in samples)
    value = units / sum(s["seconds"] for s in samples)
    out = {"metric": METRIC, "value": value, "unit": "DOF*V-cycles/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": (t1 - t0) * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": args.workload, "desc": cfg["desc"],
                      "sample": samples[-1]["sample"]},
           "cpu_baseline": {"value": value, "unit": "DOF*V-cycles/s", "cores": 1,
                            "kind": "oracle", "sample": samples[-1]["sample"]},
           "e2e": {"value": value, "unit": "DOF*V-cycles/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
