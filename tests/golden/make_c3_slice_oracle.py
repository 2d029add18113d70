"""Write c3_slice_oracle.txt: the oracle's solution on the 4x4x4-region slice of the 3D Q1
Laplacian workload (regions of 55^3 nodes, 217^3 composite nodes, right-hand side seed 2).

The oracle (plain FP64 region multigrid: Chebyshev degree 3, nu 1/1, 4 levels, PCG to a
1e-10 relative residual) solves the slice once; the file keeps the 2-norm of the solution
over all composite nodes, the number of unmasked nodes, the iteration count and the solution
at 4096 unmasked composite nodes drawn with numpy default_rng(12345). It calls only oracle/
and the input generator. The slice takes the oracle tens of minutes, which is why its
solution is stored (sampled) rather than recomputed by the tests and the benchmark.

Usage: python tests/golden/make_c3_slice_oracle.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import cycle, hierarchy, krylov  # noqa: E402

NSAMPLES = 4096


def main():
    t0 = time.perf_counter()
    p = W.q1_laplace3d(region_grid=(4, 4, 4), n=55, seed=2)
    levels = hierarchy.build(p, 4)
    mg = cycle.RegionalMG(levels, cycle.Options(smoother="chebyshev", nu1=1, nu2=1, degree=3))
    x, it, hist = krylov.pcg(p.A, p.b, krylov.regional_preconditioner(mg), rtol=1e-10)
    secs = time.perf_counter() - t0
    free = np.flatnonzero(p.dirichlet == 0)
    ids = np.sort(np.random.default_rng(12345).choice(free, NSAMPLES, replace=False))
    with open(os.path.join(HERE, "c3_slice_oracle.txt"), "w") as f:
        f.write("# oracle solution of the 4x4x4-region Q1 slice (55^3 regions, rhs seed 2);\n")
        f.write("# written by tests/golden/make_c3_slice_oracle.py (oracle/ only)\n")
        f.write(f"global_dims {p.global_dims[0]} {p.global_dims[1]} {p.global_dims[2]}\n")
        f.write(f"unknowns {free.size}\n")
        f.write(f"iterations {it}\n")
        f.write(f"final_relres {float(hist[-1])!r}\n")
        f.write(f"norm2 {float(np.linalg.norm(x))!r}\n")
        f.write(f"oracle_seconds {secs:.1f}\n")
        for g in ids:
            f.write(f"{int(g)} {float(x[g])!r}\n")


if __name__ == "__main__":
    main()
