"""Write oracle_pcg_counts.txt: the oracle's own plain FP64 Jacobi-PCG on the
2D Gaussian-bump workload (8 seeded bumps, moving disk r = 0.1, log-uniform
viscosity 1e-2..1e2, density 1 | 1000, dt = 0.01, seed 2) at 256^2, 512^2
and 1024^2, solved to a true relative residual of 1e-8: iterations, wall
time of the build, of the solve and per iteration, the threads numpy's
BLAS pool held, and the CPU.  Calls only ``oracle`` and the seeded input
generators.

    python tests/golden/make_oracle_pcg_counts.py [sizes...]

(1024^2: 135,073 iterations, about 2.8 hours on one 2.7 GHz core.)"""
import os
import platform
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import solve as So  # noqa: E402
from oracle import system as S_  # noqa: E402
from paper_1010_2832_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_pcg_counts.txt")


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return max((i.get("num_threads") or 1) for i in threadpool_info()) if threadpool_info() else 1
    except Exception:
        return None


def main(sizes):
    rows = []
    if os.path.exists(OUT):
        rows = [l.rstrip("\n") for l in open(OUT) if l.strip() and not l.startswith("#")]
    done = {int(r.split()[0]) for r in rows}
    for n in sizes:
        if n in done:
            continue
        t0 = time.perf_counter()
        wl = W.bumps_2d(n, seed=2)
        S = S_.build_system(S_.StokesInput(**wl.as_oracle_kwargs()))
        t_build = time.perf_counter() - t0
        t0 = time.perf_counter()
        x, it, rel = So.pcg(S.A, S.b, tol=1e-8, max_iter=10 ** 7)
        t_solve = time.perf_counter() - t0
        row = (f"{n} {it} {rel:.3e} {t_build:.2f} {t_solve:.1f} {1e3 * t_solve / max(it, 1):.3f} "
               f"{int(S.active.sum())} {blas_threads()}")
        print(row, flush=True)
        # rows written meanwhile by another run of this script are kept
        rows = [l.rstrip("\n") for l in open(OUT) if l.strip() and not l.startswith("#")] \
            if os.path.exists(OUT) else []
        rows = [r for r in rows if int(r.split()[0]) != n] + [row]
        with open(OUT, "w") as f:
            f.write("# The oracle's plain FP64 Jacobi-PCG (oracle.solve.pcg, tol 1e-8 on the true relative\n"
                    "# residual) on the 2D Gaussian-bump workload (workloads.bumps_2d(n, seed=2)).\n"
                    "# Written by: python tests/golden/make_oracle_pcg_counts.py [sizes...] (one row per size;\n"
                    "# rows already in the file are kept)\n"
                    f"# CPU: {cpu_model()}; {os.cpu_count()} cores; numpy {np.__version__}\n"
                    "# Columns: n iterations true_rel_residual build_s solve_s ms_per_iteration active_unknowns "
                    "blas_threads\n")
            f.write("\n".join(sorted(rows, key=lambda r: int(r.split()[0]))) + "\n")


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [256, 512, 1024])
