"""Write oracle_velocity_<workload>.txt: the oracle's velocities (sparse
direct solve of the assembled system, then recovery) at a seeded sample of
4,096 live faces of a benchmark workload, with the largest |u| over all live
faces as the scale of relative errors.  Calls only ``oracle`` and the seeded
input generators.

    python tests/golden/make_oracle_velocity_samples.py bumps1024 column256

bumps1024: the 2D 1024^2 Gaussian-bump workload (seed 2), whole system.
column256: the 3D 256^3 falling column on the 34 x 160 x 34-cell window
(cells [111, 145) x [0, 160) x [111, 145)) that holds every liquid unknown;
face indices are those of the window's face fields.  Its system is solved by
the oracle's FP64 Jacobi-PCG to a true relative residual of 1e-13 (a sparse
LU of this 3D system did not finish in hours); the 2D one by sparse LU."""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import solve as So  # noqa: E402
from oracle import system as S_  # noqa: E402
from paper_1010_2832_gb300 import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
COLUMN_WINDOW = (111, 0, 111, 34, 160, 34)
SAMPLES = 4096


def workload(name):
    if name == "bumps1024":
        return W.bumps_2d(1024, seed=2)
    if name == "column256":
        return W.column_3d(256, window=COLUMN_WINDOW)
    raise SystemExit(f"unknown workload {name}")


def main(names):
    for name in names:
        t0 = time.perf_counter()
        wl = workload(name)
        S = S_.build_system(S_.StokesInput(**wl.as_oracle_kwargs()))
        if wl.dim == 3:
            x, it, _ = So.pcg(S.A, S.b, tol=1e-13, max_iter=10 ** 6)
            how = f"FP64 Jacobi-PCG, {it} iterations"
        else:
            x = So.solve_direct(S.A, S.b, S_.pressure_null_vectors(S))
            how = "sparse direct"
        u = S_.recover_velocity(S, x)
        rel = So.relative_residual(S.A, x, S.b)
        live = np.flatnonzero(S.live)
        pick = np.sort(np.random.default_rng(0).choice(live, size=min(SAMPLES, live.size), replace=False))
        scale = float(np.abs(u[live]).max())
        with open(os.path.join(HERE, f"oracle_velocity_{name}.txt"), "w") as f:
            f.write(f"# Oracle velocities of workload {name} at {pick.size} seeded live faces ({how}\n"
                    f"# solve, relative residual {rel:.2e}); faces in field order u, v(, w), each x fastest.\n"
                    f"# Written by: python tests/golden/make_oracle_velocity_samples.py {name}\n"
                    f"# scale (max |u| over {live.size} live faces): {float(scale)!r}\n"
                    "# Columns: face_index velocity\n")
            for i in pick:
                f.write(f"{i} {float(u[i])!r}\n")
        print(name, f"{time.perf_counter() - t0:.1f} s", "rel", rel, "live", live.size, flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["bumps1024", "column256"])
