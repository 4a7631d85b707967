"""Planar viscous jet buckling (Section "Two Dimensional Jet Buckling") with
the fractional-step routine of Section "Application to Viscous Jet
Buckling" at the paper's 150 x 150 resolution, run to 2.7 s (the last frame
of the paper's figure).  The figure is qualitative; the checks are physical:
every Stokes solve converges; the liquid area grows at the inflow rate
D |U|; gravity makes the jet fall faster than the inflow speed and it
reaches the container's bottom (y = 0.1) within 0.5 to 0.8 s; and the jet,
straight and on the axis until well after impact, folds sideways above the
pool (buckling) by the end.  Frames at the figure's times (0.5 s, then every
0.2 s) and the per-step record go to $STOKES_RESULTS_DIR when set."""
import json
import os

import numpy as np
import pytest

from gpu_common import require_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_jet_2d_buckles():
    require_gpu()
    from paper_1010_2832_gb300 import jet, workloads as W
    sim = jet.JetSim(150, dt=0.002)
    out_dir = os.environ.get("STOKES_RESULTS_DIR")
    times = [round(0.5 + 0.2 * k, 2) for k in range(12)]
    sim.run(2.7, snapshot_times=times, out_dir=out_dir)
    H = sim.history
    if out_dir:
        with open(os.path.join(out_dir, "jet150_history.json"), "w") as f:
            json.dump(H, f)
    t = np.array([r["t"] for r in H])
    area = np.array([r["area"] for r in H])
    front = np.array([r["front_y"] for r in H])
    off = np.array([r["jet_offset"] for r in H])
    assert all(r["status"] == 0 and r["rel_residual"] <= 1.01e-8 for r in H)
    J = W.JET2D
    rate = np.polyfit(t[t >= 0.5], area[t >= 0.5], 1)[0]
    assert 0.8 <= rate / (J["width"] * abs(J["U"])) <= 1.2, rate
    y0 = front[0]
    assert front[np.argmin(np.abs(t - 0.5))] < y0 - abs(J["U"]) * 0.5 - 0.05     # faster than the inflow
    impact = t[np.argmax(front <= 0.1 + sim.h)]
    assert front.min() <= 0.1 + sim.h and 0.5 <= impact <= 0.8, impact
    early, late = off[(t >= 0.5) & (t <= 1.2)].max(), off[t >= 2.0].max()
    print(f"area rate {rate:.4f}, impact {impact:.3f} s, jet offset early {early / sim.h:.2f} h, "
          f"late {late / sim.h:.2f} h, median ms/step {np.median([r['ms'] for r in H]):.2f}")
    assert early <= 1.0 * sim.h and late >= 2.0 * sim.h, (early, late)
    sim.close()
