"""Planar viscous jet buckling (Section "Two Dimensional Jet Buckling") with
the two-stage fractional-step Navier-Stokes routine of Section "Application
to Viscous Jet Buckling":

  1. transport (stokes_advect): extend u^n into fluid faces without liquid,
     u* = semi-Lagrangian advection of u^n + dt g, and advect the liquid level
     set with the same velocity, united with the jet opening (the inflow);
  2. weights of the new geometry (stokes_build_weights);
  3. one implicit Stokes step from u* (stokes_solve_step) gives u^{n+1}.

Every stage runs in the library's kernels; this module only sequences the
calls, keeps the state on the device and records diagnostics (liquid area,
jet front height, spread of the liquid near the floor, solver statistics and
device time per step).  The geometry and parameters are those of the paper
(workloads.jet_2d); the time step is not given there and is a parameter.
The opening's edges lie on lattice points, so the level set vanishes there
and faces with a rounding-level liquid fraction appear: the live faces'
mass fraction is floored (stokes_set_min_face_liquid, 0.01 by default).
"""
import time

import numpy as np
import torch

from . import stokes, workloads


def _pgm(path, img):
    """Write an 8-bit grey image (row 0 at the top)."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    with open(path, "wb") as f:
        f.write(b"P5\n%d %d\n255\n" % (img.shape[1], img.shape[0]))
        f.write(img.tobytes())


class JetSim:
    """State of one planar jet simulation on the device."""

    def __init__(self, n=150, dt=0.002, ext_passes=8, min_face_liquid=0.01, options=None, stream=None):
        wl = workloads.jet_2d(n, dt)
        self.wl = wl
        self.n, self.h, self.dt = n, wl.h, dt
        self.ext_passes = ext_passes
        self.g = workloads.JET2D["g"]
        self.ctx = stokes.StokesContext(2, wl.n, wl.h, dt, wl.origin, stream=stream)
        self.ctx.set_min_face_liquid(min_face_liquid)
        d = stokes.upload_workload(wl)
        self.dev = d
        self.phi = d["phi_liquid"].clone()
        self.phi_next = torch.empty_like(self.phi)
        self.phi_src = torch.from_numpy(workloads.jet_2d_source(n)).cuda()
        self.u = [t.clone() for t in d["u_star"]]        # u^n (the initial velocity)
        self.u_star = [torch.empty_like(t) for t in self.u]
        self.tau = [torch.zeros(n * n, dtype=torch.float64, device="cuda"),
                    torch.zeros((n + 1) * (n + 1), dtype=torch.float64, device="cuda")]
        self.p = torch.zeros(n * n, dtype=torch.float64, device="cuda")
        self.opt = options or stokes.default_options(mode=stokes.FP32, precond=2, tol=1e-8, max_iter=200000)
        self.t = 0.0
        self.steps = 0
        self.history = []
        self._build()
        # fluid cells (the container's interior), for the diagnostics
        phiS = d["phi_solid"]
        self.fluid_cell = (phiS[2:2 * n + 2:2, 2:2 * n + 2:2] > 0)
        ys = (torch.arange(n, dtype=torch.float64, device="cuda") + 0.5) * self.h
        self.yc = ys.view(n, 1).expand(n, n)
        self.xc = ys.view(1, n).expand(n, n)

    def _build(self):
        d = self.dev
        self.ctx.build_weights(self.phi, d["phi_solid"], d["rho"], d["mu"], d["u_bc"])

    def step(self):
        """One time step; returns the record appended to ``history``."""
        ctx = self.ctx
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.advect(self.u, self.u_star, self.g, self.ext_passes, phi_in=self.phi, phi_out=self.phi_next,
                   phi_union=self.phi_src)
        self.phi, self.phi_next = self.phi_next, self.phi
        self._build()
        st = ctx.solve_step(self.u_star, self.u, self.tau, self.p, self.opt)
        e1.record()
        e1.synchronize()
        self.t += self.dt
        self.steps += 1
        rec = dict(step=self.steps, t=self.t, status=st.status, iterations=st.iterations,
                   rel_residual=st.rel_residual, ms=e0.elapsed_time(e1))
        rec.update(self.diagnostics())
        self.history.append(rec)
        return rec

    def liquid_cells(self):
        n = self.n
        return (self.phi[2:2 * n + 2:2, 2:2 * n + 2:2] < 0) & self.fluid_cell

    def diagnostics(self):
        """Liquid area (sum of W_L W_F over cells, h^2 each); the lowest
        liquid cell centre inside the container; the spread of the liquid
        within 0.1 of the container's bottom; the x-centroid of the liquid in
        the band 0.3 <= y <= 0.6; and the jet offset: over the rows with
        0.12 <= y <= 0.6 whose liquid is narrower than 0.15 (the jet, not the
        pool), the largest distance of the row's liquid centroid from the axis
        x = 0.5 (a buckling jet folds sideways above the pool)."""
        n, h = self.n, self.h
        wl = self.ctx.export(0)[: n * n]
        wf = self.ctx.export(1)[: n * n]
        area = float((wl * wf).sum()) * h * h
        liq = self.liquid_cells()
        out = dict(area=area)
        if bool(liq.any()):
            y = self.yc[liq]
            out["front_y"] = float(y.min())
            bottom = liq & (self.yc <= 0.2)
            out["floor_spread"] = float((self.xc[bottom] - 0.5).abs().max()) if bool(bottom.any()) else 0.0
            band = liq & (self.yc >= 0.3) & (self.yc <= 0.6)
            out["band_x"] = float(self.xc[band].mean()) if bool(band.any()) else 0.5
            lf = liq.to(torch.float64)
            cnt = lf.sum(1)
            cx = (lf * self.xc).sum(1) / cnt.clamp(min=1)
            ycol = self.yc[:, 0]
            rows = (cnt > 0) & (cnt * h < 0.15) & (ycol >= 0.12) & (ycol <= 0.6)
            out["jet_offset"] = float((cx[rows] - 0.5).abs().max()) if bool(rows.any()) else 0.0
        return out

    def image(self):
        """Grey image of the state: liquid black, air white, solid grey."""
        n = self.n
        liq = self.liquid_cells().cpu().numpy()
        fluid = self.fluid_cell.cpu().numpy()
        img = np.where(fluid, 255, 128).astype(np.uint8)
        img[liq] = 0
        return img[::-1]

    def run(self, t_end, snapshot_times=(), out_dir=None, log=None):
        """Step to t_end; at each snapshot time store an image (and write it
        as PGM into out_dir when given).  Returns {time: image}."""
        shots = {}
        pending = sorted(snapshot_times)
        wall0 = time.perf_counter()
        while self.t < t_end - 1e-12:
            rec = self.step()
            if rec["status"] != 0:
                raise RuntimeError(f"Stokes solve failed at step {self.steps}: {rec}")
            while pending and self.t >= pending[0] - 1e-9:
                tp = pending.pop(0)
                shots[tp] = self.image()
                if out_dir:
                    _pgm(f"{out_dir}/jet{self.n}_t{tp:.2f}.pgm", shots[tp])
            if log and self.steps % 50 == 0:
                log(f"t={self.t:.3f} iters={rec['iterations']} ms={rec['ms']:.2f} area={rec['area']:.5f} "
                    f"front={rec.get('front_y', float('nan')):.3f} band_x={rec.get('band_x', float('nan')):.4f} "
                    f"wall={time.perf_counter() - wall0:.1f}s")
        return shots

    def close(self):
        self.ctx.close()
