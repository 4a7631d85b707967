"""Seeded synthetic inputs for one Stokes step (shared by tests, bench and smoke).

This module only builds input arrays: level sets sampled on the half
lattice, density per velocity sample, viscosity per stress sample, the
prescribed solid velocity u_BC and the input velocity u* per face.  It holds
none of the method's arithmetic (no fractions, weights, stencils or solves).

Layouts (x varies fastest; numpy shapes are slowest-axis first):
  half lattice  2D (2ny+3, 2nx+3), 3D (2nz+3, 2ny+3, 2nx+3); point (a, b, c)
                at origin + ((a-1) h/2, (b-1) h/2, (c-1) h/2)
  u faces (ny, nx+1) | v faces (ny+1, nx)                         [2D]
  cells (ny, nx) | nodes (ny+1, nx+1)
  u (nz, ny, nx+1) | v (nz, ny+1, nx) | w (nz+1, ny, nx)          [3D]
  cells (nz, ny, nx) | xy-stress z-edges (nz, ny+1, nx+1)
  xz-stress y-edges (nz+1, ny, nx+1) | yz-stress x-edges (nz+1, ny+1, nx)
Level-set sign convention: phi_liquid < 0 inside the liquid (extended into
solids), phi_solid < 0 inside solids.  The box walls are part of phi_solid.
"""
from dataclasses import dataclass

import numpy as np

# lattice offsets of each sample kind (x, y[, z]); a = 2 i + offset
_OFF2 = {"cell": (2, 2), "node": (1, 1), "u": (1, 2), "v": (2, 1)}
_OFF3 = {"cell": (2, 2, 2), "u": (1, 2, 2), "v": (2, 1, 2), "w": (2, 2, 1),
         "exy": (1, 1, 2), "exz": (1, 2, 1), "eyz": (2, 1, 1)}
FACES = {2: ("u", "v"), 3: ("u", "v", "w")}
STRESS_SITES = {2: ("cell", "node"), 3: ("cell", "exy", "exz", "eyz")}


@dataclass
class Workload:
    name: str
    dim: int
    n: tuple            # (nx, ny) or (nx, ny, nz)
    h: float
    dt: float
    origin: tuple
    phi_liquid: np.ndarray
    phi_solid: np.ndarray
    rho: list           # per face kind
    mu: list            # per stress site kind (STRESS_SITES order)
    u_bc: list          # per face kind
    u_star: list        # per face kind

    def as_oracle_kwargs(self):
        return dict(dim=self.dim, n=tuple(self.n), h=self.h, dt=self.dt, origin=tuple(self.origin),
                    phi_liquid=self.phi_liquid, phi_solid=self.phi_solid, rho=self.rho,
                    mu=self.mu, u_bc=self.u_bc, u_star=self.u_star)


def field_shape(kind, n):
    off = (_OFF2 if len(n) == 2 else _OFF3)[kind]
    return tuple(reversed([n[d] + (off[d] == 1) for d in range(len(n))]))


def sample_points(kind, n, h, origin):
    off = (_OFF2 if len(n) == 2 else _OFF3)[kind]
    shp = field_shape(kind, n)
    axes = [origin[d] + (2 * np.arange(shp[len(n) - 1 - d]) + off[d] - 1) * (h / 2) for d in range(len(n))]
    g = np.meshgrid(*reversed(axes), indexing="ij")
    return tuple(reversed(g))


def lattice_points(n, h, origin):
    axes = [origin[d] + (np.arange(2 * n[d] + 3) - 1) * (h / 2) for d in range(len(n))]
    g = np.meshgrid(*reversed(axes), indexing="ij")
    return tuple(reversed(g))


def box_phi(X, lo, hi):
    """Signed distance-like level set of the box walls: < 0 outside [lo, hi]."""
    out = None
    for d, x in enumerate(X):
        m = np.minimum(x - lo[d], hi[d] - x)
        out = m if out is None else np.minimum(out, m)
    return out


def from_functions(name, dim, n, h, dt, origin, phiL_fn, phiS_fn, rho_fn, mu_fn, ubc_fn, ustar_fn):
    """Sample level sets on the half lattice and coefficients/velocities at
    their sample points from the given callables (X is a tuple of coordinate
    arrays; velocity callables also get the component index d)."""
    lat = lattice_points(n, h, origin)
    faces = FACES[dim]
    rho, ubc, ust = [], [], []
    for d, f in enumerate(faces):
        P = sample_points(f, n, h, origin)
        rho.append(np.ascontiguousarray(rho_fn(P), dtype=np.float64) * np.ones(P[0].shape))
        ubc.append(np.ascontiguousarray(ubc_fn(d, P), dtype=np.float64) * np.ones(P[0].shape))
        ust.append(np.ascontiguousarray(ustar_fn(d, P), dtype=np.float64) * np.ones(P[0].shape))
    mu = []
    for s in STRESS_SITES[dim]:
        P = sample_points(s, n, h, origin)
        mu.append(np.ascontiguousarray(mu_fn(P), dtype=np.float64) * np.ones(P[0].shape))
    return Workload(name, dim, tuple(n), h, dt, tuple(origin),
                    np.ascontiguousarray(phiL_fn(lat), dtype=np.float64),
                    np.ascontiguousarray(phiS_fn(lat), dtype=np.float64),
                    rho, mu, ubc, ust)


def disk_in_box(n=32, seed=1, radius=0.3):
    """2D n x n unit box with solid walls; liquid disk of radius 0.3 centred at
    (0.5, 0.5); rho = mu = 1, dt = 0.01; u* iid U[-1, 1]; static walls."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    lo, hi = (0.0, 0.0), (1.0, 1.0)
    def ustar(d, P):
        return rng.uniform(-1.0, 1.0, P[0].shape)
    return from_functions(f"disk{n}", 2, (n, n), h, 0.01, (0.0, 0.0),
                 lambda X: np.hypot(X[0] - 0.5, X[1] - 0.5) - radius,
                 lambda X: box_phi(X, lo, hi),
                 lambda P: 1.0, lambda P: 1.0, lambda d, P: 0.0, ustar)


def _smooth_ustar(d, P):
    """A smooth, non-rigid intermediate velocity (not a solution of anything)."""
    x, y = P[0], P[1]
    return np.sin(1.0 + 2.0 * x + 3.0 * y + d) + 0.5 * np.cos(3.0 * x - 2.0 * y + 2.0 * d)


def paper_disk(n):
    """Geometry of Section 9's solver-iteration test with a free surface:
    n x n grid on [-1, 1]^2 with walls, a liquid disk of radius 0.75 at the
    origin surrounded by air, rho = 1, mu = 0.1, dt = 1; smooth u*."""
    h = 2.0 / n
    lo, hi = (-1.0, -1.0), (1.0, 1.0)
    return from_functions(f"paperdisk{n}", 2, (n, n), h, 1.0, lo,
                          lambda X: np.hypot(X[0], X[1]) - 0.75, lambda X: box_phi(X, lo, hi),
                          lambda P: 1.0, lambda P: 0.1, lambda d, P: 0.0, _smooth_ustar)


def paper_annulus(n):
    """Geometry of Section 9's solver-iteration test with solid walls: n x n
    grid on [-1, 1]^2, liquid filling the annulus 0.5 <= r <= 1 between two
    static solid walls, rho = 1, mu = 0.1, dt = 1; smooth u*."""
    h = 2.0 / n
    lo, hi = (-1.0, -1.0), (1.0, 1.0)
    def phiS(X):
        r = np.hypot(X[0], X[1])
        return np.minimum(np.minimum(r - 0.5, 1.0 - r), box_phi(X, lo, hi))
    return from_functions(f"paperannulus{n}", 2, (n, n), h, 1.0, lo,
                          lambda X: -np.ones(X[0].shape), phiS,
                          lambda P: 1.0, lambda P: 0.1, lambda d, P: 0.0, _smooth_ustar)


def sphere_3d(n, half=1.25):
    """The 3D case of Section 9 (Three Dimensional Stokes Flow): a liquid
    sphere r < 1 at the origin with a free surface, a static solid sphere
    r < 0.25 inside it, rho = 1, mu = 0.1, dt = 1, and the printed input
    velocity u = (0.5 + x sin(yz), cos(y/4) + xyz/2, x + yz^2/2 + sqrt(2 + y^2)).
    The box is [-half, half]^3 (the paper does not state it), n^3 cells."""
    h = 2.0 * half / n
    lo, hi = (-half,) * 3, (half,) * 3
    def ustar(d, P):
        x, y, z = P
        if d == 0:
            return 0.5 + x * np.sin(y * z)
        if d == 1:
            return np.cos(0.25 * y) + 0.5 * x * y * z
        return x + 0.5 * y * z * z + np.sqrt(2.0 + y * y)
    R = lambda X: np.sqrt(X[0] ** 2 + X[1] ** 2 + X[2] ** 2)
    return from_functions(f"sphere{n}", 3, (n, n, n), h, 1.0, lo,
                          lambda X: R(X) - 1.0, lambda X: np.minimum(box_phi(X, lo, hi), R(X) - 0.25),
                          lambda P: 1.0, lambda P: 0.1, lambda d, P: 0.0, ustar)


# Planar jet buckling (Section "Two Dimensional Jet Buckling")
JET2D = dict(center=(0.5, 0.5), radius=0.4, ceiling=0.8, jet_x=0.5, width=0.06, U=-0.5,
             rho=1.0, mu=0.075, g=(0.0, -9.81))


def _jet_opening_phi(X, h, depth):
    """< 0 inside the jet opening [x0 - D/2, x0 + D/2] x [ceiling - depth, inf)."""
    J = JET2D
    half = J["width"] / 2
    return np.maximum(np.abs(X[0] - J["jet_x"]) - half, (J["ceiling"] - depth) - X[1])


def jet_2d(n=150, dt=0.002, stub_cells=3):
    """Planar viscous jet: n x n grid on the unit square; solid outside the
    circle of radius 0.4 centred at (0.5, 0.5) and above the ceiling
    y = 0.8; the part of the ceiling over the opening of width D = 0.06 at
    x = 0.5 moves with u_BC = (0, U), U = -0.5 (the inflow), its profile
    ramped linearly over one cell at the opening's edges so that the v faces
    carry the flux D U exactly; rho = 1, mu = 0.075.  The liquid starts as a
    stub of ``stub_cells`` cells below the opening (and fills the opening);
    u* = (0, U) everywhere (the initial velocity)."""
    J = JET2D
    h = 1.0 / n
    def phiS(X):
        r = np.hypot(X[0] - J["center"][0], X[1] - J["center"][1])
        return np.minimum(J["radius"] - r, J["ceiling"] - X[1])
    def ubc(d, P):
        if d == 0:
            return np.zeros(P[0].shape)
        ramp = np.clip((J["width"] / 2 - np.abs(P[0] - J["jet_x"])) / h + 0.5, 0.0, 1.0)
        return J["U"] * ramp * (P[1] >= J["ceiling"] - h / 4)
    return from_functions(f"jet{n}", 2, (n, n), h, dt, (0.0, 0.0),
                          lambda X: _jet_opening_phi(X, h, stub_cells * h), phiS,
                          lambda P: J["rho"], lambda P: J["mu"], ubc,
                          lambda d, P: np.full(P[0].shape, 0.0 if d == 0 else J["U"]))


def jet_2d_source(n=150):
    """Half-lattice level set of the jet opening (the inflow source region):
    the liquid level set is united with it after every advection."""
    h = 1.0 / n
    return np.ascontiguousarray(_jet_opening_phi(lattice_points((n, n), h, (0.0, 0.0)), h, 0.0))


def _bumps(rng, dim, k=8, c_lo=0.2, c_hi=0.8, s_lo=0.05, s_hi=0.12):
    c = rng.uniform(c_lo, c_hi, (k, dim))
    s = rng.uniform(s_lo, s_hi, k)
    def phi(X):
        tot = 0.0
        for i in range(k):
            r2 = sum((X[d] - c[i, d]) ** 2 for d in range(dim))
            tot = tot + np.exp(-r2 / (2 * s[i] ** 2))
        return 0.5 - tot
    return phi


def _log_viscosity(rng, dim):
    """mu = 10^(2 s), s a product of one sine and cosines: spans 1e-2 .. 1e2."""
    kk = rng.integers(1, 3, dim)
    th = rng.uniform(0.0, 1.0, dim)
    def mu(P):
        s = np.sin(2 * np.pi * (kk[0] * P[0] + th[0]))
        for d in range(1, dim):
            s = s * np.cos(2 * np.pi * (kk[d] * P[d] + th[d]))
        return 10.0 ** (2.0 * s)
    return mu


def bumps_2d(n=1024, seed=2, rho_split=True, disk_r=0.1, disk_vel=(0.5, 0.0), name=None):
    """2D n x n unit box: liquid = {sum of 8 Gaussian bumps > 0.5}; solid =
    walls + disk of radius ``disk_r`` moving at ``disk_vel``; log-uniform mu in
    [1e-2, 1e2]; rho = 1000 below y = 0.5 and 1 above (or 1 everywhere);
    dt = 0.01; u* iid U[-1, 1].  u_BC is the disk velocity on faces nearer the
    disk than the walls and 0 elsewhere."""
    rng = np.random.default_rng(seed)
    phiL = _bumps(rng, 2)
    cs = rng.uniform(0.3, 0.7, 2)
    mu = _log_viscosity(rng, 2)
    h = 1.0 / n
    lo, hi = (0.0, 0.0), (1.0, 1.0)
    disk = lambda X: np.hypot(X[0] - cs[0], X[1] - cs[1]) - disk_r
    def ubc(d, P):
        near = disk(P) < box_phi(P, lo, hi)
        return np.where(near, disk_vel[d], 0.0)
    def rho(P):
        return np.where(P[1] < 0.5, 1000.0, 1.0) if rho_split else np.ones(P[0].shape)
    def ustar(d, P):
        return rng.uniform(-1.0, 1.0, P[0].shape)
    return from_functions(name or f"bumps{n}", 2, (n, n), h, 0.01, (0.0, 0.0), phiL,
                 lambda X: np.minimum(box_phi(X, lo, hi), disk(X)), rho, mu, ubc, ustar)


def batch_instances(count=64, n_lo=64, n_hi=512, seed0=4000):
    """Uneven batch: instance i has n_i ~ U{n_lo..n_hi} (seed seed0 + i), built
    like ``bumps_2d`` with rho = 1, disk radius ~ U[0.05, 0.15] and disk
    velocity ~ U[-0.5, 0.5]^2."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(rng.integers(n_lo, n_hi + 1))
        r = float(rng.uniform(0.05, 0.15))
        vel = tuple(rng.uniform(-0.5, 0.5, 2))
        out.append(bumps_2d(n, seed=seed0 + i, rho_split=False, disk_r=r, disk_vel=vel,
                            name=f"batch{i}_{n}"))
    return out


def column_3d(n=256, window=None):
    """3D unit cube: liquid column of radius 0.05 around x = z = 0.5 below
    y = 0.6, standing on a solid floor y < 0.1 (plus walls); rho = 1000,
    mu = 10, dt = 1e-3; u* = (0, -0.5 - 9.81 dt, 0); static solids.

    ``window=(i0, j0, k0, ni, nj, nk)`` samples the same fields on the
    sub-grid of cells [i0, i0+ni) x [j0, j0+nj) x [k0, k0+nk) of the n^3 grid
    (same spacing and physical positions; the window's own boundary is a
    wall, so it reproduces the full grid's system when at least two cells of
    air or solid separate the liquid from the window's sides)."""
    h = 1.0 / n
    dt = 1e-3
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    phiL = lambda X: np.maximum(np.hypot(X[0] - 0.5, X[2] - 0.5) - 0.05, X[1] - 0.6)
    phiS = lambda X: np.minimum(box_phi(X, lo, hi), X[1] - 0.1)
    vy = -0.5 - 9.81 * dt
    dims, origin = (n, n, n), (0.0, 0.0, 0.0)
    if window is not None:
        i0, j0, k0, ni, nj, nk = window
        dims, origin = (ni, nj, nk), (i0 * h, j0 * h, k0 * h)
    return from_functions(f"column{n}", 3, dims, h, dt, origin, phiL, phiS,
                 lambda P: 1000.0, lambda P: 10.0, lambda d, P: 0.0,
                 lambda d, P: (vy if d == 1 else 0.0))


def bumps_3d(n=128, seed=5000):
    """3D analogue of ``bumps_2d``: 8 Gaussian bumps, solid = walls + sphere of
    radius 0.1 moving at (0.5, 0, 0), log-uniform mu, rho = 1000 below
    y = 0.5 else 1, dt = 0.01, u* iid U[-1, 1]."""
    rng = np.random.default_rng(seed)
    phiL = _bumps(rng, 3)
    cs = rng.uniform(0.3, 0.7, 3)
    mu = _log_viscosity(rng, 3)
    h = 1.0 / n
    lo, hi = (0.0,) * 3, (1.0,) * 3
    sph = lambda X: np.sqrt(sum((X[d] - cs[d]) ** 2 for d in range(3))) - 0.1
    vel = (0.5, 0.0, 0.0)
    def ubc(d, P):
        return np.where(sph(P) < box_phi(P, lo, hi), vel[d], 0.0)
    def ustar(d, P):
        return rng.uniform(-1.0, 1.0, P[0].shape)
    return from_functions(f"bumps3d_{n}", 3, (n, n, n), h, 0.01, (0.0,) * 3, phiL,
                 lambda X: np.minimum(box_phi(X, lo, hi), sph(X)),
                 lambda P: np.where(P[1] < 0.5, 1000.0, 1.0), mu, ubc, ustar)


def full_box(n, dim, seed=0, dt=0.01):
    """Box entirely full of liquid (every unknown active except at the walls):
    the roofline microbenchmark workload.  rho = 1, mu = 1, u* iid U[-1, 1]."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    lo, hi = (0.0,) * dim, (1.0,) * dim
    return from_functions(f"fullbox{dim}d_{n}", dim, (n,) * dim, h, dt, (0.0,) * dim,
                 lambda X: -np.ones(X[0].shape), lambda X: box_phi(X, lo, hi),
                 lambda P: 1.0, lambda P: 1.0, lambda d, P: 0.0,
                 lambda d, P: rng.uniform(-1.0, 1.0, P[0].shape))


def random_small(n=(8, 7), seed=0, dim=2):
    """Tiny random geometry for structural tests: random-blob liquid, random
    blob solid, random positive coefficients, random u* and u_BC."""
    rng = np.random.default_rng(seed)
    n = tuple(n)
    h = 1.0 / max(n)
    L = tuple(h * k for k in n)
    cL = rng.uniform(0.2, 0.8, dim) * np.array(L)
    cS = rng.uniform(0.0, 1.0, dim) * np.array(L)
    rL = rng.uniform(0.25, 0.45) * min(L)
    rS = rng.uniform(0.1, 0.3) * min(L)
    wob = rng.uniform(-0.3, 0.3, 3)
    def phiL(X):
        r = np.sqrt(sum((X[d] - cL[d]) ** 2 for d in range(dim)))
        return r - rL * (1 + wob[0] * np.sin(3 * X[0] / L[0] + wob[1]))
    def phiS(X):
        r = np.sqrt(sum((X[d] - cS[d]) ** 2 for d in range(dim)))
        return np.minimum(box_phi(X, (0.0,) * dim, L), r - rS)
    return from_functions(f"rand{dim}d_{seed}", dim, n, h, 0.05, (0.0,) * dim, phiL, phiS,
                 lambda P: rng.uniform(0.5, 2.0, P[0].shape),
                 lambda P: rng.uniform(0.1, 3.0, P[0].shape),
                 lambda d, P: rng.uniform(-1.0, 1.0, P[0].shape),
                 lambda d, P: rng.uniform(-1.0, 1.0, P[0].shape))
