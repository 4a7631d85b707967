"""FP64 reference of the fractional step around the Stokes solve (Section
"Application to Viscous Jet Buckling"), 2D, test infrastructure only.

    u* = (first-order semi-Lagrangian advection of u^n) + dt g
    phi^{n+1} = semi-Lagrangian advection of the liquid level set

Definitions (the paper names the scheme, bilinear interpolation of
velocities and a basic semi-Lagrangian level set, and leaves the rest).
Positions are in grid units, X = (x - origin) / h:
- u face (i, j) sits at (i, j + 1/2), v face (i, j) at (i + 1/2, j), the
  half-lattice point (a, b) of the level set at ((a - 1)/2, (b - 1)/2);
- a field is interpolated bilinearly between its samples; a point outside
  the samples' box is clamped onto it (constant extension);
- the departure point of a sample at X is X - (dt/h) (u(X), v(X)), with the
  sample's own velocity component and the other one interpolated; the new
  value is the old field interpolated at the departure point;
- before advection the velocity may be extended into faces that are not
  valid (e.g. carry no liquid): ``passes`` Jacobi sweeps, each giving an
  invalid face the mean of its valid 4-neighbours of the same component, if
  it has any, and marking it valid;
- gravity is added to u* after advection.
"""
import numpy as np


def _axis(n_samples, f):
    """Left index and weight of sample coordinate(s) f, clamped to the samples."""
    f = np.clip(f, 0.0, n_samples - 1.0)
    i0 = np.minimum(np.floor(f).astype(np.int64), n_samples - 2)
    return i0, f - i0


def interp(field, fx, fy):
    """Bilinear interpolation of a (ny_s, nx_s) array at sample coordinates."""
    ny_s, nx_s = field.shape
    i0, tx = _axis(nx_s, fx)
    j0, ty = _axis(ny_s, fy)
    a = field[j0, i0] * (1.0 - tx) + field[j0, i0 + 1] * tx
    b = field[j0 + 1, i0] * (1.0 - tx) + field[j0 + 1, i0 + 1] * tx
    return a * (1.0 - ty) + b * ty


def interp_u(u, X, Y):
    return interp(u, X, Y - 0.5)


def interp_v(v, X, Y):
    return interp(v, X - 0.5, Y)


def interp_phi(phi, X, Y):
    return interp(phi, 2.0 * X + 1.0, 2.0 * Y + 1.0)


def face_points(kind, n):
    """Grid-unit positions of the u or v faces of an n = (nx, ny) grid."""
    nx, ny = n
    if kind == "u":
        i, j = np.meshgrid(np.arange(nx + 1), np.arange(ny), indexing="xy")
        return i.astype(np.float64), j + 0.5
    i, j = np.meshgrid(np.arange(nx), np.arange(ny + 1), indexing="xy")
    return i + 0.5, j.astype(np.float64)


def lattice_points(shape):
    a, b = np.meshgrid(np.arange(shape[1]), np.arange(shape[0]), indexing="xy")
    return (a - 1) / 2.0, (b - 1) / 2.0


def extend(field, valid, passes):
    """Jacobi sweeps: invalid samples with valid 4-neighbours take their mean."""
    f = np.array(field, dtype=np.float64, copy=True)
    ok = np.array(valid, dtype=bool, copy=True)
    ny, nx = f.shape
    for _ in range(passes):
        s = np.zeros_like(f)
        c = np.zeros(f.shape, dtype=np.int64)
        for dj, di in ((0, -1), (0, 1), (-1, 0), (1, 0)):
            for j in range(ny):
                for i in range(nx):
                    jj, ii = j + dj, i + di
                    if 0 <= jj < ny and 0 <= ii < nx and ok[jj, ii]:
                        s[j, i] += f[jj, ii]
                        c[j, i] += 1
        fill = ~ok & (c > 0)
        f = np.where(fill, s / np.maximum(c, 1), f)
        ok = ok | fill
    return f


def advect_velocity(u, v, h, dt, g, valid_u=None, valid_v=None, passes=0):
    """u* on u and v faces (arrays shaped (ny, nx+1) and (ny+1, nx))."""
    if passes:
        u = extend(u, valid_u, passes)
        v = extend(v, valid_v, passes)
    n = (u.shape[1] - 1, u.shape[0])
    c = dt / h
    X, Y = face_points("u", n)
    us = interp_u(u, X - c * u, Y - c * interp_v(v, X, Y)) + dt * g[0]
    X, Y = face_points("v", n)
    vs = interp_v(v, X - c * interp_u(u, X, Y), Y - c * v) + dt * g[1]
    return us, vs


def advect_levelset(phi, u, v, h, dt, valid_u=None, valid_v=None, passes=0):
    """phi^{n+1} on the half lattice (shape (2ny+3, 2nx+3))."""
    if passes:
        u = extend(u, valid_u, passes)
        v = extend(v, valid_v, passes)
    c = dt / h
    X, Y = lattice_points(phi.shape)
    return interp_phi(phi, X - c * interp_u(u, X, Y), Y - c * interp_v(v, X, Y))
