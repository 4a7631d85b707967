"""Closed-form 2D test solutions of Section 9 (convergence studies).

Each case gives the final velocity through a stream function psi (with
u = (d psi/dy, -d psi/dx), the sign that makes the free-surface cases
traction-free and the moving wall turn clockwise) and a pressure p.  The
final stress is tau = mu (grad u + grad u^T) and the input velocity follows
from the backward-Euler equation (eq. stokesequations1):
    u* = u + (dt / rho) (grad p - div tau).

Geometry is laid out on the box [-1, 1]^2 (the paper does not state its
box).  Readings of the printed cases:
* free surface disk (Section 9.1): liquid r < 0.75, no solid but the box;
* solid annulus (Section 9.2): static solids r < 0.5 and r > 1;
* mixed annulus (Section 9.3): as printed the solution is traction-free at
  r = 0.65 (not 0.75) and does not vanish at the inner wall r = 0.1, so the
  free surface is placed at r = 0.65 and the inner solid moves with the
  exact velocity (u_BC = u there);
* moving inner wall (Section 9.4): solids r < 0.5 (rigid clockwise rotation,
  angular speed 2) and r > 1 (static).
"""
from functools import lru_cache

import numpy as np

CASES = ("free_surface", "solid_wall", "mixed", "moving_solid")
RHO, MU, DT = 1.0, 0.1, 1.0


@lru_cache(maxsize=None)
def _symbolic(case):
    import sympy as sy
    x, y = sy.symbols("x y", real=True)
    r = sy.sqrt(x * x + y * y)
    th = sy.atan2(y, x)
    mu = sy.Rational(1, 10)
    s3 = sy.sqrt(3)
    if case == "free_surface":
        poly = 15 - 30 * r + 16 * r ** 2
        psi = sy.Rational(128, 81) * r ** 4 * sy.cos(2 * th) * sy.cos(s3 * sy.log(r)) * poly
        p = sy.Rational(512, 81) * s3 * r ** 2 * mu * sy.sin(2 * th) * sy.sin(s3 * sy.log(r)) * poly
    elif case == "solid_wall":
        psi = 256 * r ** 4 - 768 * r ** 3 + 832 * r ** 2 - 384 * r + 64
        p = r ** 2 * sy.cos(th) * sy.sin(th)
    elif case == "mixed":
        poly = 169 - 390 * r + 240 * r ** 2
        psi = sy.Rational(80000, 371293) * sy.cos(2 * th) * r ** 4 * sy.cos(s3 * sy.log(r)) * poly
        p = sy.Rational(320000, 371293) * s3 * mu * r ** 2 * sy.sin(2 * th) * sy.sin(s3 * sy.log(r)) * poly
    elif case == "moving_solid":
        psi = r ** 4 - 3 * r ** 3 + sy.Rational(9, 4) * r ** 2 + r / 2 + sy.Rational(1, 4)
        p = r ** 2 * sy.cos(th) * sy.sin(th)
    else:
        raise ValueError(case)
    u = sy.diff(psi, y)
    v = -sy.diff(psi, x)
    txx = 2 * mu * sy.diff(u, x)
    tyy = 2 * mu * sy.diff(v, y)
    txy = mu * (sy.diff(u, y) + sy.diff(v, x))
    div_tau_x = sy.diff(txx, x) + sy.diff(txy, y)
    div_tau_y = sy.diff(txy, x) + sy.diff(tyy, y)
    us = u + (DT / RHO) * (sy.diff(p, x) - div_tau_x)
    vs = v + (DT / RHO) * (sy.diff(p, y) - div_tau_y)
    # reduced unknown tau_xx = mu (u_x - v_y) equals 2 mu u_x for div-free u
    red_txx = mu * (sy.diff(u, x) - sy.diff(v, y))
    return dict(x=x, y=y, psi=psi, p=p, u=u, v=v, txx=red_txx, txy=txy, us=us, vs=vs,
                tyy=tyy, full_txx=txx)


def _off_origin(X, Y):
    # the log-radius factors are singular at r = 0 where the fields vanish;
    # evaluate there at a point 1e-12 away (the limit value, to rounding)
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return np.where((X == 0) & (Y == 0), 1e-12, X), Y


@lru_cache(maxsize=None)
def fields(case):
    """numpy callables f(x, y) for u, v, p, txx, txy, us, vs."""
    import sympy as sy
    S = _symbolic(case)
    out = {}
    for k in ("u", "v", "p", "txx", "txy", "us", "vs"):
        f = sy.lambdify((S["x"], S["y"]), S[k], "numpy")
        out[k] = (lambda f: (lambda X, Y: np.broadcast_to(f(*_off_origin(X, Y)), np.shape(X)).astype(np.float64)))(f)
    return out


def traction(case, radius, thetas):
    """Traction (-p I + tau) n on the circle r = radius (outward normal)."""
    import sympy as sy
    S = _symbolic(case)
    x, y = S["x"], S["y"]
    tf = {k: sy.lambdify((x, y), S[k], "numpy") for k in ("p", "full_txx", "tyy", "txy")}
    X = radius * np.cos(thetas); Y = radius * np.sin(thetas)
    nx, ny = np.cos(thetas), np.sin(thetas)
    p = tf["p"](X, Y); txx = tf["full_txx"](X, Y); tyy = tf["tyy"](X, Y); txy = tf["txy"](X, Y)
    return np.stack([(-p + txx) * nx + txy * ny, txy * nx + (-p + tyy) * ny])


def geometry(case):
    """(phi_liquid(X), phi_solid(X), u_bc(d, X)) callables on the box [-1, 1]^2."""
    box = lambda X: np.minimum(np.minimum(X[0] + 1, 1 - X[0]), np.minimum(X[1] + 1, 1 - X[1]))
    R = lambda X: np.hypot(X[0], X[1])
    zero = lambda d, X: np.zeros(np.shape(X[0]))
    if case == "free_surface":
        return (lambda X: R(X) - 0.75), box, zero
    if case == "solid_wall":
        return (lambda X: -np.ones(np.shape(X[0]))), \
               (lambda X: np.minimum(box(X), np.minimum(R(X) - 0.5, 1 - R(X)))), zero
    if case == "mixed":
        f = fields(case)
        def ubc(d, X):
            val = f["u"](X[0], X[1]) if d == 0 else f["v"](X[0], X[1])
            return np.where(R(X) < 0.375, val, 0.0)
        return (lambda X: R(X) - 0.65), (lambda X: np.minimum(box(X), R(X) - 0.1)), ubc
    if case == "moving_solid":
        def ubc(d, X):
            # clockwise rigid rotation, angular speed 2: (2 y, -2 x)
            val = 2.0 * X[1] if d == 0 else -2.0 * X[0]
            return np.where(R(X) < 0.75, val, 0.0)
        return (lambda X: -np.ones(np.shape(X[0]))), \
               (lambda X: np.minimum(box(X), np.minimum(R(X) - 0.5, 1 - R(X)))), ubc
    raise ValueError(case)
