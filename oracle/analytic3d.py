"""Closed-form 3D test solutions for the stress block of the 3D system
(Section 5, trace elimination; eq. stokesmixedsystemspd).

Test infrastructure only, like the rest of ``oracle``.  The paper's only 3D
study compares against a numerical solution (Section 9, "Three Dimensional
Stokes Flow"), which cannot tell a wrong 3D stress block from a right one.
These cases can: liquid fills a spherical cavity in a solid whose boundary
velocity u_BC is the exact velocity, so any smooth divergence-free u and any
smooth p solve one backward-Euler step (eq. stokesequations1-3) from

    u* = u + (dt / rho) (grad p - div tau),   tau = mu (grad u + grad u^T).

* ``linear_strain``: u = L x with trace L = 0.  tau is constant and
  div tau = grad p = 0, so u* = u; the discrete solution is exact (centred
  differences are exact on linear fields), with
  tau_xx = 2 mu L_xx, tau_yy = 2 mu L_yy, tau_ij = mu (L_ij + L_ji) and p
  constant.  The reduced rows read (tau_xx + tau_yy / 2) / mu = u_x - w_z and
  (tau_yy + tau_xx / 2) / mu = v_y - w_z, so a wrong coupling factor or sign
  shows at rounding level.
* ``vortical``: u = curl Psi for a smooth vector potential, a smooth p; the
  velocity converges at first order (the paper's order for velocity).

The box [-1, 1]^3 with the cavity r < 0.7 about the origin; rho = mu = dt = 1
so that the viscous term changes u* by O(1) and a wrong stress block leaves
an O(1) velocity error.
"""
from functools import lru_cache

import numpy as np

RHO, MU, DT = 1.0, 1.0, 1.0
R_CAVITY = 0.7
# a traceless velocity gradient (du_i / dx_j), for ``linear_strain``
L_STRAIN = np.array([[0.8, -0.3, 0.5],
                     [0.6, -1.1, 0.2],
                     [-0.4, 0.7, 0.3]])


@lru_cache(maxsize=None)
def _symbolic(case):
    import sympy as sy
    x, y, z = sy.symbols("x y z", real=True)
    X = (x, y, z)
    if case == "linear_strain":
        L = [[sy.nsimplify(v) for v in row] for row in L_STRAIN]
        u = [sum(L[i][j] * X[j] for j in range(3)) for i in range(3)]
        p = sy.Integer(0)
    elif case == "vortical":
        psi = (sy.Rational(1, 2) * sy.sin(sy.Rational(13, 10) * y + sy.Rational(1, 5)) * sy.cos(sy.Rational(9, 10) * z),
               sy.Rational(2, 5) * sy.cos(sy.Rational(11, 10) * x) * sy.sin(sy.Rational(7, 10) * z + sy.Rational(3, 10)),
               sy.Rational(3, 5) * sy.sin(sy.Rational(4, 5) * x + sy.Rational(1, 10)) * sy.sin(sy.Rational(6, 5) * y))
        u = [sy.diff(psi[2], y) - sy.diff(psi[1], z),
             sy.diff(psi[0], z) - sy.diff(psi[2], x),
             sy.diff(psi[1], x) - sy.diff(psi[0], y)]
        p = sy.Rational(3, 10) * sy.cos(x) * sy.sin(y + z)
    else:
        raise ValueError(case)
    mu = sy.nsimplify(MU)
    grad = [[sy.diff(u[i], X[j]) for j in range(3)] for i in range(3)]
    tau = [[mu * (grad[i][j] + grad[j][i]) for j in range(3)] for i in range(3)]
    div_tau = [sum(sy.diff(tau[i][j], X[j]) for j in range(3)) for i in range(3)]
    us = [u[i] + (sy.nsimplify(DT) / sy.nsimplify(RHO)) * (sy.diff(p, X[i]) - div_tau[i]) for i in range(3)]
    return dict(X=X, u=u, us=us, p=p, tau=tau,
                div=sum(sy.diff(u[i], X[i]) for i in range(3)))


@lru_cache(maxsize=None)
def fields(case):
    """numpy callables f(x, y, z): 'u0'..'u2', 'us0'..'us2', 'p', and the
    reduced stress unknowns 'tau_xx', 'tau_yy', 'tau_xy', 'tau_xz', 'tau_yz'."""
    import sympy as sy
    S = _symbolic(case)
    exprs = {f"u{i}": S["u"][i] for i in range(3)}
    exprs.update({f"us{i}": S["us"][i] for i in range(3)})
    exprs["p"] = S["p"]
    exprs["div"] = S["div"]
    t = S["tau"]
    exprs.update(tau_xx=t[0][0], tau_yy=t[1][1], tau_xy=t[0][1], tau_xz=t[0][2], tau_yz=t[1][2])
    out = {}
    for k, e in exprs.items():
        f = sy.lambdify(S["X"], e, "numpy")
        out[k] = (lambda f: (lambda X, Y, Z: np.broadcast_to(f(X, Y, Z), np.shape(X)).astype(np.float64)))(f)
    return out


def geometry(case):
    """(phi_liquid(X), phi_solid(X), u_bc(d, X)) for the cavity: liquid
    everywhere, solid outside r = R_CAVITY (box walls included), moving with
    the exact velocity of ``case``."""
    f = fields(case)
    return (lambda X: -np.ones(np.shape(X[0])),
            lambda X: R_CAVITY - np.sqrt(X[0] ** 2 + X[1] ** 2 + X[2] ** 2),
            lambda d, X: f[f"u{d}"](X[0], X[1], X[2]))
