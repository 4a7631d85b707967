"""The 3D convergence case's inputs (workloads.sphere_3d) against what the
paper states (Section 9, "Three Dimensional Stokes Flow"): liquid inside
r = 1 (free surface), solid inside r = 0.25 and outside the box, rho = 1,
mu = 0.1, dt = 1, no solid motion, and the printed input velocity at every
face sample."""
import numpy as np

from paper_1010_2832_gb300 import workloads as W


def test_sphere_geometry_coefficients_and_input_velocity():
    n = 12
    wl = W.sphere_3d(n)
    assert wl.dim == 3 and wl.n == (n, n, n) and wl.dt == 1.0
    assert abs(wl.h - 2.5 / n) < 1e-15 and wl.origin == (-1.25, -1.25, -1.25)
    X = W.lattice_points(wl.n, wl.h, wl.origin)
    r = np.sqrt(X[0] ** 2 + X[1] ** 2 + X[2] ** 2)
    assert np.all((wl.phi_liquid < 0) == (r < 1.0))
    inner = r < 0.25 - 1e-12
    assert np.all(wl.phi_solid[inner] < 0)
    mid = (r > 0.25 + 1e-12) & (np.abs(X[0]) < 1.25 - 1e-12) & (np.abs(X[1]) < 1.25 - 1e-12) & \
          (np.abs(X[2]) < 1.25 - 1e-12)
    assert np.all(wl.phi_solid[mid] > 0)
    assert all(np.all(a == 1.0) for a in wl.rho) and all(np.all(m == 0.1) for m in wl.mu)
    assert all(np.all(u == 0.0) for u in wl.u_bc)
    exact = [lambda x, y, z: 0.5 + x * np.sin(y * z),
             lambda x, y, z: np.cos(0.25 * y) + 0.5 * x * y * z,
             lambda x, y, z: x + 0.5 * y * z ** 2 + np.sqrt(2.0 + y ** 2)]
    for d, f in enumerate(W.FACES[3]):
        P = W.sample_points(f, wl.n, wl.h, wl.origin)
        assert np.allclose(wl.u_star[d], exact[d](*P), rtol=0, atol=1e-14)
