"""Pins of the volume-fraction estimator (oracle.fractions) against facts that
do not come from it: exact areas/volumes of half-planes and half-spaces cut
from a square/cube, complement symmetry, Monte-Carlo measure of the same
piecewise-linear interpolant, and the area/volume of a disk/ball."""
import numpy as np
import pytest

from oracle import fractions as F
from oracle import grid as G


def _square_halfplane_area(n, c):
    """Area of {x in [-1,1]^2 : n.x < c} / 4 by Sutherland-Hodgman clipping."""
    poly = [(-1, -1), (1, -1), (1, 1), (-1, 1)]
    f = lambda p: n[0] * p[0] + n[1] * p[1] - c
    out = []
    for i in range(4):
        p, q = poly[i], poly[(i + 1) % 4]
        fp, fq = f(p), f(q)
        if fp < 0:
            out.append(p)
        if (fp < 0) != (fq < 0):
            t = fp / (fp - fq)
            out.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
    if len(out) < 3:
        return 0.0
    a = 0.0
    for i in range(len(out)):
        x0, y0 = out[i]; x1, y1 = out[(i + 1) % len(out)]
        a += x0 * y1 - x1 * y0
    return abs(a) / 2 / 4.0


def _cube_halfspace_volume(n, c):
    """Volume of {x in [0,1]^3 : n.x < c} for n with no zero component, by the
    inclusion-exclusion formula sum_v (-1)^|v| max(c - n.v, 0)^3 / (6 n1 n2 n3)
    (valid for positive n; negative components are mirrored first)."""
    n = np.array(n, dtype=float)
    c = float(c)
    for d in range(3):
        if n[d] < 0:          # x_d -> 1 - x_d
            c -= n[d]
            n[d] = -n[d]
    tot = 0.0
    for v in np.ndindex(2, 2, 2):
        s = (-1) ** sum(v)
        tot += s * max(c - n @ np.array(v), 0.0) ** 3
    return tot / (6 * n[0] * n[1] * n[2])


def test_linear_levelset_exact_2d():
    rng = np.random.default_rng(10)
    for _ in range(300):
        th = rng.uniform(0, 2 * np.pi)
        n = np.array([np.cos(th), np.sin(th)])
        c = rng.uniform(-1.5, 1.5)
        # lattice around one CV: CV spans lattice -1..1 -> coordinates [-1,1]
        phi = np.empty((3, 3))
        for b in range(3):
            for a in range(3):
                phi[b, a] = n[0] * (a - 1) + n[1] * (b - 1) - c
        got = F.cv_fraction_2d(phi, np.array([1]), np.array([1]))[0]
        assert abs(got - _square_halfplane_area(n, c)) < 1e-13


def test_linear_levelset_exact_3d():
    rng = np.random.default_rng(11)
    for _ in range(200):
        n = rng.normal(size=3)
        n[np.abs(n) < 0.05] = 0.05
        c = rng.uniform(-1.0, 1.0) * np.abs(n).sum()
        phi = np.empty((3, 3, 3))
        for cc in range(3):
            for b in range(3):
                for a in range(3):
                    # CV [-1,1]^3 mapped to unit cube y = (x + 1) / 2
                    phi[cc, b, a] = n @ np.array([a - 1, b - 1, cc - 1]) - c
        got = F.cv_fraction_3d(phi, np.array([1]), np.array([1]), np.array([1]))[0]
        # n.x - c < 0 with x = 2y - 1  <=>  (2n).y < c + sum(n)
        ref = _cube_halfspace_volume(2 * n, c + n.sum())
        assert abs(got - ref) < 1e-12


def test_complement_sums_to_one():
    rng = np.random.default_rng(12)
    phi = rng.normal(size=(9, 9))
    a, b = np.meshgrid(np.arange(1, 8), np.arange(1, 8))
    s = F.cv_fraction_2d(phi, a, b) + F.cv_fraction_2d(-phi, a, b)
    assert np.allclose(s, 1.0, atol=1e-14)
    phi3 = rng.normal(size=(5, 5, 5))
    c3, b3, a3 = np.meshgrid(np.arange(1, 4), np.arange(1, 4), np.arange(1, 4), indexing="ij")
    s3 = F.cv_fraction_3d(phi3, a3, b3, c3) + F.cv_fraction_3d(-phi3, a3, b3, c3)
    assert np.allclose(s3, 1.0, atol=1e-13)


def _mc_simplex(vals, rng, m=400_000):
    """Monte-Carlo measure of {interpolant < 0} on one simplex."""
    w = rng.dirichlet(np.ones(len(vals)), size=m)
    return np.mean(w @ vals < 0)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_simplex_formulas_monte_carlo(k):
    rng = np.random.default_rng(13 + k)
    for _ in range(4):
        v3 = np.concatenate([-rng.uniform(0.1, 2, k), rng.uniform(0.1, 2, 3 - k)]) if k < 3 else -rng.uniform(0.1, 2, 3)
        got = F.triangle_fraction(v3[None])[0]
        assert abs(got - _mc_simplex(v3, rng)) < 4e-3
    for kk in range(1, 4):
        for _ in range(3):
            v4 = np.concatenate([-rng.uniform(0.1, 2, kk), rng.uniform(0.1, 2, 4 - kk)])
            rng.shuffle(v4)
            got = F.tetrahedron_fraction(v4[None])[0]
            assert abs(got - _mc_simplex(v4, rng)) < 4e-3


def test_two_two_tetrahedron_degenerate_values():
    # equal negative values make the textbook divided-difference form 0/0;
    # the combined form must stay finite and match the limit
    v = np.array([[-1.0, -1.0, 1.0, 1.0], [-1e-9, -1e-9, 2.0, 3.0], [-2.0, -2.0 + 1e-12, 0.0, 0.0]])
    f = F.tetrahedron_fraction(v)
    assert np.all(np.isfinite(f))
    assert abs(f[0] - 0.5) < 1e-15
    assert f[1] < 1e-15
    assert abs(f[2] - 1.0) < 1e-12


def _disk_area(n, r):
    h = 1.0 / n
    X = G.lattice_points(h, (0.0, 0.0), n, n)
    phi = np.hypot(X[0] - 0.5, X[1] - 0.5) - r
    idx = G.lattice_index("cell", n, n)
    return F.cv_fraction(phi, idx).sum() * h * h


def test_disk_area_second_order():
    r = 0.31
    e = [abs(_disk_area(n, r) - np.pi * r * r) for n in (16, 32, 64)]
    assert e[2] < 2e-4
    assert e[0] / e[2] > 8   # ~ O(h^2)


def test_ball_volume_second_order():
    r = 0.33
    errs = []
    for n in (12, 24):
        h = 1.0 / n
        X = G.lattice_points(h, (0.0,) * 3, n, n, n)
        phi = np.sqrt((X[0] - .5) ** 2 + (X[1] - .5) ** 2 + (X[2] - .5) ** 2) - r
        vol = F.cv_fraction(phi, G.lattice_index("cell", n, n, n)).sum() * h ** 3
        errs.append(abs(vol - 4 / 3 * np.pi * r ** 3))
    assert errs[1] < 5e-4
    assert errs[0] / errs[1] > 3.5


def test_zero_and_one_decided_by_signs():
    phi = np.ones((3, 3)); phi[1, 1] = 0.0
    assert F.cv_fraction_2d(phi, np.array([1]), np.array([1]))[0] == 0.0
    phi = -np.ones((3, 3)); phi[0, 0] = 0.0
    assert F.cv_fraction_2d(phi, np.array([1]), np.array([1]))[0] == 1.0
    phi = np.ones((3, 3)); phi[2, 2] = -1e-6
    f = F.cv_fraction_2d(phi, np.array([1]), np.array([1]))[0]
    # one corner slightly negative: one triangle, area ~ phi^2 / 2 of it
    assert 0.0 < f < 1e-12
