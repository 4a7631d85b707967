"""Control-volume fractions W_L and W_F, Section 5 (volume-fraction paragraph).

The paper weights every term of the variational form by the fraction of a
cell-sized control volume (CV) centred on the sample that lies inside the
liquid (W_L, from the liquid level set phi_L < 0) or inside the fluid, i.e.
outside the solid (W_F = 1 - fraction of phi_S < 0).  It only suggests an
estimator (Min and Gibou's level-set integration).  Our reading, shared with
the GPU path by definition but not by code:

* the level set is known at the points of the half lattice (see ``grid``);
* inside a CV it is the piecewise-linear interpolant on a fixed simplex
  split that uses every lattice point of the CV: in 2D the 8 triangles
  (centre, edge midpoint, adjacent corner); in 3D the 24 tetrahedra
  (centre, face centre, two corners of one edge of that face);
* the fraction is the exact measure of {interpolant < 0}, summed over the
  simplices, divided by the CV measure.

For a linear function on an n-simplex with vertex values phi_i the measure of
{phi < 0} divided by the simplex measure is sum over negative vertices of
phi_i^n / prod_{j != i} (phi_i - phi_j) (a divided difference of the
truncated power).  Below this is written in cancellation-free form for each
count of negative vertices.  Zero values count as non-negative; a CV with no
negative lattice value has fraction exactly 0, one with no positive value
exactly 1, so "W > 0" is decided by signs alone.
"""
import numpy as np


def triangle_fraction(v):
    """Fraction of a triangle where the linear interpolant is < 0.

    ``v``: array (..., 3) of vertex values.  Closed forms by the number k of
    negative vertices (s sorted ascending):
      k = 1: s0^2 / ((s0 - s1)(s0 - s2))
      k = 2: 1 - s2^2 / ((s2 - s0)(s2 - s1))
    """
    s = np.sort(np.asarray(v, dtype=np.float64), axis=-1)
    s0, s1, s2 = s[..., 0], s[..., 1], s[..., 2]
    k = (s < 0).sum(axis=-1)
    out = np.zeros(s0.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        f1 = s0 * s0 / ((s0 - s1) * (s0 - s2))
        f2 = 1.0 - s2 * s2 / ((s2 - s0) * (s2 - s1))
    out = np.where(k == 1, f1, out)
    out = np.where(k == 2, f2, out)
    out = np.where(k == 3, 1.0, out)
    return out


def tetrahedron_fraction(v):
    """Fraction of a tetrahedron where the linear interpolant is < 0.

    ``v``: array (..., 4).  With s sorted ascending and k negative vertices:
      k = 1: s0^3 / ((s0-s1)(s0-s2)(s0-s3))
      k = 2: with x, y = s0, s1 (< 0) and p, q = s2, s3 (>= 0), the two
             divided-difference terms over a common denominator:
             [x^2 y^2 - (p+q) x y (x+y) + p q (x^2 + x y + y^2)]
             / [(x-p)(x-q)(y-p)(y-q)]   (every term is >= 0)
      k = 3: 1 - s3^3 / ((s3-s0)(s3-s1)(s3-s2))
    """
    s = np.sort(np.asarray(v, dtype=np.float64), axis=-1)
    s0, s1, s2, s3 = (s[..., i] for i in range(4))
    k = (s < 0).sum(axis=-1)
    out = np.zeros(s0.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        f1 = s0 * s0 * s0 / ((s0 - s1) * (s0 - s2) * (s0 - s3))
        x, y, p, q = s0, s1, s2, s3
        num = x * x * y * y - (p + q) * x * y * (x + y) + p * q * (x * x + x * y + y * y)
        f2 = num / ((x - p) * (x - q) * (y - p) * (y - q))
        f3 = 1.0 - s3 * s3 * s3 / ((s3 - s0) * (s3 - s1) * (s3 - s2))
    out = np.where(k == 1, f1, out)
    out = np.where(k == 2, f2, out)
    out = np.where(k == 3, f3, out)
    out = np.where(k == 4, 1.0, out)
    return out


def cv_fraction_2d(phi, a, b):
    """Fraction of {phi < 0} in the CVs centred at lattice points (a, b).

    ``phi`` is lattice-shaped (index [b, a]); the CV spans a-1..a+1, b-1..b+1.
    Eight triangles (centre, edge midpoint, corner), each 1/8 of the CV.
    """
    P = lambda da, db: phi[b + db, a + da]
    c = P(0, 0)
    ring = [P(1, 0), P(1, 1), P(0, 1), P(-1, 1), P(-1, 0), P(-1, -1), P(0, -1), P(1, -1)]
    total = 0.0
    for t in range(8):
        total = total + triangle_fraction(np.stack([c, ring[t], ring[(t + 1) % 8]], axis=-1))
    return _by_signs(np.stack([c] + ring, axis=-1), total / 8.0)


def _by_signs(vals, frac):
    """Uniform-sign CVs are exactly 0 (no value < 0) or 1 (no value > 0).
    (The simplex formulas give the same, so this only skips work.)  Mixed CVs
    keep the computed value, which may underflow to 0 for a vanishing sliver;
    every later W > 0 test is on this value."""
    neg = (vals < 0).any(axis=-1)
    pos = (vals > 0).any(axis=-1)
    return np.where(~neg, 0.0, np.where(~pos, 1.0, frac))


def cv_fraction_3d(phi, a, b, c):
    """Fraction of {phi < 0} in the CVs centred at lattice points (a, b, c).

    ``phi`` is lattice-shaped (index [c, b, a]).  Each of the 6 CV faces is
    cut into 4 triangles (face centre, two consecutive corners); with the CV
    centre they form 24 tetrahedra of volume 1/24 of the CV.
    """
    P = lambda da, db, dc: phi[c + dc, b + db, a + da]
    centre = P(0, 0, 0)
    total = 0.0
    for axis in range(3):
        for sgn in (-1, 1):
            off = [0, 0, 0]
            off[axis] = sgn
            fc = P(*off)
            u_ax, v_ax = [d for d in range(3) if d != axis]
            loop = [(-1, -1), (1, -1), (1, 1), (-1, 1)]
            corners = []
            for du, dv in loop:
                o = list(off)
                o[u_ax], o[v_ax] = du, dv
                corners.append(P(*o))
            for t in range(4):
                total = total + tetrahedron_fraction(
                    np.stack([centre, fc, corners[t], corners[(t + 1) % 4]], axis=-1))
    allv = np.stack([P(da, db, dc) for dc in (-1, 0, 1) for db in (-1, 0, 1) for da in (-1, 0, 1)], axis=-1)
    return _by_signs(allv, total / 24.0)


def cv_fraction(phi, idx):
    """Dispatch on dimension: ``idx`` is (a, b) or (a, b, c)."""
    if len(idx) == 2:
        return cv_fraction_2d(phi, *idx)
    return cv_fraction_3d(phi, *idx)
