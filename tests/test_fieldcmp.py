"""Pins of the coarse-versus-fine comparison (tests/fieldcmp.py): exact on
multilinear fields when every sample is active, exact on constants with any
activity mask, the integral norm of a constant error is that constant times
the active volume, and the sample axes sit where the layout puts them."""
import numpy as np

from fieldcmp import errors, interp_active, sample_axes
from paper_1010_2832_gb300 import workloads as W


def test_sample_axes_match_the_layout():
    n, h, o = (5, 4, 3), 0.2, (-0.5, 0.1, 0.3)
    for kind in ("cell", "u", "v", "w", "exy", "exz", "eyz"):
        P = W.sample_points(kind, n, h, o)
        ax = sample_axes(kind, n, h, o)
        assert np.allclose(P[0][0, 0, :], ax[0]) and np.allclose(P[1][0, :, 0], ax[1])
        assert np.allclose(P[2][:, 0, 0], ax[2])


def test_trilinear_field_is_reproduced_exactly():
    rng = np.random.default_rng(0)
    n, h, o = (7, 6, 5), 0.3, (-1.0, -0.7, 0.2)
    ax = sample_axes("exz", n, h, o)
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    f = lambda x, y, z: 1 + 2 * x - y + 0.5 * z + 0.3 * x * y - 0.2 * y * z + 0.7 * x * z + 0.1 * x * y * z
    pts = np.stack([rng.uniform(ax[d][0], ax[d][-1], 500) for d in range(3)], axis=1)
    got = interp_active(f(X, Y, Z), np.ones(X.shape, bool), ax, pts)
    assert np.abs(got - f(pts[:, 0], pts[:, 1], pts[:, 2])).max() < 1e-12


def test_masked_constant_and_integral_norm():
    rng = np.random.default_rng(1)
    n, h, o = (9, 8, 7), 0.25, (0.0, 0.0, 0.0)
    ax = sample_axes("cell", n, h, o)
    shape = W.field_shape("cell", n)
    act = rng.random(shape) < 0.5
    fine = np.where(act, 3.25, 1e9)                  # inactive values must not leak
    pts = np.stack([rng.uniform(ax[d][0], ax[d][-1], 400) for d in range(3)], axis=1)
    got = interp_active(fine, act, ax, pts)
    assert np.all(np.isnan(got) | (np.abs(got - 3.25) < 1e-12)) and np.isfinite(got).sum() > 300
    # coarse = fine grid itself plus a constant offset: L_inf = offset, L1 = offset * active volume
    cact = np.ones(shape, bool)
    linf, l1, cnt = errors(np.full(shape, 3.5), cact, ax, np.full(shape, 3.25), np.ones(shape, bool), ax, h)
    assert abs(linf - 0.25) < 1e-12 and abs(l1 - 0.25 * cnt * h ** 3) < 1e-12 and cnt == cact.sum()
