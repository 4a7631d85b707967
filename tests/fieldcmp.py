"""Comparison of a coarse solution with a fine numerical one (the 3D
convergence study of Section 9, which measures errors against a 155^3
solution): the fine field is interpolated multilinearly to the coarse
samples over its active samples only (the weights of inactive corners are
dropped and the rest renormalised; a point with no active corner is
skipped), and the errors are the maximum and the integral sum |e| h^d over
the coarse samples that are active.  Plain numpy; no part of the method."""
import numpy as np


def sample_axes(kind, n, h, origin):
    """Per-axis coordinates (x, y[, z]) of the samples of ``kind``."""
    from paper_1010_2832_gb300 import workloads as W
    off = (W._OFF2 if len(n) == 2 else W._OFF3)[kind]
    shp = W.field_shape(kind, n)
    dim = len(n)
    return [origin[d] + (2 * np.arange(shp[dim - 1 - d]) + off[d] - 1) * (h / 2) for d in range(dim)]


def interp_active(field, active, axes, pts):
    """Multilinear interpolation of ``field`` (numpy shape slowest axis first,
    sample coordinates ``axes`` per dimension, x first) at points pts (N, d),
    over the samples where ``active``; NaN where no corner is active.  Points
    outside the samples' box are clamped onto it."""
    dim = len(axes)
    idx, frac = [], []
    for d in range(dim):
        a = axes[d]
        s = (pts[:, d] - a[0]) / (a[1] - a[0])
        s = np.clip(s, 0.0, len(a) - 1.0)
        i0 = np.minimum(np.floor(s).astype(np.int64), len(a) - 2)
        idx.append(i0)
        frac.append(s - i0)
    num = np.zeros(len(pts))
    den = np.zeros(len(pts))
    for corner in range(1 << dim):
        w = np.ones(len(pts))
        ii = []
        for d in range(dim):
            bit = (corner >> d) & 1
            w = w * (frac[d] if bit else 1.0 - frac[d])
            ii.append(idx[d] + bit)
        sel = tuple(reversed(ii))          # numpy order: slowest axis first
        m = active[sel]
        num += np.where(m, w * field[sel], 0.0)
        den += np.where(m, w, 0.0)
    out = np.full(len(pts), np.nan)
    ok = den > 1e-12
    out[ok] = num[ok] / den[ok]
    return out


def errors(coarse, coarse_active, coarse_axes, fine, fine_active, fine_axes, h):
    """(L_inf, L1 = sum |e| h^d, compared count) over the active coarse samples."""
    dim = len(coarse_axes)
    g = np.meshgrid(*reversed(coarse_axes), indexing="ij")
    pts = np.stack([g[dim - 1 - d].ravel() for d in range(dim)], axis=1)
    sel = np.asarray(coarse_active, dtype=bool).ravel()
    ref = interp_active(fine, np.asarray(fine_active, dtype=bool), fine_axes, pts[sel])
    e = np.abs(coarse.ravel()[sel] - ref)
    e = e[~np.isnan(e)]
    return float(e.max()), float(e.sum() * h ** dim), int(e.size)
