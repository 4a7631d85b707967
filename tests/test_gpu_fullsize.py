"""Parity at the benchmark sizes, in the benchmark's launch configuration.

* 2D 1024^2 Gaussian-bump workload: the oracle assembles the whole system
  (about 3.1 M unknowns).  Fractions and masks must be bit-exact, the FP32
  apply must match A x entry by entry, and the benchmark's solve (FP32 inner
  CG with the Schwarz preconditioner inside FP64 refinement) must reach a
  true relative residual of 1e-8 as the oracle recomputes it, and its
  velocities must match the oracle's sparse direct solve at 4,096 stored
  seeded faces within 1e-6 of max |u| (measured on a GB300: 7.8e-8; plain
  FP64 PCG stopped at 1e-8: 4.5e-8).
* 3D 256^3 falling column (about 1e8 unknown slots, 0.4 % active): the
  oracle cannot assemble the full grid, but every liquid unknown lies in a
  34 x 160 x 34-cell window with at least three cells of air (or solid floor)
  around it, and on such a window the system is the same (the window's own
  wall only touches inactive unknowns).  The GPU solves the full grid; the
  oracle builds the window system, and the GPU's fractions, activity and
  solution are checked there (fractions to 1e-12: the window's lattice
  coordinates round differently from the full grid's), and the velocities
  at 4,096 stored faces of the oracle's solve of the window within 1e-6 of
  max |u|."""
import numpy as np
import pytest

from gpu_common import (abs_matvec, face_flags, golden_velocity_samples, gpu_apply_fields, gpu_context,
                        oracle_system, require_gpu)
from oracle import grid as G
from oracle import solve as So

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _solve(ctx, dev, mode, precond, tol=1e-8):
    from paper_1010_2832_gb300 import learned
    return learned.solve(ctx, dev, mode=mode, precond=precond, tol=tol)


def test_bumps1024_full_system():
    require_gpu()
    from paper_1010_2832_gb300 import workloads as W
    wl = W.bumps_2d(1024, seed=2)
    S = oracle_system(wl)
    ctx, dev = gpu_context(wl)
    kinds = list(S.W_L.keys())
    assert np.array_equal(ctx.export(0).cpu().numpy(), np.concatenate([S.W_L[k] for k in kinds]))
    assert np.array_equal(ctx.export(1).cpu().numpy(), np.concatenate([S.W_F[k] for k in kinds]))
    assert np.array_equal(ctx.export(2).cpu().numpy() & 15, face_flags(S))
    assert np.array_equal(ctx.export(3).cpu().numpy().astype(bool), S.active)
    x = np.random.default_rng(9).uniform(-1, 1, S.A.shape[0])
    y = gpu_apply_fields(ctx, x, 1)
    assert np.all(np.abs(y - S.A @ x) <= 1e-5 * abs_matvec(S.A, x) + 1e-300)
    st, ms, (u, taus, p) = _solve(ctx, dev, 1, 2)
    assert st["status"] == 0, st
    xs = torch.cat(taus + [p]).cpu().numpy()
    assert So.relative_residual(S.A, xs, S.b) <= 1.01e-8
    idx, val, scale = golden_velocity_samples("bumps1024")
    uu = torch.cat([a.reshape(-1) for a in u]).cpu().numpy()
    assert np.abs(uu[idx] - val).max() <= 1e-6 * scale


def _window_slices(kind, w):
    i0, j0, k0, ni, nj, nk = w
    shp = G.field_shape(kind, ni, nj, nk)
    return (slice(k0, k0 + shp[0]), slice(j0, j0 + shp[1]), slice(i0, i0 + shp[2]))


def test_column256_on_its_liquid_window():
    require_gpu()
    from paper_1010_2832_gb300 import workloads as W
    n = 256
    win = (111, 0, 111, 34, 160, 34)
    full = W.column_3d(n)
    ctx, dev = gpu_context(full)
    wl_w = W.column_3d(n, window=win)
    S = oracle_system(wl_w)
    kinds = G.KINDS_3D
    sizes_full = [int(np.prod(G.field_shape(k, n, n, n))) for k in kinds]
    WL = np.split(ctx.export(0).cpu().numpy(), np.cumsum(sizes_full)[:-1])
    for kd, a in zip(kinds, WL):
        sub = a.reshape(G.field_shape(kd, n, n, n))[_window_slices(kd, win)].ravel()
        assert np.abs(sub - S.W_L[kd]).max() <= 1e-12
    # activity: every active unknown of the full grid lies in the window and
    # matches the window system's
    names = ["cell", "cell", "exy", "exz", "eyz", "cell"]
    sizes_u = [int(np.prod(G.field_shape(k, n, n, n))) for k in names]
    act = np.split(ctx.export(3).cpu().numpy().astype(bool), np.cumsum(sizes_u)[:-1])
    wact, o = [], 0
    for kd, a in zip(names, act):
        full_a = a.reshape(G.field_shape(kd, n, n, n))
        sub = full_a[_window_slices(kd, win)]
        assert sub.sum() == full_a.sum()
        wact.append(sub.ravel())
    assert np.array_equal(np.concatenate(wact), S.active)
    # the benchmark's 3D solve (FP32 inner Jacobi-CG, FP64 refinement)
    st, ms, (u, taus, p) = _solve(ctx, dev, 1, 0)
    assert st["status"] == 0, st
    parts = []
    for kd, t in zip(names, taus + [p]):
        parts.append(t.cpu().numpy().reshape(G.field_shape(kd, n, n, n))[_window_slices(kd, win)].ravel())
    xw = np.concatenate(parts)
    assert So.relative_residual(S.A, xw, S.b) <= 1.01e-8
    # velocities against the oracle's solve of the window (stored at 4,096
    # seeded faces), indices mapped from the window's faces to the grid's
    import bench
    idx, val, scale = golden_velocity_samples("column256")
    uu = torch.cat([a.reshape(-1) for a in u]).cpu().numpy()
    assert np.abs(uu[bench.window_face_to_full(idx, n, win)] - val).max() <= 1e-6 * scale
