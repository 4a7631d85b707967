"""Training data, training loop and evaluation of the learned preconditioner.

Pairs come from the solver itself.  A seeded start error e0 on the active
unknowns (white noise or a sum of smooth Fourier modes) defines b = A e0;
k iterations of Jacobi-preconditioned CG on A x = b from x = 0 leave the
error e = e0 - x_k, rich in exactly the components Jacobi-PCG is slow to
remove (k = 0 keeps e0).  The residual is r = A e.  The preconditioner
adds a network correction to the Jacobi step, so the training target is
the part of e that the Jacobi step misses, e - M_J r, scaled as
stokes_learned_targets describes.  Everything runs on the GPU through the
C ABI; the random fields are seeded inputs built on the host.
"""
import time

import numpy as np
import torch

from . import stokes, workloads

_KINDS = {2: ("cell", "node", "cell"), 3: ("cell", "cell", "exy", "exz", "eyz", "cell")}


def smooth_error(ctx, wl, seed, modes=6):
    """Seeded smooth random error in FP64 slot layout, zero on inactive
    unknowns: a sum of random Fourier modes per unknown field."""
    rng = np.random.default_rng(seed)
    act = ctx.export(3).cpu().numpy().astype(bool)
    parts = []
    for kind in _KINDS[wl.dim]:
        P = workloads.sample_points(kind, wl.n, wl.h, wl.origin)
        f = np.zeros(P[0].shape)
        for _ in range(modes):
            k = rng.integers(1, 6, wl.dim)
            ph = rng.uniform(0, 2 * np.pi)
            arg = sum(2 * np.pi * k[d] * P[d] for d in range(wl.dim)) + ph
            f += rng.normal() * np.sin(arg)
        parts.append(f.ravel())
    e = np.concatenate(parts) * act
    return ctx.fields_to_slots(torch.from_numpy(e).cuda())


def white_error(ctx, seed):
    """Seeded white-noise error in FP64 slot layout, zero on inactive unknowns."""
    rng = np.random.default_rng(seed)
    act = ctx.export(3).cpu().numpy().astype(bool)
    e = rng.normal(size=act.size) * act
    return ctx.fields_to_slots(torch.from_numpy(e).cuda())


def make_pairs(ctx, wl, n_pairs, seed0, cg_iters=(0, 4, 16, 64, 256)):
    """(features, targets) device tensors for n_pairs solver-generated errors.

    Pair q starts from white noise (even q) or smooth modes (odd q) and runs
    cg_iters[q % len(cg_iters)] Jacobi-PCG iterations on it."""
    xs, ys = [], []
    b = ctx.new_vector()
    x = ctx.new_vector()
    r = ctx.new_vector()
    z32 = ctx.new_vector(torch.float32)
    for q in range(n_pairs):
        e0 = white_error(ctx, seed0 + q) if q % 2 == 0 else smooth_error(ctx, wl, seed0 + q)
        k = cg_iters[q % len(cg_iters)]
        e = e0
        if k > 0:
            ctx.apply(e0, b, stokes.FP64)
            x.zero_()
            ctx.solve_system(b, x, stokes.default_options(mode=stokes.FP64, precond=0, tol=1e-300, max_iter=k))
            e = e0 - x
        ctx.apply(e, r, stokes.FP64)
        feats, rms = stokes.learned_features(ctx, r)
        ctx.apply_preconditioner(0, r.float(), z32)
        ys.append(stokes.learned_targets(ctx, e - z32.double(), rms))
        xs.append(feats)
    return xs, ys


def train(net, data, shape, epochs=20, batch=4, lr=2e-3, seed=0, log=None):
    """Adam on the normalised squared error; data = list of (x, y)."""
    rng = np.random.default_rng(seed)
    B = batch
    D, H, W = shape
    n = len(data)
    losses = []
    for ep in range(epochs):
        order = rng.permutation(n)
        tot = 0.0
        for s in range(0, n - B + 1, B):
            idx = order[s:s + B]
            x = torch.cat([data[i][0] for i in idx])
            y = torch.cat([data[i][1] for i in idx])
            tot += net.train_step(x, y, (B, D, H, W), lr)
        losses.append(tot / max(1, n // B))
        if log:
            log(f"epoch {ep} loss {losses[-1]:.4f}")
    return losses


def solve(ctx, dev, mode, precond, tol=1e-8, max_iter=200000):
    """One implicit step; returns (stats dict, wall ms on the device)."""
    nx, ny = wl_sizes = ctx.n[0], ctx.n[1]
    sizes = _field_sizes(ctx)
    u = [torch.zeros_like(t) for t in dev["u_star"]]
    taus = [torch.zeros(s, dtype=torch.float64, device="cuda") for s in sizes[:-1]]
    p = torch.zeros(sizes[-1], dtype=torch.float64, device="cuda")
    opt = stokes.default_options(mode=mode, tol=tol, precond=precond, max_iter=max_iter)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = ctx.solve_step(dev["u_star"], u, taus, p, opt)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    return st.as_dict(), ms, (u, taus, p)


def _field_sizes(ctx):
    nx, ny = ctx.n[0], ctx.n[1]
    if ctx.dim == 2:
        return [nx * ny, (nx + 1) * (ny + 1), nx * ny]
    nz = ctx.n[2]
    return [nx * ny * nz, nx * ny * nz, nz * (ny + 1) * (nx + 1), (nz + 1) * ny * (nx + 1),
            (nz + 1) * (ny + 1) * nx, nx * ny * nz]


def crop(t, grid, channels, corner, size):
    """A size^3 (3D) or size^2 (2D) window of a flat channel-last tensor on
    the network grid (D, H, W), starting at corner (z, y, x)."""
    D, H, W = grid
    v = t.view(D, H, W, channels)
    z, y, x = corner
    if D == 1:
        return v[:, y:y + size, x:x + size, :].contiguous().view(-1)
    return v[z:z + size, y:y + size, x:x + size, :].contiguous().view(-1)


class _ErrorFields:
    """Seeded random start errors generated on the GPU for one context (the
    field-layout activity mask and sample coordinates are kept on the
    device): white noise, or a sum of smooth random Fourier modes per
    unknown field; zero on inactive unknowns."""

    def __init__(self, ctx, wl):
        act = ctx.export(3).to(torch.bool)
        self.act = act
        pts = []
        for kind in _KINDS[wl.dim]:
            P = workloads.sample_points(kind, wl.n, wl.h, wl.origin)
            pts.append(torch.stack([torch.from_numpy(np.ascontiguousarray(a).ravel()) for a in P]).cuda())
        self.pts = pts
        self.ctx = ctx
        self.dim = wl.dim

    def white(self, seed):
        g = torch.Generator(device="cuda").manual_seed(int(seed))
        e = torch.randn(self.act.numel(), generator=g, device="cuda", dtype=torch.float64) * self.act
        return self.ctx.fields_to_slots(e)

    def smooth(self, seed, modes=6):
        rng = np.random.default_rng(seed)
        parts = []
        for P in self.pts:
            f = torch.zeros(P.shape[1], dtype=torch.float64, device="cuda")
            for _ in range(modes):
                k = rng.integers(1, 6, self.dim)
                ph = rng.uniform(0, 2 * np.pi)
                arg = sum(2 * np.pi * float(k[d]) * P[d] for d in range(self.dim)) + ph
                f += float(rng.normal()) * torch.sin(arg)
            parts.append(f)
        return self.ctx.fields_to_slots(torch.cat(parts) * self.act)


def make_cropped_pairs(ctx, wl, n_pairs, seed0, size, cg_iters=(0, 4, 16, 64, 256)):
    """The pairs of make_pairs (pair q: white-noise or smooth start as q is
    even or odd, cg_iters[q % len] Jacobi-PCG iterations; the start errors
    drawn on the GPU), each cut to a seeded random window of the given size
    (corner on a multiple of 4, so the network's pooling grid is the one it
    has on the whole grid); only the windows are kept.  A window whose
    target is zero (no active unknown in it) is redrawn, up to 64 times."""
    D, H, W, cin, cout = stokes.learned_grid(ctx)
    rng = np.random.default_rng(seed0)
    lim = [(d - size) // 4 for d in (D, H, W)]
    ef = _ErrorFields(ctx, wl)
    out = []
    b = ctx.new_vector()
    x = ctx.new_vector()
    r = ctx.new_vector()
    z32 = ctx.new_vector(torch.float32)
    for q in range(n_pairs):
        e0 = ef.white(seed0 + q) if q % 2 == 0 else ef.smooth(seed0 + q)
        k = cg_iters[q % len(cg_iters)]
        e = e0
        if k > 0:
            ctx.apply(e0, b, stokes.FP64)
            x.zero_()
            ctx.solve_system(b, x, stokes.default_options(mode=stokes.FP64, precond=0, tol=1e-300, max_iter=k))
            e = e0 - x
        ctx.apply(e, r, stokes.FP64)
        feats, rms = stokes.learned_features(ctx, r)
        ctx.apply_preconditioner(0, r.float(), z32)
        targ = stokes.learned_targets(ctx, e - z32.double(), rms)
        for _ in range(64):
            corner = tuple(4 * int(rng.integers(0, m + 1)) if m > 0 else 0 for m in lim)
            yc = crop(targ, (D, H, W), cout, corner, size)
            if float(torch.linalg.norm(yc)) > 0:
                break
        out.append((crop(feats, (D, H, W), cin, corner, size), yc))
        del feats, targ
    return out


def compare_solvers(ctx, dev, net, max_iter=400000):
    """The learned flexible CG (mixed precision), the same solve with Jacobi
    alone, and plain FP64 Jacobi-PCG on one system: status, iterations,
    device and wall time, final true residual."""
    row = {}
    for name, mode, prec in (("learned", stokes.FP32, 1), ("jacobi_fp32", stokes.FP32, 0),
                             ("plain_fp64", stokes.FP64, 0)):
        if prec == 1:
            stokes.attach_network(ctx, net)
        st, ms, _ = solve(ctx, dev, mode=mode, precond=prec, max_iter=max_iter)
        row[name] = dict(status=st["status"], iterations=st["iterations"], ms_device=st["ms_solve"], ms_wall=ms,
                         rel_residual=st["rel_residual"],
                         jacobi_fallback_steps=stokes.learned_jacobi_steps(ctx) if prec == 1 else 0)
    return row


def init_network(net, seed=0):
    """He-uniform weights (limit sqrt(6 / fan_in)), zero biases, in the
    library's parameter layout."""
    rng = np.random.default_rng(seed)
    p = np.zeros(net.n, dtype=np.float32)
    for ci, co, ks, wo, bo in net.layers():
        taps = ks ** net.dim
        lim = np.sqrt(6.0 / (ci * taps))
        p[wo:wo + taps * ci * co] = rng.uniform(-lim, lim, taps * ci * co)
    net.set_params(p)


def config5(n_train=128, instances=20, pairs_per_instance=100, crop_size=64, epochs=30, batch=4, lr=2e-3,
            eval_sizes=(128, 128, 256), eval_seed0=9000, train_seed0=5000, caps=None, floor=0.01, log=None):
    """The learned preconditioner at scale: solver-generated pairs from 3D
    Gaussian-bump instances (seeds train_seed0..), cut to crop_size^3
    windows, train the BF16 U-Net on the tensor cores, then solve held-out
    instances (seeds eval_seed0.., sizes eval_sizes) with the learned
    flexible CG, the same mixed-precision CG with Jacobi alone, and plain
    FP64 Jacobi-PCG, each capped at caps[size] iterations (these systems are
    stiff: plain FP64 Jacobi-PCG needs 2.6e5 iterations at 64^3).  ``floor``
    is the face-mass floor of stokes_set_min_face_liquid for every instance
    (0: the paper's system).  Returns timings, losses and per-instance
    comparisons (status, iterations, device ms, final true residual)."""
    from . import workloads as W
    say = log or (lambda *a: None)
    caps = caps or {128: 100000, 256: 60000}
    t0 = time.perf_counter()
    data = []
    net = None
    # the network grid of an n^3 instance is (n + 1) rounded up to a multiple of 4
    eval_grids = [(s + 4) // 4 * 4 for s in eval_sizes]
    max_vox = max([batch * crop_size ** 3, ((n_train + 4) // 4 * 4) ** 3] + [g ** 3 for g in eval_grids])
    for i in range(instances):
        wl = W.bumps_3d(n_train, seed=train_seed0 + i)
        ctx, dev = stokes.context_for(wl, min_face_liquid=floor)
        if net is None:
            D, H, Wd, cin, cout = stokes.learned_grid(ctx)
            net = stokes.Net(3, cin, cout, max_vox)
            init_network(net, seed=3)
        stokes.attach_network(ctx, net)           # the features are formed on the network's grid
        data += make_cropped_pairs(ctx, wl, pairs_per_instance, seed0=100000 * (i + 1), size=crop_size)
        ctx.close()
        del dev
        torch.cuda.empty_cache()
    t_data = time.perf_counter() - t0
    say(f"pairs: {len(data)} in {t_data:.1f} s")
    t0 = time.perf_counter()
    losses = train(net, data, (crop_size,) * 3, epochs=epochs, batch=batch, lr=lr, log=say)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del data
    torch.cuda.empty_cache()
    rows = []
    for k, size in enumerate(eval_sizes):
        wl = W.bumps_3d(size, seed=eval_seed0 + k)
        ctx, dev = stokes.context_for(wl, min_face_liquid=floor)
        row = dict(n=size, seed=eval_seed0 + k, cap=caps.get(size, 30000),
                   **compare_solvers(ctx, dev, net, max_iter=caps.get(size, 30000)))
        say(f"eval {size}^3: {row}")
        rows.append(row)
        ctx.close()
        del dev
        torch.cuda.empty_cache()
    return dict(pairs=instances * pairs_per_instance, crop=crop_size, instances=instances, n_train=n_train,
                params=int(net.n), epochs=epochs, floor=floor, train_loss=losses, s_pairs=t_data, s_train=t_train,
                eval=rows)
