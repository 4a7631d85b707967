"""Learned preconditioner inside flexible CG: with any network the solve must
still reach the FP64 true residual (the flexible method plus the Jacobi
fallback and the FP64 refinement guarantee it); a network trained on
solver-generated pairs is compared, on held-out instances, with the same
mixed-precision solve preconditioned by Jacobi alone (the method without the
network) and by the untrained network.  Iterations and times are recorded
(and written to $STOKES_RESULTS_DIR/learned_vs_jacobi.json when set)."""
import json
import os

import numpy as np
import pytest

from gpu_common import oracle_system, require_gpu
from oracle import solve as So

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_fpcg_with_untrained_network_converges():
    require_gpu()
    from paper_1010_2832_gb300 import learned, stokes, workloads as W
    wl = W.bumps_2d(40, seed=21)
    ctx, dev = stokes.context_for(wl)
    D, H, Wd, cin, cout = stokes.learned_grid(ctx)
    net = stokes.Net(2, cin, cout, D * H * Wd)
    from oracle import unet as U
    net.set_params(net.from_oracle_layout(U.init_params(2, cin, cout, seed=0)))
    stokes.attach_network(ctx, net)
    st, ms, (u, taus, p) = learned.solve(ctx, dev, mode=1, precond=1, tol=1e-8)
    assert st["status"] == 0, st
    S = oracle_system(wl)
    x = torch.cat(taus + [p]).cpu().numpy()
    assert So.relative_residual(S.A, x, S.b) <= 1.01e-8


def test_trained_network_vs_jacobi(tmp_path):
    require_gpu()
    from paper_1010_2832_gb300 import learned, stokes, workloads as W
    n = 44
    train_wls = [W.bumps_2d(n, seed=500 + i, rho_split=False) for i in range(6)]
    data = []
    shape = None
    net = None
    for i, wl in enumerate(train_wls):
        ctx, dev = stokes.context_for(wl)
        D, H, Wd, cin, cout = stokes.learned_grid(ctx)
        if net is None:
            net = stokes.Net(2, cin, cout, 8 * D * H * Wd)
            from oracle import unet as U
            net.set_params(net.from_oracle_layout(U.init_params(2, cin, cout, seed=1)))
            shape = (D, H, Wd)
        stokes.attach_network(ctx, net)
        xs, ys = learned.make_pairs(ctx, wl, 12, seed0=1000 * i)
        data += list(zip(xs, ys))
    net0 = stokes.Net(2, cin, cout, 8 * shape[0] * shape[1] * shape[2])
    net0.set_params(net.get_params())          # the untrained starting point
    losses = learned.train(net, data, shape, epochs=25, batch=4, lr=2e-3)
    assert losses[-1] < losses[0]
    results = []
    for i in range(3):
        wl = W.bumps_2d(n, seed=900 + i, rho_split=False)
        ctx, dev = stokes.context_for(wl)
        S = oracle_system(wl)
        row = {}
        for name, prec, use in (("learned", 1, net), ("untrained", 1, net0), ("jacobi", 0, None)):
            if use is not None:
                stokes.attach_network(ctx, use)
            st, ms, out = learned.solve(ctx, dev, mode=1, precond=prec, max_iter=30000)
            row[name + "_status"] = st["status"]
            if name != "untrained":       # a random network may well not converge in the budget
                assert st["status"] == 0, (name, st)
                x = torch.cat(out[1] + [out[2]]).cpu().numpy()
                assert So.relative_residual(S.A, x, S.b) <= 1.01e-8, name
            row[name + "_iters"] = st["iterations"]
            row[name + "_ms"] = ms
            row[name + "_jacobi_fallback_steps"] = stokes.learned_jacobi_steps(ctx) if prec == 1 else 0
        results.append(row)
    out_dir = os.environ.get("STOKES_RESULTS_DIR")
    if out_dir:
        with open(os.path.join(out_dir, "learned_vs_jacobi.json"), "w") as f:
            json.dump(dict(train_loss=losses, results=results), f)
    print("learned vs jacobi:", results)


def test_trained_network_3d_vs_jacobi_and_plain_fp64():
    """Config 5 at reduced scale (3D Gaussian-bump instances: training on 24^3,
    evaluation on a held-out 32^3 instance): the trained network, the
    untrained one, Jacobi alone (same mixed-precision solve) and plain FP64
    Jacobi-PCG, on iterations and wall time.  These systems are stiff (tens
    of thousands of Jacobi iterations).  The learned solve must converge like
    the others; the comparison is recorded, not assumed."""
    require_gpu()
    from paper_1010_2832_gb300 import learned, stokes, workloads as W
    from oracle import unet as U
    train_wls = [W.bumps_3d(24, seed=5000 + i) for i in range(4)]
    eval_wls = [W.bumps_3d(32, seed=9000)]
    grids = []
    for wl in train_wls[:1] + eval_wls[:1]:
        ctx, dev = stokes.context_for(wl)
        grids.append(stokes.learned_grid(ctx))
    (Dt, Ht, Wt, cin, cout), (De, He, We, _, _) = grids
    net = stokes.Net(3, cin, cout, max(4 * Dt * Ht * Wt, De * He * We))
    net.set_params(net.from_oracle_layout(U.init_params(3, cin, cout, seed=3)))
    net0 = stokes.Net(3, cin, cout, De * He * We)
    net0.set_params(net.get_params())
    data = []
    for i, wl in enumerate(train_wls):
        ctx, dev = stokes.context_for(wl)
        stokes.attach_network(ctx, net)
        xs, ys = learned.make_pairs(ctx, wl, 10, seed0=2000 * (i + 1))
        data += list(zip(xs, ys))
    losses = learned.train(net, data, (Dt, Ht, Wt), epochs=10, batch=4, lr=2e-3)
    assert all(np.isfinite(losses))
    results = []
    for wl in eval_wls:
        ctx, dev = stokes.context_for(wl)
        row = {}
        for name, mode, prec, use in (("learned", 1, 1, net), ("untrained", 1, 1, net0), ("jacobi_fp32", 1, 0, None),
                                      ("plain_fp64", 0, 0, None)):
            if use is not None:
                stokes.attach_network(ctx, use)
            st, ms, _ = learned.solve(ctx, dev, mode=mode, precond=prec, max_iter=400000)
            row[name] = dict(status=st["status"], iterations=st["iterations"], ms=ms, rel=st["rel_residual"],
                             jacobi_fallback_steps=stokes.learned_jacobi_steps(ctx) if prec == 1 else 0)
            if name != "untrained":
                assert st["status"] == 0 and st["rel_residual"] <= 1.01e-8, (name, st)
        results.append(row)
    out_dir = os.environ.get("STOKES_RESULTS_DIR")
    if out_dir:
        with open(os.path.join(out_dir, "learned_3d.json"), "w") as f:
            json.dump(dict(train_loss=losses, results=results), f)
    print("learned 3D:", results)
