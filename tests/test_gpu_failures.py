"""Failure paths of the solver, through the C ABI, none of which faults,
traps or hangs the GPU:

* a NaN in the input velocity gives STOKES_ERR_NONFINITE;
* an iteration cap gives STOKES_ERR_NOT_CONVERGED with an x that reduced
  the true FP64 residual, and the reported residual is that x's;
* the bounded wait of the Schwarz local solves, run out on purpose with the
  options' test hook (a factor copy that is never issued), gives
  STOKES_ERR_TIMEOUT, and the same context then solves normally.
"""
import numpy as np
import pytest

from gpu_common import gpu_context, oracle_system, require_gpu
from oracle import solve as So
from oracle import system as S_
from paper_1010_2832_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _outputs(ctx, wl, dev):
    from paper_1010_2832_gb300 import stokes  # noqa: F401
    nx, ny = wl.n
    u = [torch.zeros_like(t) for t in dev["u_star"]]
    taus = [torch.zeros(nx * ny, dtype=torch.float64, device="cuda"),
            torch.zeros((nx + 1) * (ny + 1), dtype=torch.float64, device="cuda")]
    p = torch.zeros(nx * ny, dtype=torch.float64, device="cuda")
    return u, taus, p


def test_nan_input_velocity_is_reported_nonfinite():
    require_gpu()
    from paper_1010_2832_gb300 import stokes
    wl = W.bumps_2d(64, seed=11)
    ctx, dev = gpu_context(wl)
    u, taus, p = _outputs(ctx, wl, dev)
    us = [t.clone() for t in dev["u_star"]]
    us[0].view(-1)[us[0].numel() // 2] = float("nan")
    for opt in (stokes.default_options(mode=0), stokes.default_options(mode=1, precond=2)):
        with pytest.raises(stokes.StokesError) as ei:
            ctx.solve_step(us, u, taus, p, opt)
        assert ei.value.status == -7                     # STOKES_ERR_NONFINITE
        assert "non-finite" in str(ei.value)


def test_iteration_cap_reports_not_converged_with_the_reached_residual():
    require_gpu()
    from paper_1010_2832_gb300 import stokes
    wl = W.bumps_2d(64, seed=12)
    ctx, dev = gpu_context(wl)
    b = ctx.new_vector()
    x = ctx.new_vector()
    ctx.rhs(dev["u_star"], b)
    st = ctx.solve_system(b, x, stokes.default_options(mode=0, max_iter=5, check_every=1))
    assert st.status == -3                               # STOKES_ERR_NOT_CONVERGED
    assert st.iterations == 5
    # the reported residual is that of the returned x
    r = ctx.new_vector()
    ctx.apply(x, r)
    rel = float(torch.linalg.norm(b - r) / torch.linalg.norm(b))
    assert np.isfinite(rel) and rel > 1e-8
    assert abs(rel - st.rel_residual) <= 1e-6 * rel
    # CG's iterate is the best one so far in the energy norm: its error
    # against the oracle's direct solve is below that of x = 0
    S = oracle_system(wl)
    xs = So.solve_direct(S.A, S.b, S_.pressure_null_vectors(S))
    xg = ctx.slots_to_fields(x).cpu().numpy()
    e = xg - xs
    assert e @ (S.A @ e) < 0.9 * (xs @ (S.A @ xs))


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    require_gpu()
    from paper_1010_2832_gb300 import stokes
    wl = W.bumps_2d(96, seed=13)
    ctx, dev = gpu_context(wl)
    u, taus, p = _outputs(ctx, wl, dev)
    opt = stokes.default_options(mode=1, precond=2, wait_test=1)
    with pytest.raises(stokes.StokesError) as ei:
        ctx.solve_step(dev["u_star"], u, taus, p, opt)
    assert ei.value.status == -5                         # STOKES_ERR_TIMEOUT
    # the hook holds for that call only: the next solve on the same context
    # converges and matches a solve on a fresh context
    st = ctx.solve_step(dev["u_star"], u, taus, p, stokes.default_options(mode=1, precond=2))
    assert st.status == 0 and st.rel_residual <= 1e-8
    ctx2, dev2 = gpu_context(wl)
    u2, taus2, p2 = _outputs(ctx2, wl, dev2)
    st2 = ctx2.solve_step(dev2["u_star"], u2, taus2, p2, stokes.default_options(mode=1, precond=2))
    assert st2.status == 0
    assert st.iterations == st2.iterations
    for a, c in zip(u, u2):
        assert torch.equal(a, c)


def test_wait_test_outside_its_range_is_refused():
    require_gpu()
    from paper_1010_2832_gb300 import stokes
    wl = W.bumps_2d(32, seed=14)
    ctx, dev = gpu_context(wl)
    u, taus, p = _outputs(ctx, wl, dev)
    with pytest.raises(stokes.StokesError) as ei:
        ctx.solve_step(dev["u_star"], u, taus, p, stokes.default_options(wait_test=2))
    assert ei.value.status == -1                         # STOKES_ERR_ARG
