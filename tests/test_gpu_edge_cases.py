"""Degenerate inputs through the C ABI: a grid with no liquid, a liquid
region of a few cells, and liquid that fills the box up to its walls.
No liquid: the system is empty, the solve returns at once (0 iterations)
with the oracle's velocities for x = 0 (u_BC on solid faces, u* on the
others), and the apply is the identity.  A few cells: the FP64 solve
matches the oracle's direct solve to 1e-9 and the Schwarz-preconditioned
mixed solve reaches the FP64 residual."""
import numpy as np
import pytest

from gpu_common import gpu_context, oracle_system, require_gpu, to_gpu
from oracle import solve as So
from oracle import system as S_
from paper_1010_2832_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _outputs(ctx, dev):
    nx, ny = ctx.n[0], ctx.n[1]
    outs = [torch.zeros_like(t) for t in dev["u_star"]]
    taus = [torch.zeros(nx * ny, dtype=torch.float64, device="cuda"),
            torch.zeros((nx + 1) * (ny + 1), dtype=torch.float64, device="cuda")]
    p = torch.zeros(nx * ny, dtype=torch.float64, device="cuda")
    return outs, taus, p


@pytest.mark.parametrize("mode,precond", [(0, 1), (1, 2)])
def test_no_liquid_is_an_empty_solve_and_apply_is_identity(mode, precond):
    require_gpu()
    from paper_1010_2832_gb300 import stokes
    wl = W.disk_in_box(24, radius=-0.1)          # the level set is positive everywhere
    S = oracle_system(wl)
    assert not S.active.any()
    ctx, dev = gpu_context(wl)
    outs, taus, p = _outputs(ctx, dev)
    st = ctx.solve_step(dev["u_star"], outs, taus, p, stokes.default_options(mode=mode, precond=precond))
    assert st.status == 0 and st.iterations == 0
    u = torch.cat([o.reshape(-1) for o in outs]).cpu().numpy()
    assert np.array_equal(u, S_.recover_velocity(S, np.zeros(S.A.shape[0])))
    assert not torch.cat(taus + [p]).any()
    x = np.random.default_rng(1).uniform(-1, 1, S.A.shape[0])
    xs = ctx.fields_to_slots(to_gpu(x))
    ys = ctx.new_vector()
    ctx.apply(xs, ys, stokes.FP64)
    assert np.array_equal(ctx.slots_to_fields(ys).cpu().numpy(), x)


@pytest.mark.parametrize("radius", [0.05, 0.09])
def test_few_liquid_cells_match_oracle(radius):
    require_gpu()
    from paper_1010_2832_gb300 import stokes
    wl = W.disk_in_box(24, radius=radius)        # 1.2 and 2.2 cells of radius
    S = oracle_system(wl)
    assert 0 < S.active.sum() < 200
    ctx, dev = gpu_context(wl)
    outs, taus, p = _outputs(ctx, dev)
    st = ctx.solve_step(dev["u_star"], outs, taus, p, stokes.default_options(mode=stokes.FP64, tol=1e-12))
    assert st.status == 0
    x_ref = So.solve_direct(S.A, S.b, S_.pressure_null_vectors(S))
    u_ref = S_.recover_velocity(S, x_ref)
    u = torch.cat([o.reshape(-1) for o in outs]).cpu().numpy()
    lv = S.live
    assert np.abs(u - u_ref)[lv].max() <= 1e-9 * max(np.abs(u_ref[lv]).max(), 1e-30)
    st2 = ctx.solve_step(dev["u_star"], outs, taus, p, stokes.default_options(mode=stokes.FP32, precond=2, tol=1e-10))
    assert st2.status == 0
    x = torch.cat(taus + [p]).cpu().numpy()
    assert So.relative_residual(S.A, x, S.b) <= 1.01e-10


def test_liquid_touching_the_walls_matches_oracle():
    """A disk larger than the box: liquid fills every cell up to the walls,
    so the patches and tiles at the grid boundary are all active."""
    require_gpu()
    from paper_1010_2832_gb300 import stokes
    wl = W.disk_in_box(37, radius=0.8)
    S = oracle_system(wl)
    ctx, dev = gpu_context(wl)
    outs, taus, p = _outputs(ctx, dev)
    st = ctx.solve_step(dev["u_star"], outs, taus, p, stokes.default_options(mode=stokes.FP32, precond=2, tol=1e-10))
    assert st.status == 0
    x = torch.cat(taus + [p]).cpu().numpy()
    assert So.relative_residual(S.A, x, S.b) <= 1.01e-10
