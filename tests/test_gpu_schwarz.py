"""Additive Schwarz preconditioner (2D) against its definition written out
in the oracle (dense FP64 local solves), and solves with it.

The GPU stores the local inverses in BF16 (8-bit mantissa) and accumulates in
FP32, so the preconditioned vector agrees with the FP64 definition to about
1e-2 relative (RMS); the solve itself is still judged by the FP64 true
residual."""
import numpy as np
import pytest

from gpu_common import gpu_context, oracle_system, require_gpu
from oracle import solve as So
from oracle import system as S_
from paper_1010_2832_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {"bumps40": lambda: W.bumps_2d(40, seed=31), "rand37x23": lambda: W.random_small((37, 23), seed=3),
         "disk32": lambda: W.disk_in_box(32)}


@pytest.mark.parametrize("name", list(CASES))
def test_schwarz_matches_definition(name):
    require_gpu()
    wl = CASES[name]()
    S = oracle_system(wl)
    ctx, dev = gpu_context(wl)
    rng = np.random.default_rng(4)
    r = rng.normal(size=S.A.shape[0])
    z_ref = So.additive_schwarz(S, r)
    rs = ctx.fields_to_slots(torch.from_numpy(r).cuda()).to(torch.float32)
    zs = ctx.new_vector(torch.float32)
    ctx.apply_preconditioner(2, rs, zs)
    z = ctx.slots_to_fields(zs.to(torch.float64)).cpu().numpy()
    act = S.active
    err = np.sqrt(np.mean((z - z_ref)[act] ** 2)) / np.sqrt(np.mean(z_ref[act] ** 2))
    assert err < 1.5e-2, err
    assert np.array_equal(z[~act], r[~act].astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("name", ["bumps40", "rand37x23"])
def test_schwarz_solve_reaches_fp64_residual_with_fewer_iterations(name):
    require_gpu()
    from paper_1010_2832_gb300 import learned, stokes
    wl = CASES[name]()
    S = oracle_system(wl)
    ctx, dev = gpu_context(wl)
    st_s, _, out = learned.solve(ctx, dev, mode=1, precond=2, tol=1e-8)
    st_j, _, _ = learned.solve(ctx, dev, mode=1, precond=0, tol=1e-8)
    assert st_s["status"] == 0, st_s
    x = torch.cat(out[1] + [out[2]]).cpu().numpy()
    assert So.relative_residual(S.A, x, S.b) <= 1.01e-8
    assert st_s["iterations"] < st_j["iterations"], (st_s, st_j)
    x_ref = So.solve_direct(S.A, S.b, S_.pressure_null_vectors(S))
    u_ref = S_.recover_velocity(S, x_ref)
    u = torch.cat([a.reshape(-1) for a in out[0]]).cpu().numpy()
    lv = S.live
    assert np.abs(u - u_ref)[lv].max() <= 1e-3 * np.abs(u_ref[lv]).max()
