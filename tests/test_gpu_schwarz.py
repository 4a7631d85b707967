"""Additive Schwarz preconditioner (2D) against its definition written out
in the oracle (dense FP64 local solves), and solves with it.

The GPU assembles each local matrix in FP64, factors the unit-diagonal
matrix in FP32, stores the inverse X = L^-1 of the factor in FP16 with a
FP32 scale per row and applies D^-1/2 X^T X D^-1/2 with FP32
accumulation, so the preconditioned vector agrees with the FP64 definition to about 1e-2 relative (RMS; the
error concentrates in the worst-conditioned patches) while the
preconditioner stays symmetric positive definite (checked on random
vectors).  The solve is judged by the FP64 true residual; it must stay in
FP32 (no precision escalation) and take far fewer iterations than Jacobi."""
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
    # symmetric positive definite on the active unknowns
    vs, zs_ = [], []
    for q in range(4):
        v = rng.normal(size=S.A.shape[0]) * act
        zq = ctx.new_vector(torch.float32)
        ctx.apply_preconditioner(2, ctx.fields_to_slots(torch.from_numpy(v).cuda()).to(torch.float32), zq)
        vs.append(v)
        zs_.append(ctx.slots_to_fields(zq.to(torch.float64)).cpu().numpy())
    for a in range(4):
        assert vs[a] @ zs_[a] > 0
        for b in range(a):
            scale = np.linalg.norm(vs[a]) * np.linalg.norm(zs_[b]) + np.linalg.norm(vs[b]) * np.linalg.norm(zs_[a])
            assert abs(vs[a] @ zs_[b] - vs[b] @ zs_[a]) <= 1e-5 * scale


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
    assert st_s["precision_used"] == stokes.FP32, st_s
    assert 3 * st_s["iterations"] < st_j["iterations"], (st_s, st_j)
    x_ref = So.solve_direct(S.A, S.b, S_.pressure_null_vectors(S))
    u_ref = S_.recover_velocity(S, x_ref)
    u = torch.cat([a.reshape(-1) for a in out[0]]).cpu().numpy()
    lv = S.live
    # ten times the error measured on a GB300 (bumps40 2.1e-8, rand37x23
    # 1.8e-7): set by the 1e-8 stopping test, as for plain FP64 PCG
    tol = {"bumps40": 3e-7, "rand37x23": 2e-6}[name]
    assert np.abs(u - u_ref)[lv].max() <= tol * np.abs(u_ref[lv]).max()
