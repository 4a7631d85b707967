"""Prescribed traction (Section 6.1) on the GPU against the oracle.

stokes_traction_u_star must give the oracle's traction_u_star face by face
(FP64, to 1e-12 of the largest shift) in 2D and 3D, and a uniform surface
pressure on liquid at rest must come out of the full GPU step as the liquid
pressure, with the velocity at rest."""
import numpy as np
import pytest

from gpu_common import gpu_context, oracle_system, require_gpu
from oracle import system as S_
from paper_1010_2832_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _fields(S, x):
    """Unknown-ordered vector -> per-field CUDA tensors (stress kinds, then p)."""
    parts = S_.split_unknowns(S, x)
    names = S_.unknown_names(S.inp.dim)
    t = [torch.from_numpy(np.ascontiguousarray(parts[nm]).ravel()).cuda() for nm in names]
    return t[:-1], t[-1]


@pytest.mark.parametrize("name", ["bumps2d", "rand2d", "rand3d", "bumps3d"])
def test_traction_shift_matches_oracle(name):
    require_gpu()
    wl = {"bumps2d": lambda: W.bumps_2d(40, seed=17),
          "rand2d": lambda: W.random_small((37, 23), seed=3),
          "rand3d": lambda: W.random_small((13, 9, 11), seed=2, dim=3),
          "bumps3d": lambda: W.bumps_3d(16, seed=7)}[name]()
    S = oracle_system(wl)
    ctx, dev = gpu_context(wl)
    rng = np.random.default_rng(12)
    xbc = rng.normal(size=S.A.shape[0])
    ref = S_.traction_u_star(S, xbc)
    tau, p = _fields(S, xbc)
    out = [torch.empty_like(u) for u in dev["u_star"]]
    ctx.traction_u_star(tau, p, dev["u_star"], out)
    got = torch.cat([u.reshape(-1) for u in out]).cpu().numpy()
    shift = np.abs(ref - S.u_star).max()
    assert shift > 0
    assert np.abs(got - ref).max() <= 1e-12 * max(shift, np.abs(ref).max())


def test_uniform_surface_pressure_through_the_gpu_step():
    require_gpu()
    from paper_1010_2832_gb300 import stokes
    wl = W.disk_in_box(48, radius=0.3)
    S = oracle_system(wl)
    ctx, dev = gpu_context(wl)
    P0 = 2.5
    nx, ny = wl.n
    tau = [torch.zeros(nx * ny, dtype=torch.float64, device="cuda"),
           torch.zeros((nx + 1) * (ny + 1), dtype=torch.float64, device="cuda")]
    p_bc = torch.full((nx * ny,), P0, dtype=torch.float64, device="cuda")
    zero = [torch.zeros_like(u) for u in dev["u_star"]]
    ue = [torch.empty_like(u) for u in dev["u_star"]]
    ctx.traction_u_star(tau, p_bc, zero, ue)
    u = [torch.empty_like(x) for x in ue]
    taus = [torch.zeros_like(t) for t in tau]
    p = torch.zeros_like(p_bc)
    st = ctx.solve_step(ue, u, taus, p, stokes.default_options(mode=0, tol=1e-12))
    assert st.status == 0
    act = S_.split_unknowns(S, S.active.astype(float))
    pa = p.cpu().numpy()[act["p"].ravel() > 0]
    assert pa.size > 0 and np.abs(pa - P0).max() <= 1e-8 * P0
    for t in taus:
        assert t.abs().max().item() <= 1e-8 * P0
    assert max(x.abs().max().item() for x in u) <= 1e-8 * P0 * wl.dt / wl.h
