"""Parity of the transport stage (stokes_advect) with the FP64 reference
oracle.advect: velocity extension, semi-Lagrangian advection of the MAC
velocity plus gravity, and of the half-lattice level set (Section
"Application to Viscous Jet Buckling").  Both sides round every operation
in the same order, so the comparison is to a few ulps of the field scale;
the number of bit-identical samples is reported."""
import numpy as np
import pytest

from gpu_common import oracle_system, require_gpu, to_gpu
from oracle import advect as Ad
from oracle import system as Sy

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

G = (0.3, -9.81)


def _ctx(n, h, dt):
    from paper_1010_2832_gb300 import stokes
    return stokes.StokesContext(2, n, h, dt, (0.0, 0.0))


def _close(got, want, what):
    got = got.cpu().numpy().reshape(want.shape)
    scale = max(1.0, float(np.abs(want).max()))
    err = float(np.abs(got - want).max())
    same = float(np.mean(got == want))
    print(f"{what}: max |diff| {err:.3e} (scale {scale:.3g}), bit-identical {same:.4f}")
    assert err <= 1e-12 * scale, (what, err)


def _random_case(n, seed, amp):
    rng = np.random.default_rng(seed)
    nx, ny = n
    u = rng.normal(size=(ny, nx + 1)) * amp
    v = rng.normal(size=(ny + 1, nx)) * amp
    vu = rng.random(u.shape) < 0.4
    vv = rng.random(v.shape) < 0.4
    phi = rng.normal(size=(2 * ny + 3, 2 * nx + 3))
    src = rng.normal(size=phi.shape) + 1.0
    return u, v, vu, vv, phi, src


@pytest.mark.parametrize("n,passes,amp", [((37, 29), 3, 2.0), ((70, 45), 0, 0.5), ((2, 2), 2, 40.0),
                                          ((64, 33), 6, 25.0)])
def test_advect_matches_oracle_explicit_mask(n, passes, amp):
    """Random velocity and level set, random valid mask; several tiles of
    faces, ragged sizes, a 2 x 2 grid, and departure points far outside the
    grid (clamped)."""
    require_gpu()
    h, dt = 0.05, 0.04
    u, v, vu, vv, phi, src = _random_case(n, 11 + passes, amp)
    ctx = _ctx(n, h, dt)
    valid = to_gpu(np.concatenate([vu.ravel(), vv.ravel()]).astype(np.uint8))
    uo = [torch.empty(u.size, dtype=torch.float64, device="cuda"), torch.empty(v.size, dtype=torch.float64, device="cuda")]
    po = torch.empty(phi.size, dtype=torch.float64, device="cuda")
    ctx.advect([to_gpu(u.ravel()), to_gpu(v.ravel())], uo, G, passes, phi_in=to_gpu(phi.ravel()), phi_out=po,
               valid=valid, phi_union=to_gpu(src.ravel()))
    us, vs = Ad.advect_velocity(u, v, h, dt, G, vu, vv, passes)
    ph = np.minimum(Ad.advect_levelset(phi, u, v, h, dt, vu, vv, passes), src)
    _close(uo[0], us, "u*")
    _close(uo[1], vs, "v*")
    _close(po, ph, "phi")
    ctx.close()


@pytest.mark.parametrize("n,stub,passes", [(40, 6, 5), (150, 40, 8)])
def test_advect_validity_from_weights_jet(n, stub, passes):
    """valid = NULL takes the faces that are not fluid-without-liquid in the
    context's weights; the oracle takes the same set from its own system
    (~bad).  Jet geometry with a liquid column of ``stub`` cells below the
    opening and a seeded smooth perturbation of the velocity, at 40^2 and at
    the paper's 150^2 (every face and lattice point), with the inflow union;
    at 40^2 also u_out aliasing u_in, and no level set, no extension and no
    gravity."""
    require_gpu()
    from paper_1010_2832_gb300 import stokes, workloads as W
    wl = W.jet_2d(n, dt=0.002 if n == 150 else 0.01, stub_cells=stub)
    S = oracle_system(wl)
    rng = np.random.default_rng(n)
    k = rng.uniform(1, 4, size=4)
    def pert(x, y, c):
        return 0.3 * np.sin(2 * np.pi * (k[0 + c] * x + 0.5 * y)) * np.cos(2 * np.pi * k[2 + c] * y)
    xu, yu = Ad.face_points("u", wl.n)
    xv, yv = Ad.face_points("v", wl.n)
    u = wl.u_star[0] + pert(xu * wl.h, yu * wl.h, 0)
    v = wl.u_star[1] + pert(xv * wl.h, yv * wl.h, 1)
    ok_u, ok_v = Sy.split_faces(S, ~S.bad)
    src = W.jet_2d_source(n)
    ctx, dev = stokes.context_for(wl)
    ug = [to_gpu(u.ravel()), to_gpu(v.ravel())]
    uo = [torch.empty_like(t) for t in ug]
    po = torch.empty(wl.phi_liquid.size, dtype=torch.float64, device="cuda")
    ctx.advect(ug, uo, G, passes, phi_in=dev["phi_liquid"], phi_out=po, phi_union=to_gpu(src.ravel()))
    us, vs = Ad.advect_velocity(u, v, wl.h, wl.dt, G, ok_u, ok_v, passes)
    ph = np.minimum(Ad.advect_levelset(wl.phi_liquid, u, v, wl.h, wl.dt, ok_u, ok_v, passes), src)
    _close(uo[0], us, f"u* {n}^2")
    _close(uo[1], vs, f"v* {n}^2")
    _close(po, ph, f"phi {n}^2")
    if n == 40:
        ctx.advect(ug, ug, G, passes)                       # aliased, no level set
        _close(ug[0], us, "u* (aliased)")
        _close(ug[1], vs, "v* (aliased)")
        ug = [to_gpu(u.ravel()), to_gpu(v.ravel())]
        ctx.advect(ug, uo, (0.0, 0.0), 0)
        us, vs = Ad.advect_velocity(u, v, wl.h, wl.dt, (0.0, 0.0))
        _close(uo[0], us, "u* (no extension, no gravity)")
        _close(uo[1], vs, "v* (no extension, no gravity)")
    ctx.close()


def test_advect_argument_errors():
    require_gpu()
    from paper_1010_2832_gb300 import stokes
    ctx = _ctx((8, 8), 0.1, 0.01)
    u = [torch.zeros(8 * 9, dtype=torch.float64, device="cuda") for _ in range(2)]
    phi = torch.zeros(19 * 19, dtype=torch.float64, device="cuda")
    with pytest.raises(stokes.StokesError):          # no weights and no mask
        ctx.advect(u, u, G, 1)
    with pytest.raises(stokes.StokesError):          # phi_out aliasing phi_in
        ctx.advect(u, u, G, 0, phi_in=phi, phi_out=phi, valid=torch.ones(144, dtype=torch.uint8, device="cuda"))
    with pytest.raises(stokes.StokesError):          # negative pass count
        ctx.advect(u, u, G, -1, valid=torch.ones(144, dtype=torch.uint8, device="cuda"))
    ctx.close()
    c3 = stokes.StokesContext(3, (4, 4, 4), 0.1, 0.01)
    with pytest.raises(stokes.StokesError):          # 2D only
        c3.advect(u, u, G, 0, valid=torch.ones(144, dtype=torch.uint8, device="cuda"))
    c3.close()
