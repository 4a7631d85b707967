"""Pins of the fractional-step reference (oracle.advect): no motion is the
identity, a uniform velocity transports a linear field exactly (bilinear
interpolation reproduces it), a shift by whole cells moves samples onto
their neighbours, gravity adds dt g, shear flows are steady (each velocity
component is advected by the full velocity), departures beyond the samples
clamp onto the boundary, and the extension fills invalid samples with the
mean of their valid 4-neighbours, one ring per sweep."""
import numpy as np

from oracle import advect as Ad

H = 0.1
ORIGIN = (0.0, 0.0)
N = (12, 9)


def _faces(fu, fv):
    xu, yu = Ad.face_points("u", N)
    xv, yv = Ad.face_points("v", N)
    return fu(ORIGIN[0] + H * xu, ORIGIN[1] + H * yu), fv(ORIGIN[0] + H * xv, ORIGIN[1] + H * yv)


def _lattice(f):
    X, Y = Ad.lattice_points((2 * N[1] + 3, 2 * N[0] + 3))
    return f(ORIGIN[0] + H * X, ORIGIN[1] + H * Y)


def test_no_motion_is_the_identity():
    rng = np.random.default_rng(1)
    u = rng.normal(size=(N[1], N[0] + 1))
    v = rng.normal(size=(N[1] + 1, N[0]))
    phi = rng.normal(size=(2 * N[1] + 3, 2 * N[0] + 3))
    us, vs = Ad.advect_velocity(u, v, H, 0.0, (0.0, 0.0))
    assert np.array_equal(us, u) and np.array_equal(vs, v)
    assert np.array_equal(Ad.advect_levelset(phi, u, v, H, 0.0), phi)


def test_uniform_velocity_transports_a_linear_level_set_exactly():
    U, V, dt = 0.7, -0.4, 0.05
    u, v = _faces(lambda x, y: U + 0 * x, lambda x, y: V + 0 * x)
    phi = _lattice(lambda x, y: 0.3 + 2.0 * x - 1.5 * y)
    new = Ad.advect_levelset(phi, u, v, H, dt)
    want = _lattice(lambda x, y: 0.3 + 2.0 * (x - U * dt) - 1.5 * (y - V * dt))
    inner = (slice(2, -2), slice(2, -2))      # departure points inside the lattice
    assert np.abs(new[inner] - want[inner]).max() <= 1e-12
    # and a uniform velocity stays uniform
    us, vs = Ad.advect_velocity(u, v, H, dt, (0.0, 0.0))
    assert np.abs(us - U).max() <= 1e-15 and np.abs(vs - V).max() <= 1e-15


def test_whole_cell_shift_moves_samples_to_neighbours():
    rng = np.random.default_rng(2)
    u0 = rng.normal(size=(N[1], N[0] + 1))
    dt = 0.05
    u = np.full_like(u0, H / dt)                 # every departure point one cell to the left
    v = np.zeros((N[1] + 1, N[0]))
    phi = rng.normal(size=(2 * N[1] + 3, 2 * N[0] + 3))
    new = Ad.advect_levelset(phi, u, v, H, dt)
    assert np.abs(new[:, 2:] - phi[:, :-2]).max() <= 1e-13     # one cell = two lattice steps


def test_gravity_adds_dt_g():
    rng = np.random.default_rng(3)
    u = rng.normal(size=(N[1], N[0] + 1))
    v = rng.normal(size=(N[1] + 1, N[0]))
    a = Ad.advect_velocity(u, v, H, 0.02, (0.0, 0.0))
    b = Ad.advect_velocity(u, v, H, 0.02, (0.5, -9.81))
    assert np.allclose(b[0] - a[0], 0.02 * 0.5, atol=1e-15, rtol=0)
    assert np.allclose(b[1] - a[1], 0.02 * -9.81, atol=1e-15, rtol=0)


def test_extension_spreads_a_constant_and_keeps_valid_values():
    f = np.full((8, 9), np.nan)
    valid = np.zeros(f.shape, dtype=bool)
    valid[3:5, 4:6] = True
    f[valid] = 2.5
    g = Ad.extend(f, valid, 3)
    filled = ~np.isnan(g)
    assert np.all(g[filled] == 2.5)
    assert filled.sum() > valid.sum()
    assert np.array_equal(g[valid], f[valid])


def test_extension_rule_on_hand_worked_cases():
    """One sweep fills exactly the invalid samples with a valid 4-neighbour
    (not diagonal ones) with the mean of those neighbours; a second sweep
    continues from the first one's values."""
    row = np.array([[1.0, np.nan, np.nan, np.nan, 5.0]])
    ok = np.array([[True, False, False, False, True]])
    one = Ad.extend(row, ok, 1)
    assert one[0, 1] == 1.0 and one[0, 3] == 5.0 and np.isnan(one[0, 2])
    two = Ad.extend(row, ok, 2)
    assert two[0, 2] == 3.0                                   # mean of 1 and 5
    sq = np.full((3, 3), np.nan)
    sq[0, 0] = 2.0
    okq = np.zeros((3, 3), bool)
    okq[0, 0] = True
    g = Ad.extend(sq, okq, 1)
    assert g[0, 1] == 2.0 and g[1, 0] == 2.0 and np.isnan(g[1, 1])   # no diagonal neighbours
    g2 = Ad.extend(sq, okq, 2)
    assert g2[1, 1] == 2.0 and g2[0, 2] == 2.0 and np.isnan(g2[2, 2])


def test_shear_flows_are_steady_and_far_departures_clamp():
    """u = y (v = 0) and v = x (u = 0) are steady under pure advection: each
    component is constant along its own streamlines, so both must come back
    unchanged (a swapped component would move them); a level set that
    depends only on the coordinate the flow does not change is unchanged.
    A departure point far outside the lattice takes the boundary sample."""
    dt = 0.07
    u, v = _faces(lambda x, y: y, lambda x, y: 0.0 * x)
    us, vs = Ad.advect_velocity(u, v, H, dt, (0.0, 0.0))
    assert np.abs(us - u).max() <= 1e-14 and np.abs(vs).max() == 0.0
    phi = _lattice(lambda x, y: 0.2 + y)
    assert np.abs(Ad.advect_levelset(phi, u, v, H, dt) - phi).max() <= 1e-14
    u2, v2 = _faces(lambda x, y: 0.0 * x, lambda x, y: x)
    us2, vs2 = Ad.advect_velocity(u2, v2, H, dt, (0.0, 0.0))
    assert np.abs(vs2 - v2).max() <= 1e-14 and np.abs(us2).max() == 0.0
    # far departures: every lattice point's departure lies left of the lattice
    big = 1e3
    ub, vb = _faces(lambda x, y: big + 0 * x, lambda x, y: 0.0 * x)
    rng = np.random.default_rng(5)
    phi = rng.normal(size=(2 * N[1] + 3, 2 * N[0] + 3))
    new = Ad.advect_levelset(phi, ub, vb, H, 1.0)
    assert np.array_equal(new, np.repeat(phi[:, :1], phi.shape[1], axis=1))
