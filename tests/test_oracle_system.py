"""Pins of the assembled SPD system (oracle.system) that do not come from it:
operator identities on polynomial and rigid fields, the textbook interior
stencils, symmetry, positive definiteness, equivalence with the indefinite
KKT system, and the exactness cases of Section 9 (hydrostatic, rigid
translation and rotation), and the Schwarz preconditioner forms against
their textbook definitions."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import operators as O
from oracle import solve as So
from oracle import system as S_
from paper_1010_2832_gb300 import workloads as W


def _system(wl, **kw):
    return S_.build_system(S_.StokesInput(**wl.as_oracle_kwargs()), **kw)


def _face_field(n, h, origin, fn):
    dim = len(n)
    parts = []
    for d, f in enumerate(W.FACES[dim]):
        P = W.sample_points(f, n, h, origin)
        parts.append(np.broadcast_to(fn(d, P), P[0].shape).ravel())
    return np.concatenate(parts)


def test_divergence_of_linear_field_exact():
    n, h, o = (6, 5), 0.2, (0.0, 0.0)
    u = _face_field(n, h, o, lambda d, P: (1.5 * P[0] - 0.7 * P[1] + 0.2) if d == 0 else (0.3 * P[0] + 2.5 * P[1]))
    div = -(O.gradient_transpose(n, h) @ u)
    assert np.allclose(div, 1.5 + 2.5, atol=1e-12)


def test_deformation_rows_on_linear_field_2d():
    n, h, o = (6, 5), 0.2, (0.0, 0.0)
    # u = a x + b y, v = c x + d y:  tau_xx row -> a - d, tau_xy row -> b + c
    a, b, c, d = 1.3, -0.4, 0.9, 0.25
    u = _face_field(n, h, o, lambda k, P: (a * P[0] + b * P[1]) if k == 0 else (c * P[0] + d * P[1]))
    D = O.deformation(n, h)
    r = D @ u
    ncell = n[0] * n[1]
    assert np.allclose(r[:ncell], a - d, atol=1e-12)
    # interior nodes only (boundary node rows drop ghost faces)
    nodes = r[ncell:].reshape(n[1] + 1, n[0] + 1)
    assert np.allclose(nodes[1:-1, 1:-1], b + c, atol=1e-12)


def test_deformation_rows_on_linear_field_3d():
    n, h, o = (4, 5, 3), 0.25, (0.0, 0.0, 0.0)
    J = np.array([[0.7, -0.2, 0.4], [0.5, 1.1, -0.3], [0.2, 0.6, -0.9]])  # du_i/dx_j
    u = _face_field(n, h, o, lambda k, P: J[k, 0] * P[0] + J[k, 1] * P[1] + J[k, 2] * P[2])
    r = O.deformation(n, h) @ u
    nx, ny, nz = n
    nc = nx * ny * nz
    assert np.allclose(r[:nc], J[0, 0] - J[2, 2], atol=1e-12)
    assert np.allclose(r[nc:2 * nc], J[1, 1] - J[2, 2], atol=1e-12)
    o2 = 2 * nc
    exy = r[o2:o2 + nz * (ny + 1) * (nx + 1)].reshape(nz, ny + 1, nx + 1)
    assert np.allclose(exy[:, 1:-1, 1:-1], J[0, 1] + J[1, 0], atol=1e-12)
    o3 = o2 + exy.size
    exz = r[o3:o3 + (nz + 1) * ny * (nx + 1)].reshape(nz + 1, ny, nx + 1)
    assert np.allclose(exz[1:-1, :, 1:-1], J[0, 2] + J[2, 0], atol=1e-12)
    eyz = r[o3 + exz.size:].reshape(nz + 1, ny + 1, nx)
    assert np.allclose(eyz[1:-1, 1:-1, :], J[1, 2] + J[2, 1], atol=1e-12)


def test_rigid_rotation_has_zero_divergence_and_strain():
    n, h, o = (7, 6), 0.15, (-0.5, -0.4)
    u = _face_field(n, h, o, lambda d, P: -0.8 * P[1] if d == 0 else 0.8 * P[0])
    assert np.abs(O.gradient_transpose(n, h) @ u).max() < 1e-13
    r = O.deformation(n, h) @ u
    ncell = n[0] * n[1]
    assert np.abs(r[:ncell]).max() < 1e-13
    # boundary nodes see ghost faces (dropped), so only interior nodes vanish
    nodes = r[ncell:].reshape(n[1] + 1, n[0] + 1)
    assert np.abs(nodes[1:-1, 1:-1]).max() < 1e-13


def test_interior_stencil_is_textbook():
    """All-liquid box, no interior solid: interior rows of A are
    A22 = (dt/rho)(-Lap_h), A11[txx] = 1/mu + (dt/rho)(-Lap_h) and
    A12 = (dt/rho)(d_xx - d_yy), with the 5-point stencils on h."""
    n = 8
    rho, mu, dt = 2.0, 0.5, 0.1
    wl = W.full_box(n, 2)
    wl.rho = [np.full_like(r, rho) for r in wl.rho]
    wl.mu = [np.full_like(m, mu) for m in wl.mu]
    wl.dt = dt
    S = _system(wl)
    A = S.A.tocsr()
    h = wl.h
    nc, nn = n * n, (n + 1) ** 2
    k = dt / (rho * h * h)
    i, j = 4, 3
    c = j * n + i
    txx, p = c, nc + nn + c
    assert A[p, p] == pytest.approx(4 * k)
    assert A[p, p + 1] == pytest.approx(-k)
    assert A[p, p + n] == pytest.approx(-k)
    assert A[txx, txx] == pytest.approx(1 / mu + 4 * k)
    assert A[txx, txx + 1] == pytest.approx(-k)
    assert A[txx, txx + n] == pytest.approx(-k)
    # A12 = (dt/rho) (delta_xx - delta_yy) p
    assert A[txx, p] == pytest.approx(0.0, abs=1e-9)
    assert A[txx, p + 1] == pytest.approx(k)
    assert A[txx, p - 1] == pytest.approx(k)
    assert A[txx, p + n] == pytest.approx(-k)
    # tau_xy node (i, j): (1/mu) + (dt/rho)(-Lap_h) on nodes
    t = nc + j * (n + 1) + i
    assert A[t, t] == pytest.approx(1 / mu + 4 * k)
    assert A[t, t + 1] == pytest.approx(-k)


CASES = [(2, (8, 7)), (2, (12, 12)), (2, (10, 6)), (3, (5, 4, 6)), (3, (6, 6, 5))]


@pytest.mark.parametrize("dim,n", CASES)
@pytest.mark.parametrize("seed", range(4))
def test_symmetric_positive_definite_and_kkt_equivalent(dim, n, seed):
    S = _system(W.random_small(n, seed=seed, dim=dim))
    A = S.A
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
    nulls = S_.pressure_null_vectors(S)
    if not nulls:
        assert So.cholesky_ok(A)
    x = So.solve_direct(A, S.b, nulls)
    Kmat, r, lv, ac = S_.kkt_system(S)
    z = spla.spsolve(Kmat.tocsc(), r)
    u = S_.recover_velocity(S, x)
    scale_u = max(np.abs(z[:lv.size]).max(), 1e-30)
    assert np.abs(u[lv] - z[:lv.size]).max() <= 1e-7 * scale_u
    if not nulls:
        scale_x = max(np.abs(z[lv.size:]).max(), 1e-30)
        assert np.abs(x[ac] - z[lv.size:]).max() <= 1e-6 * scale_x


def test_solid_side_rule_removes_a_null_space():
    """Without the solid-side invalidation (a face next to a zero-fluid-weight
    multiplier) the pressure and stress of a fully solid cell that touches one
    live face form a null vector; with it the matrix is definite."""
    wl = W.bumps_2d(24, seed=7, rho_split=False)
    S1 = _system(wl, solid_side_rule=False)
    S2 = _system(wl)
    assert not So.cholesky_ok(S1.A)
    assert So.cholesky_ok(S2.A)


def _exactness_system(wl):
    S = _system(wl)
    x = So.solve_direct(S.A, S.b, S_.pressure_null_vectors(S))
    return S, x, S_.recover_velocity(S, x)


def test_rigid_translation_free_blob_is_exact():
    U = (0.37, -0.81)
    wl = W.from_functions("blob", 2, (20, 20), 1 / 20, 0.05, (0, 0),
                          lambda X: np.hypot(X[0] - .48, X[1] - .53) - 0.27 * (1 + 0.2 * np.sin(5 * X[0])),
                          lambda X: W.box_phi(X, (0, 0), (1, 1)),
                          lambda P: 1.0 + P[0], lambda P: 0.2 + P[1], lambda d, P: 0.0, lambda d, P: U[d])
    S, x, u = _exactness_system(wl)
    assert np.abs(x).max() < 1e-10
    assert np.abs(u[S.live] - S.u_star[S.live]).max() < 1e-12


def test_rigid_rotation_free_blob_is_exact():
    w = 1.7
    rot = lambda d, P: -w * (P[1] - 0.5) if d == 0 else w * (P[0] - 0.5)
    wl = W.from_functions("blob", 2, (22, 22), 1 / 22, 0.1, (0, 0),
                          lambda X: np.hypot(X[0] - .5, X[1] - .5) - 0.3 - 0.04 * np.cos(3 * np.arctan2(X[1] - .5, X[0] - .5)),
                          lambda X: W.box_phi(X, (0, 0), (1, 1)),
                          lambda P: 1.0, lambda P: 0.3 + P[0] * P[1], lambda d, P: 0.0, rot)
    S, x, u = _exactness_system(wl)
    assert np.abs(x).max() < 1e-9
    assert np.abs(u[S.live] - S.u_star[S.live]).max() < 1e-11


def test_rigid_rotation_3d_is_exact():
    w = np.array([0.3, -0.5, 0.8])
    c = np.array([0.5, 0.5, 0.5])
    def rot(d, P):
        r = [P[k] - c[k] for k in range(3)]
        cross = [w[1] * r[2] - w[2] * r[1], w[2] * r[0] - w[0] * r[2], w[0] * r[1] - w[1] * r[0]]
        return cross[d]
    wl = W.from_functions("ball", 3, (9, 9, 9), 1 / 9, 0.1, (0, 0, 0),
                          lambda X: np.sqrt((X[0] - .5) ** 2 + (X[1] - .5) ** 2 + (X[2] - .5) ** 2) - 0.33,
                          lambda X: W.box_phi(X, (0,) * 3, (1,) * 3),
                          lambda P: 1.0, lambda P: 0.5, lambda d, P: 0.0, rot)
    S, x, u = _exactness_system(wl)
    assert np.abs(x).max() < 1e-9
    assert np.abs(u[S.live] - S.u_star[S.live]).max() < 1e-11


@pytest.mark.parametrize("solid", [False, True])
def test_hydrostatic_is_exact(solid):
    """Liquid at rest under gravity in a box (optionally around a solid disk)
    with a flat free surface: u* = (0, -g dt) gives u = 0."""
    g, dt = 9.81, 0.02
    surf = 0.613
    phiS = (lambda X: np.minimum(W.box_phi(X, (0, 0), (1, 1)), np.hypot(X[0] - .4, X[1] - .25) - .12)) if solid \
        else (lambda X: W.box_phi(X, (0, 0), (1, 1)))
    wl = W.from_functions("hydro", 2, (24, 24), 1 / 24, dt, (0, 0),
                          lambda X: X[1] - surf, phiS, lambda P: 1.3, lambda P: 0.7,
                          lambda d, P: 0.0, lambda d, P: 0.0 if d == 0 else -g * dt)
    S, x, u = _exactness_system(wl)
    assert np.abs(u[S.live]).max() < 1e-10
    nc = S.sizes["cell"]
    assert np.abs(x[:-nc]).max() < 1e-9          # all stresses vanish


def test_moving_solid_translation_is_exact():
    U = (0.5, -0.2)
    disk = lambda X: np.hypot(X[0] - .5, X[1] - .45) - .15
    wl = W.from_functions("trans", 2, (24, 24), 1 / 24, 0.05, (0, 0),
                          lambda X: np.hypot(X[0] - .5, X[1] - .5) - 0.4,
                          lambda X: np.minimum(W.box_phi(X, (0, 0), (1, 1)), disk(X)),
                          lambda P: 1.0, lambda P: 0.4, lambda d, P: U[d], lambda d, P: U[d])
    S, x, u = _exactness_system(wl)
    assert np.abs(x).max() < 1e-9
    assert np.abs(u[S.live] - U[0] * 0 - S.u_star[S.live]).max() < 1e-11


def test_pcg_matches_direct():
    S = _system(W.disk_in_box(16))
    xd = So.solve_direct(S.A, S.b)
    x, it, rr = So.pcg(S.A, S.b, tol=1e-13)
    assert rr <= 1e-13
    assert np.abs(x - xd).max() <= 1e-9 * np.abs(xd).max()


def test_additive_schwarz_single_patch_is_exact_inverse():
    """A grid small enough for one patch to hold every unknown: the Schwarz
    operator is A^-1 on the active unknowns."""
    wl = W.random_small((3, 3), seed=2)
    S = _system(wl)
    r = np.random.default_rng(0).normal(size=S.A.shape[0]) * S.active
    z = So.additive_schwarz(S, r)
    x = spla.spsolve(S.A.tocsc(), r)
    assert np.allclose(z, x, rtol=1e-10, atol=1e-12 * np.abs(x).max())


def test_additive_schwarz_is_symmetric_positive():
    S = _system(W.bumps_2d(20, seed=3))
    rng = np.random.default_rng(1)
    a = rng.normal(size=S.A.shape[0]) * S.active
    b = rng.normal(size=S.A.shape[0]) * S.active
    Ma, Mb = So.additive_schwarz(S, a), So.additive_schwarz(S, b)
    assert abs(Ma @ b - a @ Mb) <= 1e-10 * np.linalg.norm(Ma) * np.linalg.norm(b)
    assert a @ Ma > 0


def test_multiplicative_schwarz_single_patch_is_exact_inverse():
    """One patch holding every unknown: one local solve is the exact inverse,
    and every later colour sweep finds a zero residual."""
    S = _system(W.random_small((3, 3), seed=2))
    r = np.random.default_rng(0).normal(size=S.A.shape[0]) * S.active
    z = So.multiplicative_schwarz(S, r)
    x = spla.spsolve(S.A.tocsc(), r)
    assert np.allclose(z, x, rtol=1e-10, atol=1e-12 * np.abs(x).max())


def test_schwarz_colours_are_disjoint_and_cover_the_patches():
    """The widened patches of one colour share no unknown (so their solves
    are independent), and the coloured patches are those of the additive
    form: the additive operator rebuilt from them matches it."""
    S = _system(W.bumps_2d(24, seed=3))
    patches = So.schwarz_colour_patches(S)
    assert {c for c, _ in patches} == {0, 1, 2, 3}
    for c in range(4):
        idx = np.concatenate([i for cc, i in patches if cc == c])
        assert idx.size == np.unique(idx).size
    A = S.A.tocsr()
    r = np.random.default_rng(2).normal(size=S.A.shape[0]) * S.active
    z = np.zeros(r.size)
    for _, idx in patches:
        z[idx] += np.linalg.solve(A[idx][:, idx].toarray(), r[idx])
    assert np.allclose(z, So.additive_schwarz(S, r), rtol=1e-12, atol=1e-12 * np.abs(z).max())


def test_multiplicative_schwarz_error_propagator_is_the_product_of_colour_projections():
    """Textbook form of multiplicative Schwarz (Smith, Bjorstad and Gropp,
    Domain Decomposition, ch. 1): I - M A = prod_k (I - B_{c_k} A) over the
    sweep order, B_c = sum_{p in c} R_p^T A_p^-1 R_p.  M A is taken column by
    column through the sweeps; the product is formed from explicit dense
    matrices.  A sweep that skipped its residual update, updated it with the
    wrong sign or solved on r instead of the current residual fails here."""
    S = _system(W.bumps_2d(14, seed=4))
    act = np.flatnonzero(S.active)
    A = S.A.tocsr()
    Ad = A[act][:, act].toarray()
    n = act.size
    pos = -np.ones(S.A.shape[0], dtype=int)
    pos[act] = np.arange(n)
    patches = So.schwarz_colour_patches(S)
    B = {c: np.zeros((n, n)) for c in range(4)}
    for c, idx in patches:
        k = pos[idx]
        B[c][np.ix_(k, k)] += np.linalg.inv(Ad[np.ix_(k, k)])
    order = (0, 1, 2, 3, 2, 1, 0)
    E = np.eye(n)
    for c in order:                       # the first colour acts first: rightmost factor
        E = (np.eye(n) - B[c] @ Ad) @ E
    MA = np.zeros((n, n))
    for j in range(n):
        col = np.zeros(S.A.shape[0])
        col[act] = Ad[:, j]
        MA[:, j] = So.multiplicative_schwarz(S, col, order=order)[act]
    assert np.allclose(np.eye(n) - MA, E, atol=1e-9)


def test_multiplicative_schwarz_is_symmetric_positive_and_beats_additive():
    """Palindromic sweeps give a symmetric positive-definite operator; as a
    CG preconditioner it takes fewer iterations than the additive form."""
    S = _system(W.bumps_2d(24, seed=3))
    rng = np.random.default_rng(1)
    a = rng.normal(size=S.A.shape[0]) * S.active
    b = rng.normal(size=S.A.shape[0]) * S.active
    Ma, Mb = So.multiplicative_schwarz(S, a), So.multiplicative_schwarz(S, b)
    assert abs(Ma @ b - a @ Mb) <= 1e-10 * np.linalg.norm(Ma) * np.linalg.norm(b)
    assert a @ Ma > 0
    # inactive unknowns (identity rows) pass through: z = r there
    full = rng.normal(size=S.A.shape[0])
    zf = So.multiplicative_schwarz(S, full)
    assert (~S.active).any() and np.array_equal(zf[~S.active], full[~S.active])

    def cg_iterations(M):
        A = S.A.tocsr()
        x = np.zeros(S.b.size); r = S.b.copy(); z = M(r); p = z.copy(); rz = r @ z
        for it in range(1, 2000):
            q = A @ p; al = rz / (p @ q); x += al * p; r -= al * q
            if np.linalg.norm(r) <= 1e-8 * np.linalg.norm(S.b):
                return it
            z = M(r); rzn = r @ z; p = z + (rzn / rz) * p; rz = rzn
        return 2000

    it_m = cg_iterations(lambda r: So.multiplicative_schwarz(S, r))
    it_a = cg_iterations(lambda r: So.additive_schwarz(S, r))
    assert it_m < it_a


def _x_bc(S, tau=None, p=None):
    """(tau_BC, p_BC) in unknown order from per-sample callables or zeros."""
    parts = []
    nx, ny, nz = S_._nx_ny_nz(S.inp.n)
    names = S_.unknown_names(S.inp.dim)
    kinds = S_.unknown_kinds(S.inp.dim)
    for name, kind in zip(names, kinds):
        size = S.sizes[kind]
        fn = p if name == "p" else (tau or {}).get(name)
        if fn is None:
            parts.append(np.zeros(size))
        else:
            P = W.sample_points(kind, S.inp.n, S.inp.h, S.inp.origin)
            parts.append(np.ravel(fn(P) * np.ones(P[0].shape)))
    return np.concatenate(parts)


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_surface_pressure_is_hydrostatic(dim):
    """A uniform prescribed pressure P0 on a free surface, liquid at rest and no
    body force: the liquid pressure is P0, the stresses and velocities zero
    (Section 6.1's traction terms, with the sign that makes this hold)."""
    if dim == 2:
        wl = W.disk_in_box(24, radius=0.3)
    else:
        lo, hi = (0.0,) * 3, (1.0,) * 3
        wl = W.from_functions("ball", 3, (10, 10, 10), 0.1, 0.01, lo,
                              lambda X: np.sqrt(sum((x - 0.5) ** 2 for x in X)) - 0.3, lambda X: W.box_phi(X, lo, hi),
                              lambda P: 1.0, lambda P: 1.0, lambda d, P: 0.0, lambda d, P: 0.0)
    S = _system(wl)
    P0 = 2.5
    xbc = _x_bc(S, p=lambda P: P0)
    zero = np.zeros_like(S.u_star)
    ue = S_.traction_u_star(S, xbc, u_star=zero)
    b = S_.rhs(S, ue) if np.all(S.u_bc == 0) else None
    if b is None:
        pytest.skip("moving boundary in this geometry")
    x = So.solve_direct(S.A, b, S_.pressure_null_vectors(S))
    parts = S_.split_unknowns(S, x)
    act = S_.split_unknowns(S, S.active.astype(float))
    pa = parts["p"][act["p"] > 0]
    assert pa.size > 0
    assert np.abs(pa - P0).max() <= 1e-9 * P0
    for name in parts:
        if name != "p":
            assert np.abs(parts[name]).max() <= 1e-9 * P0
    u = S_.recover_velocity(S, x, u_star=ue)
    assert np.abs(u[S.live]).max() <= 1e-9 * P0 * S.inp.dt / S.inp.h


def test_traction_terms_match_the_kkt_system():
    """The SPD route with u* + dt f/(rho W_L) equals the KKT solve with the
    force added to the first block row (weighted like the mass term), and
    the force is linear in (tau_BC, p_BC)."""
    wl = W.bumps_2d(20, seed=9, rho_split=False)
    S = _system(wl)
    rng = np.random.default_rng(3)
    xbc = rng.normal(size=S.A.shape[0])
    f = S_.traction_force(S, xbc)
    ue = S_.traction_u_star(S, xbc)
    x = So.solve_direct(S.A, S_.rhs(S, ue), S_.pressure_null_vectors(S))
    u = S_.recover_velocity(S, x, u_star=ue)
    Kmat, r, lv, ac = S_.kkt_system(S, face_force=f)
    z = spla.spsolve(Kmat.tocsc(), r)
    scale = max(np.abs(z[:lv.size]).max(), 1e-30)
    assert np.abs(u[lv] - z[:lv.size]).max() <= 1e-7 * scale
    x2 = rng.normal(size=xbc.size)
    f2 = S_.traction_force(S, x2)
    assert np.allclose(S_.traction_force(S, 2 * xbc - 3 * x2), 2 * f - 3 * f2, atol=1e-12 * np.abs(f).max())
    # no force far from the air: on a live face whose neighbouring unknowns
    # are all active with W_L = 1 (and W_L^u = 1) both terms cancel
    far = (S.WLu == 1.0) & S.live
    nb_full = np.abs(S.M.T) @ ((S.WLx * S.active) < 1.0).astype(float) == 0
    sel = far & nb_full
    assert sel.any()
    assert np.abs(f[sel]).max() <= 1e-12 * np.abs(f).max()


def test_min_face_liquid_floor():
    """Floor of the face mass fraction (min_face_liquid): a floor at or below
    the smallest live W_L^u leaves A and b unchanged; on the jet geometry,
    whose opening edges put level-set zeros on lattice points (faces with a
    rounding-level liquid fraction), the floored system has K <= dt W_F /
    (rho eps), its SPD solve plus velocity recovery equals the KKT solve with
    the same floored mass, and its condition number drops from > 1e12 to
    < 1e6."""
    wl = W.bumps_2d(24, seed=4, rho_split=False)
    S0 = _system(wl)
    eps = 0.5 * S0.WLu[S0.live].min()
    S1 = _system(wl, min_face_liquid=eps)
    assert (S0.A != S1.A).nnz == 0 and np.array_equal(S0.b, S1.b)

    wl = W.jet_2d(150)
    S0 = _system(wl)
    eps = 0.01
    S = _system(wl, min_face_liquid=eps)
    lv = S.live
    assert S0.WLu[lv].min() < 1e-12                      # the slivers are there
    assert np.all(S.K[lv] <= S.inp.dt * S.effWF[lv] / (S.rho[lv] * eps) * (1 + 1e-15))
    assert np.array_equal(S.K[lv & (S.WLu >= eps)], S0.K[lv & (S.WLu >= eps)])
    nulls = S_.pressure_null_vectors(S)
    x = So.solve_direct(S.A, S.b, nulls)
    u = S_.recover_velocity(S, x)
    Kmat, r, lvi, ac = S_.kkt_system(S)
    z = spla.spsolve(Kmat.tocsc(), r)
    scale = max(np.abs(z[:lvi.size]).max(), 1e-30)
    assert np.abs(u[lvi] - z[:lvi.size]).max() <= 1e-7 * scale
    act = np.flatnonzero(S.active)
    def cond(T):
        w = np.linalg.eigvalsh(T.A[act][:, act].toarray())
        return w.max() / w.min()
    assert cond(S0) > 1e12 and cond(S) < 1e6
