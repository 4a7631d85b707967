"""The pressure-stress SPD system of one backward-Euler Stokes step.

Implements, in FP64 and with explicitly assembled scipy matrices:

* weights W_L, W_F per sample type (Section 5; estimator in ``fractions``);
* null-space elimination (Section 8) in our reading, stated in full below;
* the SPD matrix of eq. stokesmixedsystemspd,
      A = C + B K B^T,  B = [W_L^tau D ; W_L^p G^T],
      K = dt P^-1 (W_L^u)^-1 W_F^u  (diagonal on faces),
  where C is the stress block, i.e. the reduced-unknown form of the paper's
  (1/2) M^-1 W_L^tau W_F^tau: with the unknowns of ``operators`` the stress
  part of the variational form, -(dt/4 mu) |tau|_F^2, has Hessian
  (dt/mu) * [1] for tau_xx, tau_xy in 2D and (dt/mu) * [[1, 1/2], [1/2, 1]]
  for (tau_xx, tau_yy) plus (dt/mu) for each edge stress in 3D; dividing by
  dt as the paper does gives C.  (This reproduces the paper's
  "tau_xx + tau_yy / 2 = mu (u_x - w_z)" of Section 5.)
* the right-hand side with prescribed solid velocities (Section 6.2, applied
  to the combined system by weighting each row by its own W_L):
      b_s = W_L^s [ (R (W_F^u u* + W_S^u u_BC))_s - W_S^s (R u_BC)_s ]
  with R = D for stress rows and R = G^T for pressure rows;
* the indefinite KKT system (eq. stokesmixedsystem with the same reduced D
  and C and the same right-hand side) used to cross-check the Schur step;
* velocity recovery from the first block row of eq. stokesmixedsystem:
      u = u* - dt P^-1 (W_L^u)^-1 (D^T W_L^tau tau + G W_L^p p).

Null-space elimination (Section 8), as read here:

1. Faces on the grid boundary are static solid wall: effective W_F^u = 0.
2. Solid side: a face with W_F^u > 0 that is coupled (through D or G^T) to
   a stress or pressure sample whose own weights are W_L > 0 and W_F = 0 is
   invalid and takes its boundary value u_BC (effective W_F^u = 0).
3. A face is live if effective W_F^u > 0 and W_L^u > 0, and "bad" if
   effective W_F^u > 0 and W_L^u = 0.
4. Free-surface side: a stress or pressure unknown with W_L > 0 that is
   coupled to a bad face is invalid.  The unknowns at one cell (tau_xx,
   [tau_yy,] p) share one control volume and share validity; pressure is
   coupled to every face of the cell, so it decides for all of them.
5. An unknown is active if W_L > 0, it is not invalid, and its diagonal
   entry in A is positive (for a cell: the pressure's).
6. Inactive unknowns are fixed to their boundary value 0: identity rows and
   zero right-hand side.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import grid as G_
from . import fractions as F_
from . import operators as O_


@dataclass
class StokesInput:
    """Inputs of one step.  Field arrays use ``grid.field_shape`` layouts.

    rho:  list of face arrays [u, v(, w)]   density per velocity sample (P)
    mu:   2D [cell, node]; 3D [cell, exy, exz, eyz]  viscosity per stress sample (M)
    """
    dim: int
    n: tuple
    h: float
    dt: float
    origin: tuple
    phi_liquid: np.ndarray
    phi_solid: np.ndarray
    rho: list
    mu: list
    u_bc: list
    u_star: list


@dataclass
class StokesSystem:
    inp: StokesInput
    W_L: dict = field(default_factory=dict)
    W_F: dict = field(default_factory=dict)
    # face-ordered vectors
    WLu: np.ndarray = None
    WLm: np.ndarray = None
    WFu: np.ndarray = None
    effWF: np.ndarray = None
    invalid_face: np.ndarray = None
    live: np.ndarray = None
    bad: np.ndarray = None
    K: np.ndarray = None
    rho: np.ndarray = None
    u_bc: np.ndarray = None
    u_star: np.ndarray = None
    # unknown-ordered vectors
    WLx: np.ndarray = None
    WFx: np.ndarray = None
    mux: np.ndarray = None
    active: np.ndarray = None
    a: np.ndarray = None
    # operators
    M: sp.csr_matrix = None      # [D ; G^T]  (unknowns x faces), unweighted
    B: sp.csr_matrix = None      # diag(a) M
    C: sp.csr_matrix = None      # stress block on active unknowns
    A: sp.csr_matrix = None
    b: np.ndarray = None
    sizes: dict = field(default_factory=dict)


def _nx_ny_nz(n):
    return (n[0], n[1], None) if len(n) == 2 else tuple(n)


def sample_sizes(dim, n):
    nx, ny, nz = _nx_ny_nz(n)
    kinds = G_.KINDS_2D if dim == 2 else G_.KINDS_3D
    return {k: int(np.prod(G_.field_shape(k, nx, ny, nz))) for k in kinds}


def unknown_kinds(dim):
    """Kinds of the unknown blocks in x order: stresses then pressure."""
    return list(O_.stress_kinds(dim)) + ["cell"]


def unknown_names(dim):
    return list(O_.STRESS_NAMES_2D if dim == 2 else O_.STRESS_NAMES_3D) + ["p"]


def compute_fractions(inp):
    """W_L and W_F for every sample type (Section 5)."""
    nx, ny, nz = _nx_ny_nz(inp.n)
    kinds = G_.KINDS_2D if inp.dim == 2 else G_.KINDS_3D
    W_L, W_F = {}, {}
    for k in kinds:
        idx = G_.lattice_index(k, nx, ny, nz)
        W_L[k] = F_.cv_fraction(inp.phi_liquid, idx).ravel()
        W_F[k] = 1.0 - F_.cv_fraction(inp.phi_solid, idx).ravel()
    return W_L, W_F


def _stress_block_C(dim, n, WLx, WFx, mux, active, sizes):
    """C on the active unknowns (zero on pressure rows)."""
    d = np.where(active, WLx * WFx / np.where(mux > 0, mux, 1.0), 0.0)
    ntot = d.size
    nc = sizes["cell"]
    d = d.copy()
    d[ntot - nc:] = 0.0          # pressure rows carry no stress term
    if dim == 2:
        return sp.diags(d, format="csr")
    # 3D: (tau_xx, tau_yy) of one cell are coupled by d_cell / 2, where
    # d_cell = W_L W_F / mu of that cell (blocks 0 and 1 hold the same value)
    ii = np.arange(nc)
    off = 0.5 * d[ii]
    Coff = sp.csr_matrix((np.concatenate([off, off]),
                          (np.concatenate([ii, nc + ii]), np.concatenate([nc + ii, ii]))),
                         shape=(ntot, ntot))
    return (sp.diags(d, format="csr") + Coff).tocsr()


def build_system(inp: StokesInput, solid_side_rule: bool = True, min_face_liquid: float = 0.0) -> StokesSystem:
    """Assemble A and b.  ``solid_side_rule=False`` skips step 2 of the
    null-space elimination (kept only to show in a test why it is needed).

    ``min_face_liquid`` = eps > 0 floors the liquid fraction of live faces
    where it is the face's mass (K, the velocity recovery, the traction
    force): W_L^u -> max(W_L^u, eps).  The paper is silent on slivers; a
    face whose control volume holds a rounding-level amount of liquid (a
    level set that vanishes on lattice points) otherwise makes K, and the
    condition number, arbitrarily large.  eps = 0 (the default) is the
    paper's system unchanged."""
    S = StokesSystem(inp=inp)
    dim, n, h, dt = inp.dim, tuple(inp.n), inp.h, inp.dt
    sizes = sample_sizes(dim, n)
    S.sizes = sizes
    S.W_L, S.W_F = compute_fractions(inp)
    fk = O_.face_kinds(dim)
    uk = unknown_kinds(dim)

    S.WLu = np.concatenate([S.W_L[k] for k in fk])
    S.WFu = np.concatenate([S.W_F[k] for k in fk])
    S.rho = np.concatenate([np.ravel(r) for r in inp.rho])
    S.u_bc = np.concatenate([np.ravel(r) for r in inp.u_bc])
    S.u_star = np.concatenate([np.ravel(r) for r in inp.u_star])
    S.WLx = np.concatenate([S.W_L[k] for k in uk])
    S.WFx = np.concatenate([S.W_F[k] for k in uk])
    if dim == 2:
        mu_blocks = [inp.mu[0], inp.mu[1], inp.mu[0]]
    else:
        mu_blocks = [inp.mu[0], inp.mu[0], inp.mu[1], inp.mu[2], inp.mu[3], inp.mu[0]]
    S.mux = np.concatenate([np.ravel(m) for m in mu_blocks])

    S.M = sp.vstack([O_.deformation(n, h), O_.gradient_transpose(n, h)], format="csr")
    adj = S.M.copy()
    adj.data = np.ones_like(adj.data)

    # 1. grid boundary faces are wall
    effWF = S.WFu.copy()
    effWF[O_.boundary_face_mask(n)] = 0.0
    # 2. solid side: faces coupled to a zero-fluid-weight multiplier
    zwm = ((S.WLx > 0) & (S.WFx == 0)).astype(np.float64)
    S.invalid_face = (adj.T @ zwm > 0) & (effWF > 0) & solid_side_rule
    effWF[S.invalid_face] = 0.0
    S.effWF = effWF
    # 3. live / bad faces
    S.live = (effWF > 0) & (S.WLu > 0)
    S.bad = (effWF > 0) & (S.WLu == 0)
    S.WLm = np.where(S.live, np.maximum(S.WLu, min_face_liquid), S.WLu)   # face mass fraction
    S.K = np.zeros_like(effWF)
    S.K[S.live] = dt * effWF[S.live] / (S.rho[S.live] * S.WLm[S.live])
    # 4. free-surface side: unknowns coupled to a bad face
    touches_bad = (adj @ S.bad.astype(np.float64)) > 0
    cand = (S.WLx > 0) & ~touches_bad
    nunk = S.WLx.size
    nc = sizes["cell"]
    cell_blocks = [0] if dim == 2 else [0, 1]  # stress blocks living at cells
    boff = np.concatenate([[0], np.cumsum([sizes[k] for k in uk])])
    p_sl = slice(boff[-2], boff[-1])
    for blk in cell_blocks:
        cand[boff[blk]:boff[blk + 1]] = cand[p_sl]
    # 5. positive diagonal
    a_c = S.WLx * cand
    Bc = sp.diags(a_c) @ S.M
    diagBKB = np.asarray((Bc.multiply(Bc)) @ S.K).ravel()
    Cc = _stress_block_C(dim, n, S.WLx, S.WFx, S.mux, cand, sizes)
    diag = Cc.diagonal() + diagBKB
    active = cand & (diag > 0)
    for blk in cell_blocks:
        active[boff[blk]:boff[blk + 1]] = active[p_sl]
    S.active = active
    # 6. assemble on the active set
    S.a = S.WLx * active
    S.B = (sp.diags(S.a) @ S.M).tocsr()
    S.C = _stress_block_C(dim, n, S.WLx, S.WFx, S.mux, active, sizes)
    S.A = (S.C + S.B @ sp.diags(S.K) @ S.B.T + sp.diags((~active).astype(np.float64))).tocsr()
    S.A.eliminate_zeros()
    S.b = rhs(S)
    return S


def rhs(S: StokesSystem, u_star=None) -> np.ndarray:
    """b of eq. stokesmixedsystemspd with the prescribed-velocity terms (Section 6.2)."""
    us = S.u_star if u_star is None else u_star
    WSu = 1.0 - S.effWF
    v = S.effWF * us + WSu * S.u_bc
    WSx = 1.0 - S.WFx
    return S.a * (S.M @ v) - S.a * WSx * (S.M @ S.u_bc)


def traction_force(S: StokesSystem, x_bc: np.ndarray) -> np.ndarray:
    """Face force of prescribed surface pressure and deviatoric stress
    (Section 6.1), x_bc = (tau_BC, p_BC) in unknown order, at every sample:

        f = W_A^u (M^T x_BC) - M^T (W_A^x x_BC),   W_A = 1 - W_L (air fraction),

    with M^T = [D^T | G].  The section prints the opposite sign; with it a
    uniform surface pressure P0 on liquid at rest gives liquid pressure -P0.
    The boundary integral it starts from carries the traction's work with the
    liquid's outward normal while its integration by parts uses the air's, so
    the sign is taken that gives +P0 (tested).  The air fraction of an
    unknown's sample is 1 - W_L if the unknown is active and 1 if it was
    eliminated (Section 8): an eliminated unknown carries no liquid, and
    with this reading the uniform-pressure state is exact."""
    WAx = 1.0 - S.WLx * S.active
    WAu = 1.0 - S.WLu
    return WAu * (S.M.T @ x_bc) - S.M.T @ (WAx * x_bc)


def traction_u_star(S: StokesSystem, x_bc: np.ndarray, u_star=None) -> np.ndarray:
    """u* carrying the prescribed-traction terms: the force f enters the first
    block row of eq. stokesmixedsystem weighted like the mass term (by W_F^u,
    the same reading as for the prescribed-velocity terms), so eliminating the
    velocity gives u* + dt f / (rho W_L^u) on live faces and u* elsewhere.
    Solve with rhs(S, result) and recover with it."""
    us = S.u_star if u_star is None else u_star
    f = traction_force(S, x_bc)
    out = np.array(us, dtype=np.float64, copy=True)
    lv = S.live
    out[lv] = us[lv] + S.inp.dt / (S.rho[lv] * S.WLm[lv]) * f[lv]
    return out


def recover_velocity(S: StokesSystem, x: np.ndarray, u_star=None):
    """Face velocities from (tau, p); first block row of eq. stokesmixedsystem.

    Live faces: u* - dt/(rho W_L^u) (B^T x).  Faces with effective W_F^u = 0
    (solid, wall, invalid): u_BC.  Bad faces (fluid but no liquid): u*.
    """
    us = S.u_star if u_star is None else u_star
    Btx = S.B.T @ x
    u = np.where(S.effWF == 0, S.u_bc, us)
    lv = S.live
    u = u.copy()
    u[lv] = us[lv] - S.inp.dt / (S.rho[lv] * S.WLm[lv]) * Btx[lv]
    return u


def kkt_system(S: StokesSystem, face_force=None):
    """Indefinite KKT of eq. stokesmixedsystem on (live faces, active unknowns).

    Returns (matrix, rhs, live_index, active_index).  Row 1 keeps the paper's
    W_F^u scaling; the constraint rows carry the prescribed-velocity terms
    g = W_L^s [ -(R W_S^u u_BC)_s + W_S^s (R u_BC)_s ].
    """
    dt = S.inp.dt
    lv = np.flatnonzero(S.live)
    ac = np.flatnonzero(S.active)
    mass = (S.rho * S.effWF * S.WLm / dt)[lv]
    Bw = (S.B @ sp.diags(S.effWF)).tocsr()[ac][:, lv]
    Cm = S.C.tocsr()[ac][:, ac]
    top = sp.hstack([sp.diags(mass), Bw.T])
    bot = sp.hstack([Bw, -Cm])
    Kmat = sp.vstack([top, bot], format="csc")
    WSu = 1.0 - S.effWF
    WSx = 1.0 - S.WFx
    g = -S.a * (S.M @ (WSu * S.u_bc)) + S.a * WSx * (S.M @ S.u_bc)
    top_rhs = mass * S.u_star[lv]
    if face_force is not None:           # prescribed traction, weighted like the mass term
        top_rhs = top_rhs + (S.effWF * face_force)[lv]
    r = np.concatenate([top_rhs, g[ac]])
    return Kmat, r, lv, ac


def split_unknowns(S: StokesSystem, x: np.ndarray):
    """Unknown vector -> dict of field-shaped arrays (tau_*, p)."""
    nx, ny, nz = _nx_ny_nz(S.inp.n)
    out = {}
    o = 0
    for name, k in zip(unknown_names(S.inp.dim), unknown_kinds(S.inp.dim)):
        sz = S.sizes[k]
        out[name] = x[o:o + sz].reshape(G_.field_shape(k, nx, ny, nz))
        o += sz
    return out


def split_faces(S: StokesSystem, u: np.ndarray):
    nx, ny, nz = _nx_ny_nz(S.inp.n)
    out = []
    o = 0
    for k in O_.face_kinds(S.inp.dim):
        sz = S.sizes[k]
        out.append(u[o:o + sz].reshape(G_.field_shape(k, nx, ny, nz)))
        o += sz
    return out


def pressure_null_vectors(S: StokesSystem, rtol=1e-12):
    """Null vectors of A from liquid regions enclosed by solid (Section 8, last
    paragraph): per connected set of active cells joined by live faces, the
    vector with p = 1 / W_L^p there (so W_L^p p is constant) is kept if A
    maps it to zero.  Returned as a list of unknown-length vectors."""
    dim = S.inp.dim
    nunk = S.a.size
    nc = S.sizes["cell"]
    p0 = nunk - nc
    GT = S.M[p0:, :]  # cells x faces
    act_c = S.active[p0:]
    # cell-cell adjacency through live faces
    L = GT[:, S.live]
    L = L.copy(); L.data = np.ones_like(L.data)
    adjc = (L @ L.T).tocsr()
    adjc = adjc[act_c][:, act_c]
    from scipy.sparse.csgraph import connected_components
    ncomp, lab = connected_components(adjc, directed=False)
    idx_act = np.flatnonzero(act_c)
    out = []
    scale = abs(S.A).max()
    for c in range(ncomp):
        cells = idx_act[lab == c]
        v = np.zeros(nunk)
        v[p0 + cells] = 1.0 / S.a[p0 + cells]
        r = S.A @ v
        if np.abs(r).max() <= rtol * scale * np.abs(v).max():
            out.append(v)
    return out
