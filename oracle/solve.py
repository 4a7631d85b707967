"""Solves of the SPD pressure-stress system (eq. stokesmixedsystemspd).

The method's result is the exact solution of a linear system, so the oracle
solves it directly where it can and by plain FP64 Jacobi-preconditioned CG
(the textbook algorithm; the paper used CG with a domain-decomposition
preconditioner, Section 9) where it cannot.  The relative residual is
||b - A x||_2 / ||b||_2, recomputed from scratch.
"""
import time

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def relative_residual(A, x, b):
    nb = np.linalg.norm(b)
    if nb == 0:
        return float(np.linalg.norm(A @ x))
    return float(np.linalg.norm(b - A @ x) / nb)


def solve_direct(A, b, null_vectors=()):
    """Sparse LU solve.  Each null vector v (enclosed-liquid pressure mode,
    Section 8, last paragraph: pressures that differ by a constant give the
    same velocities) is handled in two steps.  First the component of b
    along v is removed: a prescribed wall velocity whose discrete flux out of
    the enclosed region is not exactly zero (any non-rigid u_BC; the defect
    is a discretization error) makes A x = b inconsistent, and then fixing a
    pressure would put the whole defect into the equation of the pinned cell
    (a point source of mass there).  Then one entry of v is fixed to zero, as
    the paper suggests.  For consistent data the first step changes b only
    by rounding; the result is the solution that conjugate gradients
    converges to, up to the null component of x, which does not change the
    velocities."""
    n = A.shape[0]
    b = np.asarray(b, dtype=np.float64).copy()
    for v in null_vectors:
        b -= (v @ b) / (v @ v) * v
    pin = [int(np.flatnonzero(v)[0]) for v in null_vectors]
    keep = np.setdiff1d(np.arange(n), pin)
    Ak = A.tocsc()[keep][:, keep]
    x = np.zeros(n)
    x[keep] = spla.spsolve(Ak, b[keep])
    return x


def cholesky_ok(A):
    """Dense Cholesky of a small matrix: True if A is positive definite."""
    try:
        sla.cholesky(A.toarray(), lower=True)
        return True
    except sla.LinAlgError:
        return False


def pcg(A, b, tol=1e-8, max_iter=100000, x0=None, M_inv=None, true_check=True):
    """Jacobi-preconditioned conjugate gradient in FP64.

    Stops when the recurrence residual satisfies ||r|| <= tol ||b||; then the
    true residual is recomputed and, if it is above tol, CG restarts from the
    current x with r = b - A x.  Returns (x, iterations, true relative residual).
    """
    A = sp.csr_matrix(A)
    n = b.size
    if M_inv is None:
        d = A.diagonal()
        M_inv = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)
    x = np.zeros(n) if x0 is None else x0.astype(np.float64).copy()
    nb = np.linalg.norm(b)
    if nb == 0:
        return np.zeros(n), 0, 0.0
    it = 0
    for _restart in range(20):
        r = b - A @ x
        if np.linalg.norm(r) <= tol * nb:
            break
        z = M_inv * r
        p = z.copy()
        rz = r @ z
        while it < max_iter:
            q = A @ p
            pq = p @ q
            if pq <= 0:
                break
            alpha = rz / pq
            x += alpha * p
            r -= alpha * q
            it += 1
            if np.linalg.norm(r) <= tol * nb:
                break
            z = M_inv * r
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
        if not true_check or it >= max_iter:
            break
    return x, it, relative_residual(A, x, b)


def slot_coordinates_2d(S):
    """(i, j) slot of every unknown in the oracle's 2D order [txx, txy, p]."""
    nx, ny = S.inp.n
    ci = np.tile(np.arange(nx), ny); cj = np.repeat(np.arange(ny), nx)
    ni = np.tile(np.arange(nx + 1), ny + 1); nj = np.repeat(np.arange(ny + 1), nx + 1)
    return np.concatenate([ci, ni, ci]), np.concatenate([cj, nj, cj])


def additive_schwarz(S, r, core=4, ring=1):
    """z = sum_p R_p^T (R_p A R_p^T)^-1 R_p r (2D) over the patches whose core
    (core x core slots) holds an active unknown; patch p takes the active
    unknowns of its core widened by ``ring`` slots.  Inactive unknowns: z = r.
    Dense FP64 local solves; the definition of the GPU's Schwarz
    preconditioner written out."""
    A = S.A.tocsr()
    si, sj = slot_coordinates_2d(S)
    act = S.active
    z = np.where(act, 0.0, r)
    nx, ny = S.inp.n
    for J in range(0, (ny + 1 + core - 1) // core):
        for I in range(0, (nx + 1 + core - 1) // core):
            incore = act & (si >= core * I) & (si < core * I + core) & (sj >= core * J) & (sj < core * J + core)
            if not incore.any():
                continue
            m = act & (si >= core * I - ring) & (si < core * I + core + ring) & \
                (sj >= core * J - ring) & (sj < core * J + core + ring)
            idx = np.flatnonzero(m)
            Ap = A[idx][:, idx].toarray()
            z[idx] += np.linalg.solve(Ap, r[idx])
    return z


def schwarz_colour_patches(S, core=4, ring=1):
    """The patches of ``additive_schwarz`` (same cores, same widening), each
    with its colour (I mod 2) + 2 (J mod 2): [(colour, indices), ...].  Cores
    of one colour are one core apart, so with 2 ring <= core their widened
    patches are pairwise disjoint."""
    si, sj = slot_coordinates_2d(S)
    act = S.active
    nx, ny = S.inp.n
    out = []
    for J in range(0, (ny + 1 + core - 1) // core):
        for I in range(0, (nx + 1 + core - 1) // core):
            incore = act & (si >= core * I) & (si < core * I + core) & (sj >= core * J) & (sj < core * J + core)
            if not incore.any():
                continue
            m = act & (si >= core * I - ring) & (si < core * I + core + ring) & \
                (sj >= core * J - ring) & (sj < core * J + core + ring)
            out.append(((I % 2) + 2 * (J % 2), np.flatnonzero(m)))
    return out


def multiplicative_schwarz(S, r, core=4, ring=1, order=(0, 1, 2, 3, 2, 1, 0)):
    """Symmetric multiplicative overlapping Schwarz (2D), the form of
    preconditioner the paper used with CG (Section 9, the paragraph before
    Table solveriterations), on the patches of ``additive_schwarz`` coloured
    by ``schwarz_colour_patches``.  Starting from z = 0 and the residual
    e = r, each colour c of ``order`` in turn solves the local problems of
    its patches on the current residual, adds the corrections to z and
    updates the residual:

        d = sum_{p in c} R_p^T (R_p A R_p^T)^-1 R_p e,   z += d,   e -= A d.

    The patches of one colour are disjoint, so their solves are independent.
    A palindromic order makes the operator symmetric; its error propagator
    is I - M A = (I - B_c1 A)(I - B_c2 A) ... (I - B_c1 A) with
    B_c = sum_{p in c} R_p^T A_p^-1 R_p.  Inactive unknowns: z = r.  Dense
    FP64 local solves."""
    A = S.A.tocsr()
    act = S.active
    patches = schwarz_colour_patches(S, core, ring)
    z = np.zeros(r.size)
    e = np.where(act, r, 0.0)
    for c in order:
        d = np.zeros(r.size)
        for colour, idx in patches:
            if colour == c:
                d[idx] += np.linalg.solve(A[idx][:, idx].toarray(), e[idx])
        z += d
        e -= A @ d
    return np.where(act, z, r)


def time_pcg_iterations(A, b, iters):
    """Wall time of ``iters`` iterations of ``pcg`` (no convergence test), for
    the CPU baseline.  Returns seconds."""
    A = sp.csr_matrix(A)
    d = A.diagonal()
    M_inv = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)
    x = np.zeros(b.size)
    r = b.copy()
    z = M_inv * r
    p = z.copy()
    rz = r @ z
    t0 = time.perf_counter()
    for _ in range(iters):
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        np.linalg.norm(r)
        z = M_inv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return time.perf_counter() - t0
