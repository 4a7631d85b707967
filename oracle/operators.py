"""Centred staggered difference operators G and D, Section 5.

G is the discrete gradient from cell centres to faces and -G^T the discrete
divergence.  D is the discrete deformation rate acting on face velocities,
written for the unknowns the paper keeps (Section 5, trace elimination): with
tau_yy = -tau_xx in 2D (tau_zz = -(tau_xx + tau_yy) in 3D) and one unknown
per symmetric off-diagonal pair, the pairing tau : D(u) of the variational
form becomes

  2D: tau_xx (u_x - v_y) + tau_xy (u_y + v_x)
  3D: tau_xx (u_x - w_z) + tau_yy (v_y - w_z)
      + tau_xy (u_y + v_x) + tau_xz (u_z + w_x) + tau_yz (v_z + w_y),

so each row of D is one of these brackets, differenced at the stress sample.

Every difference is a centred one over one grid spacing: the derivative along
axis d of a face field at a sample located at half-lattice point L is
(f(L + e_d) - f(L - e_d)) / h, where the two faces sit half a cell away on
either side.  Faces outside the grid ("ghost" faces, needed only by stress
samples on the grid boundary) are dropped: they carry zero fluid weight and a
zero boundary velocity, so they contribute nothing to the matrix or the
right-hand side.

Orderings (all C-order flattenings of the ``grid.field_shape`` arrays):
  faces      2D [u, v]          3D [u, v, w]
  stresses   2D [tau_xx, tau_xy] 3D [tau_xx, tau_yy, tau_xy, tau_xz, tau_yz]
  pressure   cells
"""
import numpy as np
import scipy.sparse as sp

from . import grid as G_

FACES_2D = ("u", "v")
FACES_3D = ("u", "v", "w")
STRESS_2D = ("cell", "node")                 # tau_xx, tau_xy
STRESS_3D = ("cell", "cell", "exy", "exz", "eyz")  # tau_xx, tau_yy, tau_xy, tau_xz, tau_yz
STRESS_NAMES_2D = ("tau_xx", "tau_xy")
STRESS_NAMES_3D = ("tau_xx", "tau_yy", "tau_xy", "tau_xz", "tau_yz")


def _dims(n):
    return (n[0], n[1], None) if len(n) == 2 else tuple(n)


def _offsets(kinds, n):
    nx, ny, nz = _dims(n)
    sizes = [int(np.prod(G_.field_shape(k, nx, ny, nz))) for k in kinds]
    return np.concatenate([[0], np.cumsum(sizes)]), sizes


def _flat_index(kind, lat, n):
    """Flat index of the sample of ``kind`` at lattice coords ``lat`` (tuple of
    arrays, x first), or -1 where no such sample exists in the grid."""
    nx, ny, nz = _dims(n)
    off = (G_._OFF_2D if nz is None else G_._OFF_3D)[kind]
    shp = G_.field_shape(kind, nx, ny, nz)
    dims_xfirst = list(reversed(shp))
    ok = np.ones(lat[0].shape, dtype=bool)
    idx = []
    for d, L in enumerate(lat):
        q = L - off[d]
        ok &= (q % 2 == 0)
        i = q // 2
        ok &= (i >= 0) & (i < dims_xfirst[d])
        idx.append(i)
    flat = np.zeros(lat[0].shape, dtype=np.int64)
    stride = 1
    for d in range(len(lat)):
        flat += np.where(ok, idx[d], 0) * stride
        stride *= dims_xfirst[d]
    return np.where(ok, flat, -1)


def difference(target_kind, face_kind, axis, n, h):
    """Sparse (targets x faces of face_kind) centred difference d/d(axis)."""
    nx, ny, nz = _dims(n)
    lat = G_.lattice_index(target_kind, nx, ny, nz)
    lat = tuple(np.ravel(L) for L in lat)
    rows = np.arange(lat[0].size)
    nt = lat[0].size
    nf = int(np.prod(G_.field_shape(face_kind, nx, ny, nz)))
    R, C, V = [], [], []
    for sgn in (+1, -1):
        nb = list(lat)
        nb[axis] = lat[axis] + sgn
        f = _flat_index(face_kind, tuple(nb), n)
        ok = f >= 0
        R.append(rows[ok]); C.append(f[ok]); V.append(np.full(ok.sum(), sgn / h))
    return sp.csr_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))), shape=(nt, nf))


def _hstack_faces(blocks, n):
    return sp.hstack(blocks, format="csr")


def gradient_transpose(n, h):
    """G^T (cells x faces): (G^T u)_c = -(div u)_c."""
    faces = FACES_2D if len(n) == 2 else FACES_3D
    blocks = [-difference("cell", f, d, n, h) for d, f in enumerate(faces)]
    return _hstack_faces(blocks, n)


def deformation(n, h):
    """Reduced deformation operator D (stresses x faces), rows as in the module docstring."""
    if len(n) == 2:
        dx_u = difference("cell", "u", 0, n, h)
        dy_v = difference("cell", "v", 1, n, h)
        row_xx = sp.hstack([dx_u, -dy_v])
        dy_u = difference("node", "u", 1, n, h)
        dx_v = difference("node", "v", 0, n, h)
        row_xy = sp.hstack([dy_u, dx_v])
        return sp.vstack([row_xx, row_xy], format="csr")
    Z = lambda t, f: sp.csr_matrix((int(np.prod(G_.field_shape(t, *_dims(n)))),
                                    int(np.prod(G_.field_shape(f, *_dims(n))))))
    dx_u = difference("cell", "u", 0, n, h)
    dy_v = difference("cell", "v", 1, n, h)
    dz_w = difference("cell", "w", 2, n, h)
    row_xx = sp.hstack([dx_u, Z("cell", "v"), -dz_w])
    row_yy = sp.hstack([Z("cell", "u"), dy_v, -dz_w])
    row_xy = sp.hstack([difference("exy", "u", 1, n, h), difference("exy", "v", 0, n, h), Z("exy", "w")])
    row_xz = sp.hstack([difference("exz", "u", 2, n, h), Z("exz", "v"), difference("exz", "w", 0, n, h)])
    row_yz = sp.hstack([Z("eyz", "u"), difference("eyz", "v", 2, n, h), difference("eyz", "w", 1, n, h)])
    return sp.vstack([row_xx, row_yy, row_xy, row_xz, row_yz], format="csr")


def face_kinds(dim):
    return FACES_2D if dim == 2 else FACES_3D


def stress_kinds(dim):
    return STRESS_2D if dim == 2 else STRESS_3D


def boundary_face_mask(n):
    """Faces lying on the grid boundary (normal component on a wall), flattened."""
    nx, ny, nz = _dims(n)
    out = []
    for d, f in enumerate(face_kinds(len(n))):
        shp = G_.field_shape(f, nx, ny, nz)
        m = np.zeros(shp, dtype=bool)
        ax = len(shp) - 1 - d  # numpy axis of the face normal
        sl_lo = [slice(None)] * len(shp); sl_lo[ax] = 0
        sl_hi = [slice(None)] * len(shp); sl_hi[ax] = -1
        m[tuple(sl_lo)] = True
        m[tuple(sl_hi)] = True
        out.append(m.ravel())
    return np.concatenate(out)
