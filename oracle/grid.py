"""Sample placement on the staggered (MAC) grid, Section 5 (Figs. macgrid, macgrid3d).

Pressure and the diagonal stresses sit at cell centres, velocity components on
the faces normal to them, and the off-diagonal stresses on nodes (2D) or on
cell edges (3D): tau_xy on edges parallel to z, tau_xz on edges parallel to y,
tau_yz on edges parallel to x.  Arrays are numpy arrays with x varying fastest
(shape ``(ny, nx)`` in 2D, ``(nz, ny, nx)`` in 3D for cells).

Level sets are sampled on the "half lattice": the lattice of spacing h/2 that
contains every sample position, padded by one half step on every side so that
the cell-sized control volume of every sample (including samples on the grid
boundary) lies inside it.  Lattice point (a, b[, c]) sits at
``origin + ((a-1) h/2, (b-1) h/2[, (c-1) h/2])``; so a = 1 is the grid's
lower x wall and the lattice has 2 nx + 3 points along x.
"""
import numpy as np

KINDS_2D = ("cell", "node", "u", "v")
KINDS_3D = ("cell", "u", "v", "w", "exy", "exz", "eyz")

# lattice offset (per axis, x first) of sample (i, j[, k]): a = 2 i + off
_OFF_2D = {"cell": (2, 2), "node": (1, 1), "u": (1, 2), "v": (2, 1)}
_OFF_3D = {
    "cell": (2, 2, 2),
    "u": (1, 2, 2), "v": (2, 1, 2), "w": (2, 2, 1),
    "exy": (1, 1, 2), "exz": (1, 2, 1), "eyz": (2, 1, 1),
}


def field_shape(kind, nx, ny, nz=None):
    """numpy shape (slowest axis first) of the field of samples of ``kind``.

    An axis has n + 1 samples where the sample sits on grid lines of that axis
    (lattice offset 1) and n samples where it sits between them (offset 2).
    """
    if nz is None:
        ox, oy = _OFF_2D[kind]
        return (ny + (oy == 1), nx + (ox == 1))
    ox, oy, oz = _OFF_3D[kind]
    return (nz + (oz == 1), ny + (oy == 1), nx + (ox == 1))


def lattice_shape(nx, ny, nz=None):
    if nz is None:
        return (2 * ny + 3, 2 * nx + 3)
    return (2 * nz + 3, 2 * ny + 3, 2 * nx + 3)


def lattice_index(kind, nx, ny, nz=None):
    """Half-lattice indices (a, b[, c]) of every sample of ``kind``, field-shaped."""
    shp = field_shape(kind, nx, ny, nz)
    if nz is None:
        ox, oy = _OFF_2D[kind]
        J, I = np.meshgrid(np.arange(shp[0]), np.arange(shp[1]), indexing="ij")
        return 2 * I + ox, 2 * J + oy
    ox, oy, oz = _OFF_3D[kind]
    K, J, I = np.meshgrid(np.arange(shp[0]), np.arange(shp[1]), np.arange(shp[2]), indexing="ij")
    return 2 * I + ox, 2 * J + oy, 2 * K + oz


def lattice_points(h, origin, nx, ny, nz=None):
    """Physical coordinates (x, y[, z]) of every half-lattice point, lattice-shaped."""
    shp = lattice_shape(nx, ny, nz)
    axes = [origin[d] + (np.arange(n) - 1) * (h / 2) for d, n in enumerate(reversed(shp))]
    grids = np.meshgrid(*reversed(axes), indexing="ij")
    return tuple(reversed(grids))


def sample_points(kind, h, origin, nx, ny, nz=None):
    """Physical coordinates (x, y[, z]) of every sample of ``kind``, field-shaped."""
    idx = lattice_index(kind, nx, ny, nz)
    return tuple(origin[d] + (idx[d] - 1) * (h / 2) for d in range(len(idx)))
