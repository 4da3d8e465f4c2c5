"""Lattice geometry for the oracle (test infrastructure only).

The paper describes the lattice only as sites with neighbours joined by SU(3) links
(Sec. 1); the conventions below are readings, stated once here:

* extents ``(Lx, Ly, Lz, Lt)``, all even, periodic in every direction;
* ``lex = x + Lx*(y + Ly*(z + Lz*t))``; a full-lattice field is stored as a numpy array of
  shape ``(Lt, Lz, Ly, Lx, ...)`` so that its C-order flattening is lex order, and direction
  mu = 0, 1, 2, 3 (x, y, z, t) is array axis 3, 2, 1, 0;
* parity ``(x + y + z + t) mod 2``, even = 0;
* checkerboard index ``cb = lex >> 1`` within a parity, i.e. the parity's sites in lex order;
* staggered phases eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y), eta_t = (-1)^(x+y+z).
"""
from __future__ import annotations

import numpy as np

AXIS = (3, 2, 1, 0)  # array axis of direction mu


def shape(dims):
    Lx, Ly, Lz, Lt = dims
    return (Lt, Lz, Ly, Lx)


def coords(dims):
    """Coordinate fields x, y, z, t, each of shape (Lt, Lz, Ly, Lx)."""
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in shape(dims)], indexing="ij")
    return x, y, z, t


def parity(dims):
    x, y, z, t = coords(dims)
    return (x + y + z + t) % 2


def eta(dims):
    """Staggered phases, array of shape (4, Lt, Lz, Ly, Lx) with entries +-1."""
    x, y, z, t = coords(dims)
    one = np.ones_like(x)
    return np.stack([one, (-1) ** x, (-1) ** (x + y), (-1) ** (x + y + z)]).astype(np.float64)


def gauge_lattice(U, dims):
    """Canonical gauge field (4, V, 3, 3) -> (4, Lt, Lz, Ly, Lx, 3, 3) (a view)."""
    return np.asarray(U).reshape((4,) + shape(dims) + (3, 3))


def cb_to_full(v_cb, dims, par):
    """Fermion field on parity ``par`` (Vh, 3) -> full lattice (Lt, Lz, Ly, Lx, 3), zero on
    the other parity."""
    full = np.zeros(shape(dims) + (3,), dtype=np.complex128)
    mask = parity(dims) == par
    full[mask] = np.asarray(v_cb)
    return full


def full_to_cb(v_full, dims, par):
    """Full-lattice field -> its values on parity ``par`` in checkerboard order (Vh, 3)."""
    mask = parity(dims) == par
    return np.asarray(v_full)[mask]


def neighbour_lex(dims, lex, mu, step):
    """Lex index of the site ``step`` (+1 or -1) hops from ``lex`` in direction mu, periodic.
    Plain integer arithmetic, written separately from the array shifts used by the stencil."""
    Lx, Ly, Lz, Lt = dims
    c = [lex % Lx, (lex // Lx) % Ly, (lex // (Lx * Ly)) % Lz, lex // (Lx * Ly * Lz)]
    c[mu] = (c[mu] + step) % dims[mu]
    return c[0] + Lx * (c[1] + Ly * (c[2] + Lz * c[3]))


def site_coords(dims, lex):
    Lx, Ly, Lz, Lt = dims
    return (lex % Lx, (lex // Lx) % Ly, (lex // (Lx * Ly)) % Lz, lex // (Lx * Ly * Lz))
