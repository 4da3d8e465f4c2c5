"""Domain decomposition of the staggered Dslash in the t direction (test infrastructure only).

The paper runs MILC in a "parallel" mode on several processes (Table 4) and its timing model
(Sec. 4) has a communication term that grows with the process count; it does not describe
the decomposition.  Reading used here (the one the library's halo path implements):

* the lattice (Lx, Ly, Lz, Lt) is cut into P sub-domains of Lt / P consecutive time slices,
  Lt / P even, so that a site keeps its parity and its checkerboard index follows from its
  local coordinates exactly as on a whole lattice (local t = global t - t0, t0 even);
* a field on one parity of the whole lattice is split by slicing: the sites of parity p in
  global slices [t0, t0 + Lt/P) are the contiguous checkerboard range
  [t0 * Vs/2, (t0 + Lt/P) * Vs/2), Vs = Lx Ly Lz; the gauge field likewise
  (U[mu][t0 * Vs : (t0 + Lt/P) * Vs]);
* the half Dslash of sub-domain k needs, besides its own links and input, one face from
  each t neighbour: ``ghost_fwd``, the input on the first slice of sub-domain k + 1, and
  ``ghost_bwd``, the input on the last slice of sub-domain k - 1 (both cyclic), each the
  Vs/2 sites of the input parity in checkerboard order within the slice -- which is the
  first / last Vs/2 entries of that sub-domain's own array; and the links U_t on the last
  slice of sub-domain k - 1 (all Vs sites, lex order within the slice), the backward links
  of its first slice.  A site (x, y, z) of either face has within-face index
  (x + Lx (y + Ly z)) >> 1.
"""
from __future__ import annotations

import numpy as np

from . import geometry as geo
from .su3 import mult_su3_mat_vec, mult_adj_su3_mat_vec


def local_dims(dims, P):
    Lx, Ly, Lz, Lt = dims
    if Lt % P or (Lt // P) % 2:
        raise ValueError(f"Lt = {Lt} must split into {P} even parts")
    return (Lx, Ly, Lz, Lt // P)


def split_gauge(U, dims, P):
    """Canonical (4, V, 3, 3) -> list of P local canonical gauges."""
    Vs = dims[0] * dims[1] * dims[2]
    n = dims[3] // P
    return [np.ascontiguousarray(U[:, k * n * Vs:(k + 1) * n * Vs]) for k in range(P)]


def split_vec(v, dims, P):
    """One-parity field (..., Vh, 3) -> list of P local fields (..., Vh/P, 3)."""
    Vsh = dims[0] * dims[1] * dims[2] // 2
    n = dims[3] // P
    return [np.ascontiguousarray(v[..., k * n * Vsh:(k + 1) * n * Vsh, :]) for k in range(P)]


def join_vec(parts):
    return np.concatenate(parts, axis=-2)


def faces(v_loc, dims_loc):
    """(first-slice face, last-slice face) of a local one-parity field (..., Vh_loc, 3)."""
    Vsh = dims_loc[0] * dims_loc[1] * dims_loc[2] // 2
    return v_loc[..., :Vsh, :].copy(), v_loc[..., -Vsh:, :].copy()


def last_slice_links(U_loc, dims_loc):
    """U_t on the last local slice, (Vs, 3, 3) in lex order within the slice: the ghost
    links the next sub-domain needs."""
    Vs = dims_loc[0] * dims_loc[1] * dims_loc[2]
    return U_loc[3, -Vs:].copy()


def dslash_eo_halo(U_loc, ghost_Ut, chi, ghost_bwd, ghost_fwd, dims_loc, out_parity):
    """Half Dslash on one sub-domain: ``chi`` (Vh_loc, 3) on parity 1 - out_parity, faces of
    the neighbours as described in the module docstring.  Plain loops with integer
    neighbour arithmetic; t hops that leave the sub-domain read the ghosts."""
    Lx, Ly, Lz, Lt = dims_loc
    V = Lx * Ly * Lz * Lt
    U_loc = np.asarray(U_loc).reshape(4, V, 3, 3)
    par = geo.parity(dims_loc).reshape(-1)
    sites = np.flatnonzero(par == out_parity)
    out = np.zeros((len(sites), 3), dtype=np.complex128)
    for n, x in enumerate(sites):
        c = geo.site_coords(dims_loc, int(x))
        eta = (1, (-1) ** c[0], (-1) ** (c[0] + c[1]), (-1) ** (c[0] + c[1] + c[2]))
        face = (c[0] + Lx * (c[1] + Ly * c[2])) >> 1
        acc = np.zeros(3, dtype=np.complex128)
        for mu in range(4):
            yf = geo.neighbour_lex(dims_loc, int(x), mu, +1)
            yb = geo.neighbour_lex(dims_loc, int(x), mu, -1)
            vf = ghost_fwd[face] if (mu == 3 and c[3] == Lt - 1) else chi[yf >> 1]
            if mu == 3 and c[3] == 0:
                Ub, vb = ghost_Ut[c[0] + Lx * (c[1] + Ly * c[2])], ghost_bwd[face]
            else:
                Ub, vb = U_loc[mu, yb], chi[yb >> 1]
            acc += eta[mu] * (mult_su3_mat_vec(U_loc[mu, x], vf) - mult_adj_su3_mat_vec(Ub, vb))
        out[n] = acc
    return out
