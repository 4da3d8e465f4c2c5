"""Staggered Dslash, its even/odd blocks and the normal operator, FP64 (test infrastructure).

The paper names the SU(3) routines a staggered lattice code spends its time in (Table 1,
Sec. 4) and says each site is updated from its neighbours through the links (Sec. 1); it
does not write the operator down.  The operator built from those routines is

    (D chi)(x) = sum_mu eta_mu(x) [ U_mu(x) chi(x + mu) - U_mu(x - mu)^dag chi(x - mu) ]

with no factor 1/2, periodic boundaries and the phases of ``geometry.eta`` (readings).  The
forward hop is mult_su3_mat_vec (summed over mu as in mult_su3_mat_vec_sum_4dir) and the
backward hop is mult_adj_su3_mat_vec (Eqs. (1.1)-(2.3)).  D maps one parity to the other;
``dslash_eo(U, chi, dims, p)`` is the block that produces parity ``p`` from parity ``1-p``.

Normal operator on even sites: M = m^2 - D_eo D_oe, where D_oe is the block producing odd
sites from even ones; since D is anti-Hermitian, M = m^2 + D_oe^dag D_oe (Hermitian,
positive definite).

``dense_D`` assembles D as an explicit (3V x 3V) matrix with its own loop over sites and
integer neighbour arithmetic; it shares nothing with the stencil and is the brute-force pin.
"""
from __future__ import annotations

import numpy as np

from . import geometry as geo
from .su3 import mult_su3_mat_vec, mult_adj_su3_mat_vec


def dslash_full(U, chi_full, dims):
    """Stencil D on the full lattice.  ``U`` canonical (4, V, 3, 3); ``chi_full`` of shape
    (Lt, Lz, Ly, Lx, 3).  Returns the same shape."""
    Ul = geo.gauge_lattice(U, dims)
    eta = geo.eta(dims)
    out = np.zeros_like(chi_full, dtype=np.complex128)
    for mu in range(4):
        ax = geo.AXIS[mu]
        chi_fwd = np.roll(chi_full, -1, axis=ax)       # chi(x + mu)
        chi_bwd = np.roll(chi_full, +1, axis=ax)       # chi(x - mu)
        U_bwd = np.roll(Ul[mu], +1, axis=ax)           # U_mu(x - mu)
        hop = mult_su3_mat_vec(Ul[mu], chi_fwd) - mult_adj_su3_mat_vec(U_bwd, chi_bwd)
        out += eta[mu][..., None] * hop
    return out


def dslash_eo(U, chi_cb, dims, out_parity):
    """Half Dslash in canonical checkerboard layout: ``chi_cb`` (Vh, 3) on parity
    1 - out_parity -> (Vh, 3) on ``out_parity``."""
    full = geo.cb_to_full(chi_cb, dims, 1 - out_parity)
    return geo.full_to_cb(dslash_full(U, full, dims), dims, out_parity)


def dslash_eo_multi(U, chi, dims, out_parity):
    """``dslash_eo`` applied to each right-hand side of ``chi`` (nrhs, Vh, 3)."""
    return np.stack([dslash_eo(U, c, dims, out_parity) for c in chi])


def normal_op(U, p_cb, mass, dims):
    """M p = m^2 p - D_eo (D_oe p) on even sites (p of shape (Vh, 3))."""
    return mass * mass * p_cb - dslash_eo(U, dslash_eo(U, p_cb, dims, 1), dims, 0)


def dense_D(U, dims):
    """Explicit matrix of D, index (lex, colour); built site by site (small lattices only).

    D[(x,a),(y,b)] = sum_mu eta_mu(x) ( [y = x+mu] U_mu(x)_ab - [y = x-mu] conj(U_mu(y)_ba) );
    where x+mu and x-mu coincide (extent 2) both terms land on the same entry and add.
    """
    dims = tuple(dims)
    V = int(np.prod(dims))
    U = np.asarray(U).reshape(4, V, 3, 3)
    D = np.zeros((3 * V, 3 * V), dtype=np.complex128)
    for x in range(V):
        cx = geo.site_coords(dims, x)
        phases = (1, (-1) ** cx[0], (-1) ** (cx[0] + cx[1]), (-1) ** (cx[0] + cx[1] + cx[2]))
        for mu in range(4):
            yf = geo.neighbour_lex(dims, x, mu, +1)
            yb = geo.neighbour_lex(dims, x, mu, -1)
            for a in range(3):
                for b in range(3):
                    D[3 * x + a, 3 * yf + b] += phases[mu] * U[mu, x, a, b]
                    D[3 * x + a, 3 * yb + b] -= phases[mu] * np.conj(U[mu, yb, b, a])
    return D


def parity_indices(dims, par):
    """Lex indices of the sites of parity ``par`` in checkerboard order."""
    return np.flatnonzero(geo.parity(dims).reshape(-1) == par)


def dense_block(D, dims, out_parity):
    """Rows of parity ``out_parity`` and columns of the other parity of a dense (3V x 3V)
    operator, both in checkerboard order with colour fastest."""
    rows = parity_indices(dims, out_parity)
    cols = parity_indices(dims, 1 - out_parity)
    r = (3 * rows[:, None] + np.arange(3)).reshape(-1)
    c = (3 * cols[:, None] + np.arange(3)).reshape(-1)
    return D[np.ix_(r, c)]


def dense_normal(U, mass, dims):
    """Dense M = m^2 - D_eo D_oe on even sites, (3Vh x 3Vh)."""
    D = dense_D(U, dims)
    Doe = dense_block(D, dims, 1)
    Deo = dense_block(D, dims, 0)
    return mass * mass * np.eye(Doe.shape[1]) - Deo @ Doe


def dslash_eo_sites(U, chi_cb, dims, out_parity, cb_sites):
    """``dslash_eo`` evaluated only at the checkerboard sites ``cb_sites`` of parity
    ``out_parity`` (for sampled checks on lattices too large for the full oracle).  Plain
    loops with integer neighbour arithmetic; ``chi_cb`` is (Vh, 3) on the other parity."""
    dims = tuple(dims)
    V = int(np.prod(dims))
    U = np.asarray(U).reshape(4, V, 3, 3)
    par = geo.parity(dims).reshape(-1)
    lex_of = {p: np.flatnonzero(par == p) for p in (0, 1)}
    out = np.zeros((len(cb_sites), 3), dtype=np.complex128)
    for n, cb in enumerate(cb_sites):
        x = int(lex_of[out_parity][cb])
        cx = geo.site_coords(dims, x)
        phases = (1, (-1) ** cx[0], (-1) ** (cx[0] + cx[1]), (-1) ** (cx[0] + cx[1] + cx[2]))
        acc = np.zeros(3, dtype=np.complex128)
        for mu in range(4):
            yf = geo.neighbour_lex(dims, x, mu, +1)
            yb = geo.neighbour_lex(dims, x, mu, -1)
            acc += phases[mu] * mult_su3_mat_vec(U[mu, x], chi_cb[yf >> 1])
            acc -= phases[mu] * mult_adj_su3_mat_vec(U[mu, yb], chi_cb[yb >> 1])
        out[n] = acc
    return out
