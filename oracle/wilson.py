"""Wilson hopping term (the Wilson Dslash) and its half-spinor form, FP64 (test
infrastructure only).

Table 1 (Sec. 4) lists the two Wilson half-vector routines, mult_su3_mat_hwvec and
mult_adj_su3_mat_hwvec, without the operator they serve.  Readings (the standard Wilson
hopping term, with a sign that selects the operator or its adjoint):

    (D psi)(x) = sum_mu [ (1 - s gamma_mu) U_mu(x) psi(x+mu)
                        + (1 + s gamma_mu) U_mu(x-mu)^dag psi(x-mu) ],   s = +1 or -1

* gamma matrices in the DeGrand-Rossi (chiral) basis, ``GAMMA`` below; gamma_5 =
  gamma_x gamma_y gamma_z gamma_t = diag(1, 1, -1, -1);
* no mass, kappa or 1/2 factor; periodic boundaries; geometry, parity and checkerboard
  order as in ``geometry``;
* a spinor is a complex array ``(..., 4, 3)``, [spin][colour]; an even/odd field is
  ``(Vh, 4, 3)`` in checkerboard order.

``wilson_full`` is the definition with full 4x4 spin matrices; ``dense_wilson`` the explicit
matrix; ``wilson_full_projected`` the half-spinor form: (1 -+ gamma_mu) has rank two, so
the hop multiplies only a half Wilson vector (two spin components) by the link, with the
two Table 1 routines, and rebuilds the other two spin components afterwards.
"""
from __future__ import annotations

import numpy as np

from . import geometry as geo
from .su3 import mult_su3_mat_hwvec, mult_adj_su3_mat_hwvec

_i = 1j
GAMMA = np.array([
    # gamma_x
    [[0, 0, 0, _i], [0, 0, _i, 0], [0, -_i, 0, 0], [-_i, 0, 0, 0]],
    # gamma_y
    [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
    # gamma_z
    [[0, 0, _i, 0], [0, 0, 0, -_i], [-_i, 0, 0, 0], [0, _i, 0, 0]],
    # gamma_t
    [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
], dtype=np.complex128)
ID4 = np.eye(4, dtype=np.complex128)


def gamma5():
    return GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]


def spin_mul(G, psi):
    """(G psi)_s = sum_t G_st psi_t for a 4x4 spin matrix G and spinors (..., 4, 3)."""
    return np.einsum("st,...tc->...sc", G, psi)


def colour_mul(U, psi, adjoint=False):
    """U (or U^dag) times each spin component: U (..., 3, 3), psi (..., 4, 3)."""
    M = np.conj(np.swapaxes(U, -1, -2)) if adjoint else U
    return np.einsum("...ab,...sb->...sa", M, psi)


def cb_to_full(psi_cb, dims, par):
    full = np.zeros(geo.shape(dims) + (4, 3), dtype=np.complex128)
    full[geo.parity(dims) == par] = np.asarray(psi_cb)
    return full


def full_to_cb(psi_full, dims, par):
    return np.asarray(psi_full)[geo.parity(dims) == par]


def wilson_full(U, psi_full, dims, sign=1):
    """The definition on the full lattice; psi_full of shape (Lt, Lz, Ly, Lx, 4, 3)."""
    Ul = geo.gauge_lattice(U, dims)
    out = np.zeros_like(psi_full, dtype=np.complex128)
    for mu in range(4):
        ax = geo.AXIS[mu]
        fwd = colour_mul(Ul[mu], np.roll(psi_full, -1, axis=ax))
        bwd = colour_mul(np.roll(Ul[mu], 1, axis=ax), np.roll(psi_full, 1, axis=ax), adjoint=True)
        out += spin_mul(ID4 - sign * GAMMA[mu], fwd) + spin_mul(ID4 + sign * GAMMA[mu], bwd)
    return out


def wilson_eo(U, psi_cb, dims, out_parity, sign=1):
    """Half operator: (Vh, 4, 3) on parity 1 - out_parity -> (Vh, 4, 3) on out_parity."""
    full = cb_to_full(psi_cb, dims, 1 - out_parity)
    return full_to_cb(wilson_full(U, full, dims, sign), dims, out_parity)


def dense_wilson(U, dims, sign=1):
    """Explicit (12V x 12V) matrix, index 12*lex + 3*spin + colour, site by site with integer
    neighbour arithmetic (when an extent is 2 both hops reach the same site and add)."""
    dims = tuple(dims)
    V = int(np.prod(dims))
    U = np.asarray(U).reshape(4, V, 3, 3)
    D = np.zeros((12 * V, 12 * V), dtype=np.complex128)
    for x in range(V):
        for mu in range(4):
            yf = geo.neighbour_lex(dims, x, mu, 1)
            yb = geo.neighbour_lex(dims, x, mu, -1)
            Pm = ID4 - sign * GAMMA[mu]
            Pp = ID4 + sign * GAMMA[mu]
            for s in range(4):
                for t in range(4):
                    for a in range(3):
                        for b in range(3):
                            D[12 * x + 3 * s + a, 12 * yf + 3 * t + b] += Pm[s, t] * U[mu, x, a, b]
                            D[12 * x + 3 * s + a, 12 * yb + 3 * t + b] += Pp[s, t] * np.conj(U[mu, yb, b, a])
    return D


def half_project(psi, mu, eps):
    """Upper two spin components of (1 + eps gamma_mu) psi, a half Wilson vector (..., 2, 3).

    In the chiral basis gamma_mu = [[0, B], [B^dag, 0]] with B unitary, so
    (1 + eps gamma_mu) psi = (h, eps B^dag h) with h = psi_up + eps B psi_down.
    """
    B = GAMMA[mu][0:2, 2:4]
    return psi[..., 0:2, :] + eps * np.einsum("st,...tc->...sc", B, psi[..., 2:4, :])


def half_reconstruct(h, mu, eps):
    """The full spinor (h, eps B^dag h) of a projected half Wilson vector."""
    Bd = np.conj(GAMMA[mu][0:2, 2:4]).T
    return np.concatenate([h, eps * np.einsum("st,...tc->...sc", Bd, h)], axis=-2)


def wilson_full_projected(U, psi_full, dims, sign=1):
    """The same operator through half Wilson vectors and the two Table 1 routines."""
    Ul = geo.gauge_lattice(U, dims)
    out = np.zeros_like(psi_full, dtype=np.complex128)
    for mu in range(4):
        ax = geo.AXIS[mu]
        hf = half_project(np.roll(psi_full, -1, axis=ax), mu, -sign)
        out += half_reconstruct(mult_su3_mat_hwvec(Ul[mu], hf), mu, -sign)
        hb = half_project(np.roll(psi_full, 1, axis=ax), mu, +sign)
        out += half_reconstruct(mult_adj_su3_mat_hwvec(np.roll(Ul[mu], 1, axis=ax), hb), mu, +sign)
    return out


def wilson_eo_sites(U, psi_cb, dims, out_parity, cb_sites, sign=1):
    """``wilson_eo`` at the chosen checkerboard sites only (plain loops over the hops)."""
    dims = tuple(dims)
    V = int(np.prod(dims))
    U = np.asarray(U).reshape(4, V, 3, 3)
    lex_of = np.flatnonzero(geo.parity(dims).reshape(-1) == out_parity)
    out = np.zeros((len(cb_sites), 4, 3), dtype=np.complex128)
    for i, cb in enumerate(cb_sites):
        x = int(lex_of[cb])
        acc = np.zeros((4, 3), dtype=np.complex128)
        for mu in range(4):
            yf = geo.neighbour_lex(dims, x, mu, 1)
            yb = geo.neighbour_lex(dims, x, mu, -1)
            acc += spin_mul(ID4 - sign * GAMMA[mu], colour_mul(U[mu, x], psi_cb[yf >> 1]))
            acc += spin_mul(ID4 + sign * GAMMA[mu], colour_mul(U[mu, yb], psi_cb[yb >> 1], adjoint=True))
        out[i] = acc
    return out
