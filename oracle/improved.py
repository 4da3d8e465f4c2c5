"""Improved staggered Dslash with one-hop ("fat") and three-hop ("long", Naik) links, FP64
(test infrastructure only).

The paper's application, MILC's improved staggered dynamical code (Table 4, Sec. 4), spends
its time in this operator; the paper does not write it down.  Reading (the standard
improved staggered form):

    (D chi)(x) = sum_mu eta_mu(x) [ F_mu(x) chi(x+mu)    - F_mu(x-mu)^dag  chi(x-mu)
                                   + L_mu(x) chi(x+3mu)  - L_mu(x-3mu)^dag chi(x-3mu) ]

with the phases, boundaries and layouts of ``dslash``.  F and L are inputs: any 3x3 complex
link fields (the fat-link smearing coefficients are not in the paper).  ``long_links``
builds the Naik links L_mu(x) = c * U_mu(x) U_mu(x+mu) U_mu(x+2mu) from thin links.
Both hops change parity (1 and 3 are odd), so D is even/odd block off-diagonal again.
"""
from __future__ import annotations

import numpy as np

from . import geometry as geo
from .su3 import mult_su3_mat_vec, mult_adj_su3_mat_vec, mult_su3_nn


def long_links(U, dims, coeff):
    """L_mu(x) = coeff * U_mu(x) U_mu(x+mu) U_mu(x+2mu), canonical (4, V, 3, 3)."""
    Ul = geo.gauge_lattice(U, dims)
    L = np.empty_like(Ul)
    for mu in range(4):
        ax = geo.AXIS[mu]
        L[mu] = coeff * mult_su3_nn(mult_su3_nn(Ul[mu], np.roll(Ul[mu], -1, axis=ax)),
                                    np.roll(Ul[mu], -2, axis=ax))
    return L.reshape(np.shape(U))


def dslash_improved_full(F, L, chi_full, dims):
    """Stencil on the full lattice; chi_full of shape (Lt, Lz, Ly, Lx, 3)."""
    Fl = geo.gauge_lattice(F, dims)
    Ll = geo.gauge_lattice(L, dims)
    eta = geo.eta(dims)
    out = np.zeros_like(chi_full, dtype=np.complex128)
    for mu in range(4):
        ax = geo.AXIS[mu]
        hop = (mult_su3_mat_vec(Fl[mu], np.roll(chi_full, -1, axis=ax))
               - mult_adj_su3_mat_vec(np.roll(Fl[mu], 1, axis=ax), np.roll(chi_full, 1, axis=ax))
               + mult_su3_mat_vec(Ll[mu], np.roll(chi_full, -3, axis=ax))
               - mult_adj_su3_mat_vec(np.roll(Ll[mu], 3, axis=ax), np.roll(chi_full, 3, axis=ax)))
        out += eta[mu][..., None] * hop
    return out


def dslash_improved_eo(F, L, chi_cb, dims, out_parity):
    """Half operator in checkerboard layout: (Vh, 3) on 1 - out_parity -> (Vh, 3)."""
    full = geo.cb_to_full(chi_cb, dims, 1 - out_parity)
    return geo.full_to_cb(dslash_improved_full(F, L, full, dims), dims, out_parity)


def dense_D_improved(F, L, dims):
    """Explicit (3V x 3V) matrix, site by site with integer neighbour arithmetic."""
    dims = tuple(dims)
    V = int(np.prod(dims))
    F = np.asarray(F).reshape(4, V, 3, 3)
    L = np.asarray(L).reshape(4, V, 3, 3)
    D = np.zeros((3 * V, 3 * V), dtype=np.complex128)

    def hop(x, mu, n):
        y = x
        for _ in range(abs(n)):
            y = geo.neighbour_lex(dims, y, mu, 1 if n > 0 else -1)
        return y

    for x in range(V):
        cx = geo.site_coords(dims, x)
        ph = (1, (-1) ** cx[0], (-1) ** (cx[0] + cx[1]), (-1) ** (cx[0] + cx[1] + cx[2]))
        for mu in range(4):
            for n, W in ((1, F), (3, L)):
                yf, yb = hop(x, mu, n), hop(x, mu, -n)
                for a in range(3):
                    for b in range(3):
                        D[3 * x + a, 3 * yf + b] += ph[mu] * W[mu, x, a, b]
                        D[3 * x + a, 3 * yb + b] -= ph[mu] * np.conj(W[mu, yb, b, a])
    return D


def dslash_improved_eo_sites(F, L, chi_cb, dims, out_parity, cb_sites):
    """``dslash_improved_eo`` at the chosen checkerboard sites only (plain loops)."""
    from .su3 import mult_su3_mat_vec as mv, mult_adj_su3_mat_vec as amv
    dims = tuple(dims)
    V = int(np.prod(dims))
    F = np.asarray(F).reshape(4, V, 3, 3)
    L = np.asarray(L).reshape(4, V, 3, 3)
    par = geo.parity(dims).reshape(-1)
    lex_of = np.flatnonzero(par == out_parity)

    def hop(x, mu, n):
        y = x
        for _ in range(abs(n)):
            y = geo.neighbour_lex(dims, y, mu, 1 if n > 0 else -1)
        return y

    out = np.zeros((len(cb_sites), 3), dtype=np.complex128)
    for i, cb in enumerate(cb_sites):
        x = int(lex_of[cb])
        c = geo.site_coords(dims, x)
        ph = (1, (-1) ** c[0], (-1) ** (c[0] + c[1]), (-1) ** (c[0] + c[1] + c[2]))
        acc = np.zeros(3, dtype=np.complex128)
        for mu in range(4):
            for n, W in ((1, F), (3, L)):
                yf, yb = hop(x, mu, n), hop(x, mu, -n)
                acc += ph[mu] * (mv(W[mu, x], chi_cb[yf >> 1]) - amv(W[mu, yb], chi_cb[yb >> 1]))
        out[i] = acc
    return out
