"""Pseudofermion action, its gradients and the projected fermion force, FP64
(test infrastructure only).

The paper lists su3_projector (the outer product C_ij = a_i conj(b_j)), mult_su3_na and
scalar_mult_add_su3_matrix among the routines a lattice code spends its time in (Table 1,
Sec. 4) but does not write the force out.  Readings:

* chi lives on the even sites; S = Re chi^dag M chi = m^2 ||chi||^2 + ||D_oe chi||^2, with
  M = m^2 - D_eo D_oe (``dslash.normal_op``);
* dS/dchi = 2 M chi, in the convention where the gradient of a real function of a complex
  variable z = a + ib is dS/da + i dS/db (so the gradient of |z|^2 is 2z);
* dS/dU: with psi = D_oe chi on the odd sites, for each link U_mu(y)
      Z_mu(y) =  eta_mu(y) chi(y + mu) psi(y)^dag      y odd
      Z_mu(y) = -eta_mu(y) psi(y + mu) chi(y)^dag      y even
  (both outer products are su3_projector), and G_mu(y) = 2 Z_mu(y)^dag, so that
  dS = Re sum Tr(G^dag dU), i.e. G is the gradient in the same convention as dS/dchi;
* projected force F_mu(y) = TA(U_mu(y) G_mu(y)^dag) with
  TA(A) = (A - A^dag)/2 - Tr(A - A^dag)/6 * 1, so that for every traceless anti-Hermitian X,
  d/de S(exp(e X) U_mu(y)) at e = 0 equals Tr(X F_mu(y)).
"""
from __future__ import annotations

import numpy as np

from . import geometry as geo
from .dslash import dslash_eo, normal_op
from .su3 import adj, mult_su3_na, su3_projector


def action(U, chi, mass, dims):
    """S = m^2 ||chi||^2 + ||D_oe chi||^2 for chi (Vh, 3) on even sites."""
    psi = dslash_eo(U, chi, dims, 1)
    return mass * mass * float(np.vdot(chi, chi).real) + float(np.vdot(psi, psi).real)


def dS_dchi(U, chi, mass, dims):
    """2 M chi."""
    return 2.0 * normal_op(U, chi, mass, dims)


def link_gradient(U, chi, mass, dims):
    """G = dS/dU, canonical shape (4, V, 3, 3)."""
    psi = dslash_eo(U, chi, dims, 1)
    chi_f = geo.cb_to_full(chi, dims, 0)      # zero on odd sites
    psi_f = geo.cb_to_full(psi, dims, 1)      # zero on even sites
    eta = geo.eta(dims)
    G = np.empty((4,) + geo.shape(dims) + (3, 3), dtype=np.complex128)
    for mu in range(4):
        ax = geo.AXIS[mu]
        # each product vanishes on the parity it does not belong to
        Z = (su3_projector(np.roll(chi_f, -1, axis=ax), psi_f)
             - su3_projector(np.roll(psi_f, -1, axis=ax), chi_f))
        G[mu] = 2.0 * adj(eta[mu][..., None, None] * Z)
    return G.reshape(np.shape(U))


def ta(A):
    """Traceless anti-Hermitian part: (A - A^dag)/2 - Tr(A - A^dag)/6 * 1."""
    K = A - adj(A)
    tr = np.trace(K, axis1=-2, axis2=-1)
    return 0.5 * K - (tr / 6.0)[..., None, None] * np.eye(3)


def force_ta(U, G):
    """F = TA(U G^dag) per link."""
    return ta(mult_su3_na(U, G))


def link_gradient_sites(U, chi, mass, dims, links):
    """G = dS/dU at the chosen links only, ``links`` a list of (mu, lex); for lattices too
    large for ``link_gradient``.  psi is evaluated only at the odd sites the links touch."""
    from .dslash import dslash_eo_sites
    dims = tuple(dims)
    V = int(np.prod(dims))
    U = np.asarray(U).reshape(4, V, 3, 3)
    touched = sorted({s for _, s in links} | {geo.neighbour_lex(dims, s, mu, +1) for mu, s in links})
    odd = [s for s in touched if sum(geo.site_coords(dims, s)) % 2 == 1]
    cb_of_odd = {s: int(np.count_nonzero(geo.parity(dims).reshape(-1)[:s] == 1)) for s in odd}
    psi = dict(zip(odd, dslash_eo_sites(U, chi, dims, 1, [cb_of_odd[s] for s in odd])))
    chi_at = {}
    par = geo.parity(dims).reshape(-1)
    out = np.empty((len(links), 3, 3), dtype=np.complex128)
    for n, (mu, s) in enumerate(links):
        c = geo.site_coords(dims, s)
        eta = (1, (-1) ** c[0], (-1) ** (c[0] + c[1]), (-1) ** (c[0] + c[1] + c[2]))[mu]
        f = geo.neighbour_lex(dims, s, mu, +1)
        if par[s] == 1:
            e = f
            if e not in chi_at:
                chi_at[e] = chi[int(np.count_nonzero(par[:e] == 0))]
            Z = eta * su3_projector(chi_at[e], psi[s])
        else:
            if s not in chi_at:
                chi_at[s] = chi[int(np.count_nonzero(par[:s] == 0))]
            Z = -eta * su3_projector(psi[f], chi_at[s])
        out[n] = 2.0 * adj(Z)
    return out
