"""Molecular-dynamics update of the links and momenta, FP64 (test infrastructure only).

The paper lists scalar_mult_add_su3_matrix (C = A + s B, Table 1) among the routines of the
dynamical application; the update it serves is not written down.  Readings:

* momenta P_mu(x) are traceless anti-Hermitian 3x3 matrices, one per link;
* momentum update P <- P + s F with F the projected force (``force.force_ta``): for
  U' = P U and H = -1/2 sum Tr(P^2) + S(U), dH/dt = 0 requires P' = F, because
  d/de S(exp(e X) U) = Tr(X F) for traceless anti-Hermitian X;
* link update U <- reunit(exp(e P) U): exp through the eigen-decomposition of the
  Hermitian matrix -i e P; reunit re-orthonormalises rows 0 and 1 and sets
  row 2 = conj(row0 x row1);
* leapfrog: P += e/2 F(U); U <- reunit(exp(e P) U); P += e/2 F(U), repeated.
"""
from __future__ import annotations

import numpy as np

from .precision import third_row
from .su3 import mult_su3_nn, scalar_mult_add_su3_matrix


def expm_antihermitian(X):
    """exp(X) for a stack of anti-Hermitian 3x3 matrices (X = i H, H Hermitian)."""
    w, v = np.linalg.eigh(-1j * X)
    return (v * np.exp(1j * w)[..., None, :]) @ np.conj(np.swapaxes(v, -1, -2))


def reunitarize(U):
    """Rows 0, 1 Gram-Schmidt orthonormalised; row 2 = conj(row0 x row1)."""
    U = np.array(U, dtype=np.complex128)
    r0 = U[..., 0, :] / np.linalg.norm(U[..., 0, :], axis=-1)[..., None]
    r1 = U[..., 1, :] - np.sum(np.conj(r0) * U[..., 1, :], axis=-1)[..., None] * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1)[..., None]
    U[..., 0, :], U[..., 1, :] = r0, r1
    U[..., 2, :] = third_row(r0, r1)
    return U


def update_links(U, P, eps):
    """U <- reunit(exp(eps P) U), canonical (4, V, 3, 3)."""
    return reunitarize(mult_su3_nn(expm_antihermitian(eps * P), U))


def update_momenta(P, F, s):
    """P <- P + s F (scalar_mult_add_su3_matrix, Table 1)."""
    return scalar_mult_add_su3_matrix(P, F, s)


def kinetic(P):
    """-1/2 sum Tr(P^2) = 1/2 ||P||_F^2 for anti-Hermitian P."""
    return 0.5 * float(np.sum(np.abs(P) ** 2))
