"""The SU(3) routines of Table 1 (Sec. 4), FP64, batched over leading axes (test infrastructure).

A matrix is a complex array ``(..., 3, 3)`` indexed ``[row, col]``; a colour vector is
``(..., 3)``.  "Adjoint" is the conjugate transpose.  Each routine is the plain definition
from its Table 1 description; the adjoint mat-vec is written component by component as
Eqs. (1.1)-(2.3) give it (first output component there; the other two are the same sum
with the next column of A, as the text following those equations states).

The two Wilson half-vector routines of Table 1 (mult_su3_mat_hwvec, mult_adj_su3_mat_hwvec)
act on a half Wilson vector: two colour vectors (two spin components), array ``(..., 2, 3)``.
"""
from __future__ import annotations

import numpy as np


def adj(A):
    return np.conj(np.swapaxes(A, -1, -2))


def add_su3_vector(a, b):
    """Table 1: c = a + b."""
    return a + b


def scalar_mult_add_su3_vector(a, b, s):
    """Table 1: c = a + s*b (s real)."""
    return a + s * b


def sub_four_su3_vecs(a, b):
    """Table 1: a - (b[0] + b[1] + b[2] + b[3]); ``b`` has a leading axis of length 4."""
    return a - (b[0] + b[1] + b[2] + b[3])


def mult_su3_mat_vec(A, b):
    """Table 1: c_i = sum_j A_ij b_j."""
    return np.einsum("...ij,...j->...i", A, b)


def mult_adj_su3_mat_vec(A, b):
    """Table 1 / Eqs. (1.1)-(2.3): c = A^dag b, in real arithmetic:

    c_i.re = sum_k  A_ki.re * b_k.re + A_ki.im * b_k.im      (1.1)-(1.3) for i = 0
    c_i.im = sum_k  A_ki.re * b_k.im - A_ki.im * b_k.re      (2.1)-(2.3) for i = 0
    """
    Ar, Ai = A.real, A.imag
    br, bi = b.real, b.imag
    re = np.zeros(np.broadcast_shapes(A.shape[:-2], b.shape[:-1]) + (3,))
    im = np.zeros_like(re)
    for i in range(3):
        for k in range(3):
            re[..., i] += Ar[..., k, i] * br[..., k] + Ai[..., k, i] * bi[..., k]
            im[..., i] += Ar[..., k, i] * bi[..., k] - Ai[..., k, i] * br[..., k]
    return re + 1j * im


def mult_adj_su3_mat_vec_4dir(A, b):
    """Table 1: four outputs c[mu] = A[mu]^dag b; ``A`` has a leading axis of length 4."""
    return np.stack([mult_adj_su3_mat_vec(A[mu], b) for mu in range(4)])


def mult_adj_su3_mat_4vec(A, b):
    """Table 1: the adjoint of each of four matrices times one vector, four separate outputs."""
    return tuple(mult_adj_su3_mat_vec(A[mu], b) for mu in range(4))


def mult_su3_mat_vec_sum_4dir(A, b):
    """Table 1: c = sum_mu A[mu] b[mu]."""
    return sum(mult_su3_mat_vec(A[mu], b[mu]) for mu in range(4))


def mult_su3_nn(A, B):
    """Table 1: C = A B."""
    return np.einsum("...ik,...kj->...ij", A, B)


def mult_su3_an(A, B):
    """Table 1: C = A^dag B."""
    return np.einsum("...ki,...kj->...ij", np.conj(A), B)


def mult_su3_na(A, B):
    """Table 1: C = A B^dag."""
    return np.einsum("...ik,...jk->...ij", A, np.conj(B))


def scalar_mult_add_su3_matrix(A, B, s):
    """Table 1: C = A + s*B (s real)."""
    return A + s * B


def su3_projector(a, b):
    """Table 1: outer product C_ij = a_i * conj(b_j)."""
    return a[..., :, None] * np.conj(b[..., None, :])


def mult_su3_mat_hwvec(A, h):
    """Table 1: each of the two colour vectors of the half Wilson vector h times A."""
    return np.stack([mult_su3_mat_vec(A, h[..., s, :]) for s in range(2)], axis=-2)


def mult_adj_su3_mat_hwvec(A, h):
    """Table 1: each of the two colour vectors of the half Wilson vector h times A^dag."""
    return np.stack([mult_adj_su3_mat_vec(A, h[..., s, :]) for s in range(2)], axis=-2)
