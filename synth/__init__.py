"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module draws random numbers and lays them out in the canonical host layouts; it holds
none of the staggered-Dslash / CG / force arithmetic.  Everything here is numpy, seeded
through ``numpy.random.PCG64`` so that a seed gives the same bytes on every machine.

Canonical layouts (the same ones the C-ABI accepts):

* lattice extents ``dims = (Lx, Ly, Lz, Lt)``, all even; ``V = Lx*Ly*Lz*Lt``, ``Vh = V/2``;
* lexicographic site index ``lex = x + Lx*(y + Ly*(z + Lz*t))``;
* gauge field ``U[mu][lex][a][b]``, complex128, shape ``(4, V, 3, 3)``: the SU(3) link from
  site ``x`` to ``x + mu`` (mu = 0..3 is x, y, z, t);
* fermion field on one parity, ``chi[rhs][cb][a]``, complex128, shape ``(nrhs, Vh, 3)``:
  checkerboard index ``cb = lex >> 1`` over the sites of that parity, in lex order.

Link generators:

* ``haar``: a 3x3 complex Gaussian matrix, orthonormalised column by column (Gram-Schmidt
  with re-orthogonalisation, which leaves every R_ii real and positive, so Q is Haar on
  U(3)), then multiplied by ``exp(-i*theta/3)`` with ``theta = arg det Q`` on the principal
  branch, giving det = 1.
* ``near_identity``: ``exp(i*eps*H)`` with H a Gaussian traceless Hermitian matrix, computed
  through the eigen-decomposition of H, then re-orthonormalised and det-fixed as above.
* ``unit``: every link the identity (free field).

Vectors: each colour component complex Gaussian with Re, Im ~ N(0, 1) independently.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng", "volume", "check_dims", "complex_gaussian", "haar_su3", "near_identity_su3",
    "gauge_field", "fermion_field", "su3_pairs", "momenta",
]

_CHUNK = 1 << 18  # matrices generated per batch, bounds host memory for large lattices


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def check_dims(dims) -> tuple:
    dims = tuple(int(d) for d in dims)
    if len(dims) != 4 or any(d <= 0 or d % 2 for d in dims):
        raise ValueError(f"lattice extents must be four positive even integers, got {dims}")
    return dims


def volume(dims) -> int:
    Lx, Ly, Lz, Lt = check_dims(dims)
    return Lx * Ly * Lz * Lt


def complex_gaussian(g: np.random.Generator, shape) -> np.ndarray:
    shape = tuple(shape)
    z = g.standard_normal(shape + (2,))
    return z[..., 0] + 1j * z[..., 1]


def _orthonormal_columns(Z: np.ndarray) -> np.ndarray:
    """Gram-Schmidt on the columns of a stack of 3x3 complex matrices (positive R_ii)."""
    Q = np.empty_like(Z)
    for j in range(3):
        v = Z[..., :, j].copy()
        for _ in range(2):  # a second sweep restores orthogonality to rounding level
            for k in range(j):
                qk = Q[..., :, k]
                v -= np.sum(np.conj(qk) * v, axis=-1)[..., None] * qk
        v /= np.sqrt(np.sum(np.abs(v) ** 2, axis=-1))[..., None]
        Q[..., :, j] = v
    return Q


def _fix_det(Q: np.ndarray) -> np.ndarray:
    theta = np.angle(np.linalg.det(Q))  # principal branch, (-pi, pi]
    return Q * np.exp(-1j * theta / 3.0)[..., None, None]


def haar_su3(g: np.random.Generator, n: int) -> np.ndarray:
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for s in range(0, n, _CHUNK):
        m = min(_CHUNK, n - s)
        out[s:s + m] = _fix_det(_orthonormal_columns(complex_gaussian(g, (m, 3, 3))))
    return out


def near_identity_su3(g: np.random.Generator, n: int, eps: float) -> np.ndarray:
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for s in range(0, n, _CHUNK):
        m = min(_CHUNK, n - s)
        A = complex_gaussian(g, (m, 3, 3))
        H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
        tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
        H = H - tr[:, None, None] * np.eye(3)
        w, vec = np.linalg.eigh(H)
        U = (vec * np.exp(1j * eps * w)[:, None, :]) @ np.conj(np.swapaxes(vec, -1, -2))
        out[s:s + m] = _fix_det(_orthonormal_columns(U))
    return out


def gauge_field(dims, kind: str = "haar", seed: int = 1, eps: float = 0.3) -> np.ndarray:
    """Canonical gauge field ``(4, V, 3, 3)`` complex128 (see module docstring)."""
    V = volume(dims)
    g = rng(seed)
    if kind == "haar":
        U = haar_su3(g, 4 * V)
    elif kind == "near_identity":
        U = near_identity_su3(g, 4 * V, eps)
    elif kind == "unit":
        U = np.broadcast_to(np.eye(3, dtype=np.complex128), (4 * V, 3, 3)).copy()
    else:
        raise ValueError(f"unknown gauge kind {kind!r}")
    return U.reshape(4, V, 3, 3)


def fermion_field(dims, nrhs: int = 1, seed: int = 2, sites: str = "half") -> np.ndarray:
    """Gaussian colour vectors, ``(nrhs, Vh, 3)`` (``sites='half'``) or ``(nrhs, V, 3)``."""
    V = volume(dims)
    n = V // 2 if sites == "half" else V
    return complex_gaussian(rng(seed), (nrhs, n, 3))


def spinor_field(dims, nrhs: int = 1, seed: int = 2, sites: str = "half") -> np.ndarray:
    """Gaussian Wilson spinors (4 spins x 3 colours), ``(nrhs, Vh, 4, 3)`` or ``(nrhs, V, 4, 3)``."""
    V = volume(dims)
    n = V // 2 if sites == "half" else V
    return complex_gaussian(rng(seed), (nrhs, n, 4, 3))


def hwvec_batch(n: int, seed: int = 2) -> tuple:
    """``n`` Haar SU(3) matrices and ``n`` Gaussian half Wilson vectors (2 x 3 complex)."""
    g = rng(seed)
    return haar_su3(g, n), complex_gaussian(g, (n, 2, 3))


def su3_pairs(n: int, seed: int = 2) -> tuple:
    """``n`` pairs of Haar SU(3) matrices (for the batched SU(3) products)."""
    g = rng(seed)
    return haar_su3(g, n), haar_su3(g, n)


def momenta(dims, seed: int = 8, scale: float = 1.0) -> np.ndarray:
    """Canonical (4, V, 3, 3) field of i*H, H a Gaussian traceless Hermitian 3x3 matrix
    (anti-Hermitian, traceless), scaled by ``scale``."""
    V = volume(dims)
    g = rng(seed)
    A = complex_gaussian(g, (4 * V, 3, 3))
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[:, None, None] * np.eye(3)
    return (1j * scale * H).reshape(4, V, 3, 3)
