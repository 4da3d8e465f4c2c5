"""Storage rounding and 12-real link compression (test infrastructure only).

The paper's finding that single precision gains more than double (abstract; Sec. 4, the
paragraph after the timing model) is what the reduced-precision storage formats serve.
The formats themselves are readings: IEEE binary32, IEEE binary16 and bfloat16 (8
significant bits, binary32 exponent range), each reached from an FP64 value by ONE
round-to-nearest-even step (no intermediate rounding through binary32).

12-real compression keeps rows 0 and 1 of an SU(3) link and rebuilds row 2 as
conj(row0 x row1), which holds for every special unitary 3x3 matrix (the rows of U are
orthonormal and det U = 1).
"""
from __future__ import annotations

import numpy as np

PRECISIONS = ("f64", "f32", "bf16", "f16")


def round_bf16(x):
    """Round FP64 values to the nearest bfloat16 value (ties to even); returns FP64."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    bits = x.view(np.uint64)
    drop = np.uint64(52 - 7)                      # fraction bits removed (52 -> 7)
    lsb = (bits >> drop) & np.uint64(1)
    half = np.uint64((1 << (52 - 7 - 1)) - 1)
    rounded = (bits + half + lsb) & ~np.uint64((1 << (52 - 7)) - 1)
    return rounded.view(np.float64).reshape(x.shape)


def round_real(x, prec):
    x = np.asarray(x, dtype=np.float64)
    if prec == "f64":
        return x.copy()
    if prec == "f32":
        return x.astype(np.float32).astype(np.float64)
    if prec == "f16":
        return x.astype(np.float16).astype(np.float64)
    if prec == "bf16":
        return round_bf16(x)
    raise ValueError(f"unknown precision {prec!r}")


def round_complex(z, prec):
    z = np.asarray(z, dtype=np.complex128)
    return round_real(z.real, prec) + 1j * round_real(z.imag, prec)


def third_row(r0, r1):
    """Row 2 of an SU(3) matrix from rows 0 and 1: conj(r0 x r1)."""
    c = np.stack([r0[..., 1] * r1[..., 2] - r0[..., 2] * r1[..., 1],
                  r0[..., 2] * r1[..., 0] - r0[..., 0] * r1[..., 2],
                  r0[..., 0] * r1[..., 1] - r0[..., 1] * r1[..., 0]], axis=-1)
    return np.conj(c)


def quantize_links(U, prec, recon=18):
    """The links a kernel with (prec, recon) storage actually multiplies by, in FP64:
    every stored real rounded to ``prec``; with recon 12 row 2 is rebuilt from the
    rounded rows 0 and 1."""
    Q = round_complex(U, prec)
    if recon == 12:
        Q[..., 2, :] = third_row(Q[..., 0, :], Q[..., 1, :])
    elif recon != 18:
        raise ValueError("recon must be 18 or 12")
    return Q
