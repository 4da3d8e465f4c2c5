"""Conjugate gradient on M = m^2 - D_eo D_oe (even sites), FP64 and mixed precision
(test infrastructure only).

The paper does not describe the solver; it only motivates reduced precision by the larger
single-precision gains it measured (abstract; Sec. 4).  Readings used here:

* plain CG (Hestenes-Stiefel) from x0 = 0; the iterated residual only triggers the stop,
  after which the true residual ||b - M x|| / ||b|| is recomputed; if it is still above
  ``tol`` the residual is replaced by the true one and the iteration continues;
* mixed precision: the inner iteration multiplies by M built from links rounded to the
  inner storage format (``precision.quantize_links``), keeps its vectors rounded to
  ``vec_prec`` and forms every inner product in FP64.  A reliable update -- x_hi += x_lo,
  r_hi = b - M_fp64 x_hi in FP64, r_lo = round(r_hi), x_lo = 0, p kept -- happens every
  ``reliable_every`` inner iterations, or earlier when ||r_lo|| < delta * ||r_hi|| of the
  last update, or when the iterated residual reaches ``tol``.  The solve stops when the
  FP64 true residual is <= tol.  ``maxiter`` counts inner iterations.
* beta after a residual replacement (both solvers): the Polak-Ribiere form
      beta = max(0, Re<r_new, r_new - r_k>) / ||r_k||^2,
  r_k being the residual that entered the last iteration.  Between replacements
  <r_{k+1}, r_k> vanishes up to rounding, so this is the usual ||r_{k+1}||^2 / ||r_k||^2;
  at a replacement the new residual is not the iterated one and the Polak-Ribiere form
  (the choice of flexible CG, for operators that change between iterations: Golub & Ye
  1999, Notay 2000) keeps p conjugate-like where the Fletcher-Reeves form would carry a
  direction built from the rounded operator into the corrected residual.  With BF16 links
  (8 significant bits) on Haar links at m = 0.01 the Fletcher-Reeves form stalls near 1e-4
  while this form reaches 1e-10; with FP32 and FP16 links it takes as many or fewer
  iterations.  A negative value restarts p = r (beta = 0).
"""
from __future__ import annotations

import numpy as np

from .dslash import normal_op
from .precision import quantize_links, round_complex


def _dot(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


def _norm2(a):
    return float(np.vdot(a.reshape(-1), a.reshape(-1)).real)


def replaced_beta(r_new, r_k, rr_k):
    """beta after a residual replacement: max(0, Re<r_new, r_new - r_k>) / ||r_k||^2."""
    return max(0.0, (_norm2(r_new) - _dot(r_k, r_new).real) / rr_k)


def cg(U, b, mass, dims, tol=1e-10, maxiter=10000, max_restarts=5):
    """FP64 CG.  Returns (x, info) with info = dict(iters, true_rel_resid, restarts)."""
    b = np.asarray(b, dtype=np.complex128)
    bb = _norm2(b)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = _norm2(r)
    it = 0
    restarts = 0
    while it < maxiter:
        r_k = r.copy()
        Ap = normal_op(U, p, mass, dims)
        alpha = rr / _dot(p, Ap).real
        x += alpha * p
        r -= alpha * Ap
        rr_new = _norm2(r)
        it += 1
        beta = rr_new / rr
        if rr_new <= tol * tol * bb:
            r_true = b - normal_op(U, x, mass, dims)
            if np.sqrt(_norm2(r_true) / bb) <= tol or restarts >= max_restarts:
                break
            restarts += 1
            r = r_true
            rr_new = _norm2(r)
            beta = replaced_beta(r, r_k, rr)
        p = r + beta * p
        rr = rr_new
    res = np.sqrt(_norm2(b - normal_op(U, x, mass, dims)) / bb)
    return x, dict(iters=it, true_rel_resid=res, restarts=restarts)


def mixed_cg(U, b, mass, dims, tol=1e-10, prec="bf16", recon=12, vec_prec="f32",
             reliable_every=100, delta=0.1, maxiter=20000):
    """Mixed-precision CG with FP64 reliable updates.  Returns (x, info)."""
    b = np.asarray(b, dtype=np.complex128)
    U_lo = quantize_links(U, prec, recon)
    rnd = (lambda v: round_complex(v, vec_prec))
    bb = _norm2(b)
    x_hi = np.zeros_like(b)
    r_hi = b.copy()
    r_hi_norm = np.sqrt(bb)
    r = rnd(r_hi)
    x = np.zeros_like(b)
    p = r.copy()
    rr = _norm2(r)
    it = 0
    since = 0
    updates = 0
    while it < maxiter:
        r_k = r
        Ap = rnd(normal_op(U_lo, p, mass, dims))
        alpha = rr / _dot(p, Ap).real
        x = rnd(x + alpha * p)
        r = rnd(r - alpha * Ap)
        rr_new = _norm2(r)
        it += 1
        since += 1
        beta = rr_new / rr
        if (since >= reliable_every or np.sqrt(rr_new) < delta * r_hi_norm
                or rr_new <= tol * tol * bb):
            x_hi += x
            r_hi = b - normal_op(U, x_hi, mass, dims)
            r_hi_norm = np.sqrt(_norm2(r_hi))
            updates += 1
            since = 0
            if r_hi_norm <= tol * np.sqrt(bb):
                break
            x = np.zeros_like(b)
            r = rnd(r_hi)
            rr_new = _norm2(r)
            beta = replaced_beta(r, r_k, rr)
        p = rnd(r + beta * p)
        rr = rr_new
    if since:
        x_hi += x
    res = np.sqrt(_norm2(b - normal_op(U, x_hi, mass, dims)) / bb)
    return x_hi, dict(iters=it, reliable_updates=updates, true_rel_resid=res)
