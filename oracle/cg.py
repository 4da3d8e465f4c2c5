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
  r_hi = b - M_fp64 x_hi in FP64, r_lo = round(r_hi), x_lo = 0, p kept, beta formed with the
  new r_lo -- happens every ``reliable_every`` inner iterations, or earlier when
  ||r_lo|| < delta * ||r_hi|| of the last update, or when the iterated residual reaches
  ``tol``.  The solve stops when the FP64 true residual is <= tol.  ``maxiter`` counts
  inner iterations.
"""
from __future__ import annotations

import numpy as np

from .dslash import normal_op
from .precision import quantize_links, round_complex


def _dot(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


def _norm2(a):
    return float(np.vdot(a.reshape(-1), a.reshape(-1)).real)


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
        Ap = normal_op(U, p, mass, dims)
        alpha = rr / _dot(p, Ap).real
        x += alpha * p
        r -= alpha * Ap
        rr_new = _norm2(r)
        it += 1
        if rr_new <= tol * tol * bb:
            r_true = b - normal_op(U, x, mass, dims)
            if np.sqrt(_norm2(r_true) / bb) <= tol or restarts >= max_restarts:
                break
            restarts += 1
            r = r_true
            rr_new = _norm2(r)
        p = r + (rr_new / rr) * p
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
        Ap = rnd(normal_op(U_lo, p, mass, dims))
        alpha = rr / _dot(p, Ap).real
        x = rnd(x + alpha * p)
        r = rnd(r - alpha * Ap)
        rr_new = _norm2(r)
        it += 1
        since += 1
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
        p = rnd(r + (rr_new / rr) * p)
        rr = rr_new
    if since:
        x_hi += x
    res = np.sqrt(_norm2(b - normal_op(U, x_hi, mass, dims)) / bb)
    return x_hi, dict(iters=it, reliable_updates=updates, true_rel_resid=res)
