"""Python binding of ``liblqcd.so``, the GB300 staggered Dslash / CG / force library.

Argument marshalling only: every function here forwards to the C entry point of the same
name (``include/lqcd.h``) with tensor data pointers and the current CUDA stream; all
arithmetic runs in the library's CUDA kernels.  PyTorch supplies device memory and
streams.  The binding never falls back to another implementation: if the library is not
built, or a call fails, it raises.

Vector and matrix tensors use the canonical layouts of ``lqcd.h``: complex128 / complex64
tensors for FP64 / FP32, and real tensors with a trailing (re, im) axis of dtype bfloat16
or float16 for the 16-bit formats.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB, build as _build  # noqa: F401

LQ_F64, LQ_F32, LQ_BF16, LQ_F16 = 0, 1, 2, 3
PREC = {"f64": LQ_F64, "f32": LQ_F32, "bf16": LQ_BF16, "f16": LQ_F16}
PREC_NAME = {v: k for k, v in PREC.items()}
LQ_RECON_18, LQ_RECON_12 = 18, 12

_lib = None


class LQError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status}: {msg}")
        self.status = status


class lq_cg_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int),
                ("reliable_every", ctypes.c_int), ("delta", ctypes.c_double),
                ("check_every", ctypes.c_int)]


class lq_cg_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("true_rel_resid", ctypes.c_double), ("seconds", ctypes.c_double)]


def library_path() -> str:
    return LIB


def load(path: str | None = None):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1309_0551_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sigs = {
        "lq_create": ([ctypes.POINTER(P), I], I),
        "lq_destroy": ([P], I),
        "lq_last_error": ([P], ctypes.c_char_p),
        "lq_status_string": ([I], ctypes.c_char_p),
        "lq_set_tuning": ([P, I], I),
        "lq_set_tune_cache": ([P, ctypes.c_char_p], I),
        "lq_fp64_fma_rate": ([P, ctypes.POINTER(D)], I),
        "lq_sync": ([P, P], I),
        "lq_inject_status": ([P, ctypes.c_uint, P], I),
        "lq_selftest_wait_timeout": ([P, P], I),
        "lq_tune_report": ([P, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], I),
        "lq_gauge_pack": ([P, ctypes.POINTER(I), P, I, I, ctypes.POINTER(P), P], I),
        "lq_gauge_free": ([P, P], I),
        "lq_gauge_repack": ([P, P, P, P], I),
        "lq_gauge_set_halo": ([P, P, P, P], I),
        "dslash_eo_halo": ([P, P, P, P, P, P, I, I, I, D, P, D, P], I),
        "lq_vec_axpby": ([P, L, D, P, D, P, I, P], I),
        "lq_vec_dot": ([P, L, P, P, I, P, P], I),
        "md_leapfrog": ([P, P, P, P, P, D, D, I, P, ctypes.POINTER(D), P], I),
        "lq_gauge_info": ([P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                           ctypes.POINTER(ctypes.c_size_t)], I),
        "su3_mul_batch": ([P, P, P, P, L, I, I, I, P], I),
        "su3_matvec_batch": ([P, P, P, P, L, I, I, P], I),
        "su3_matvec_batch_ex": ([P, P, P, P, L, I, I, I, I, P], I),
        "dslash_eo": ([P, P, P, P, I, I, I, P], I),
        "cg_solve": ([P, P, P, D, P, P, I, ctypes.POINTER(lq_cg_params),
                      ctypes.POINTER(lq_cg_stats), P], I),
        "cg_solve_noalloc": ([P, P, P, D, P, P, I, ctypes.POINTER(lq_cg_params),
                              ctypes.POINTER(lq_cg_stats), P], I),
        "cg_solve_batched": ([P, I, P, P, P, P, P, I, ctypes.POINTER(lq_cg_params),
                              ctypes.POINTER(lq_cg_stats), P], I),
        "dslash_force": ([P, P, D, P, P, P, P, ctypes.POINTER(D), P], I),
        "dslash_eo_multi": ([P, I, P, P, P, I, I, I, P], I),
        "lq_vec_pair": ([P, I, I, P, P, P], I),
        "lq_vec_unpair": ([P, I, I, P, P, P], I),
        "dslash_eo_paired": ([P, P, P, P, I, I, P], I),
        "dslash_eo_improved": ([P, P, P, P, P, I, I, I, P], I),
        "lq_long_links": ([P, ctypes.POINTER(I), P, D, P, P], I),
        "su3_scalar_mult_add_batch": ([P, P, P, P, D, L, I, P], I),
        "su3_exp_mul_batch": ([P, P, P, P, D, L, I, P], I),
        "su3_mat_hwvec_batch": ([P, P, P, P, L, I, I, P], I),
        "dslash_wilson_eo": ([P, P, P, P, I, I, I, I, P], I),
    }
    for name, (args, res) in sigs.items():
        if hasattr(lib, name):
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
    _lib = lib
    return lib


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


class Context:
    """An ``lq_context``: device, scratch space, tuning table, last error."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        st = self.lib.lq_create(ctypes.byref(h), int(device))
        if st != 0:
            raise LQError(self.lib.lq_status_string(st).decode(), f"lq_create(device={device}) failed")
        self.handle = h
        self.device = device

    def check(self, st):
        if st != 0:
            raise LQError(self.lib.lq_status_string(st).decode(),
                          self.lib.lq_last_error(self.handle).decode())

    def close(self):
        if self.handle:
            self.lib.lq_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, mode):
        """0/False: off; 1/True: shapes for lone launches; 2: for concurrent launches."""
        self.check(self.lib.lq_set_tuning(self.handle, int(mode)))

    def sync(self, stream=None):
        """lq_sync: synchronise the stream and raise LQError (LQ_ERR_TIMEOUT) if a bounded
        device wait gave up since the last sync."""
        self.check(self.lib.lq_sync(self.handle, _stream(stream)))

    def inject_status(self, flags: int, stream=None):
        """lq_inject_status: set device status flags from the host (error-path tests)."""
        self.check(self.lib.lq_inject_status(self.handle, int(flags), _stream(stream)))

    def selftest_wait_timeout(self, stream=None):
        """lq_selftest_wait_timeout: a bounded TMA wait that runs out with nothing in flight."""
        self.check(self.lib.lq_selftest_wait_timeout(self.handle, _stream(stream)))

    def set_tune_cache(self, path):
        """lq_set_tune_cache: load launch shapes from `path` and save new ones to it."""
        self.check(self.lib.lq_set_tune_cache(self.handle, None if path is None else str(path).encode()))

    def fp64_fma_rate(self) -> float:
        """lq_fp64_fma_rate: measured FP64 FMA rate of the device in GFLOP/s."""
        g = ctypes.c_double()
        self.check(self.lib.lq_fp64_fma_rate(self.handle, ctypes.byref(g)))
        return g.value

    def tune_report(self) -> str:
        need = ctypes.c_size_t()
        self.check(self.lib.lq_tune_report(self.handle, None, 0, ctypes.byref(need)))
        buf = ctypes.create_string_buffer(need.value)
        self.check(self.lib.lq_tune_report(self.handle, buf, need.value, None))
        return buf.value.decode()


class Gauge:
    """A packed gauge field (``lq_gauge``), freed with the object."""

    def __init__(self, ctx: Context, handle, dims, prec, recon):
        self.ctx, self.handle, self.dims, self.prec, self.recon = ctx, handle, tuple(dims), prec, recon

    @property
    def nbytes(self) -> int:
        n = ctypes.c_size_t()
        self.ctx.check(self.ctx.lib.lq_gauge_info(self.handle, None, None, None, ctypes.byref(n)))
        return n.value

    def free(self):
        if self.handle:
            self.ctx.lib.lq_gauge_free(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def vec_prec_of(t) -> int:
    import torch
    return {torch.complex128: LQ_F64, torch.complex64: LQ_F32,
            torch.bfloat16: LQ_BF16, torch.float16: LQ_F16}[t.dtype]


def lq_gauge_pack(ctx: Context, dims, U, prec, recon=18, stream=None) -> Gauge:
    """Pack a canonical complex128 gauge field (4, V, 3, 3) on the device."""
    import torch
    if U.dtype != torch.complex128 or not U.is_cuda or not U.is_contiguous():
        raise ValueError("U must be a contiguous complex128 CUDA tensor of shape (4, V, 3, 3)")
    prec = PREC[prec] if isinstance(prec, str) else int(prec)
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    h = ctypes.c_void_p()
    ctx.check(ctx.lib.lq_gauge_pack(ctx.handle, d, _ptr(U), prec, int(recon), ctypes.byref(h),
                                    _stream(stream)))
    return Gauge(ctx, h, dims, prec, int(recon))


def dslash_eo(ctx: Context, U: Gauge, inp, out, out_parity: int, nrhs: int = 1, vec_prec=None,
              stream=None):
    """out = D inp on parity ``out_parity`` (canonical [nrhs][Vh][3] vectors)."""
    vp = vec_prec_of(inp) if vec_prec is None else vec_prec
    ctx.check(ctx.lib.dslash_eo(ctx.handle, U.handle, _ptr(inp), _ptr(out), int(out_parity),
                                int(nrhs), int(vp), _stream(stream)))


def dslash_eo_improved(ctx: Context, fat: Gauge, lng: Gauge, inp, out, out_parity: int, nrhs: int = 1,
                       vec_prec=None, stream=None):
    """Improved staggered half Dslash (fat one-hop + Naik three-hop links)."""
    vp = vec_prec_of(inp) if vec_prec is None else vec_prec
    ctx.check(ctx.lib.dslash_eo_improved(ctx.handle, fat.handle, lng.handle, _ptr(inp), _ptr(out),
                                         int(out_parity), int(nrhs), int(vp), _stream(stream)))


def dslash_wilson_eo(ctx: Context, U: Gauge, inp, out, out_parity: int, nrhs: int = 1, vec_prec=None,
                     sign: int = 1, stream=None):
    """Wilson hopping term on parity ``out_parity`` (canonical [nrhs][Vh][4][3] spinors);
    ``sign`` -1 applies the adjoint."""
    vp = vec_prec_of(inp) if vec_prec is None else vec_prec
    ctx.check(ctx.lib.dslash_wilson_eo(ctx.handle, U.handle, _ptr(inp), _ptr(out), int(out_parity),
                                       int(nrhs), int(vp), int(sign), _stream(stream)))


def lq_long_links(ctx: Context, dims, U, coeff: float, L, stream=None):
    """L_mu(x) = coeff * U_mu(x) U_mu(x+mu) U_mu(x+2mu) (canonical complex128 tensors)."""
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    ctx.check(ctx.lib.lq_long_links(ctx.handle, d, _ptr(U), float(coeff), _ptr(L), _stream(stream)))


def dslash_eo_multi(ctx: Context, Us, ins, outs, out_parity: int, nrhs: int = 1, vec_prec=None,
                    stream=None):
    """The half Dslash on several lattices in one persistent launch (lists, one per lattice)."""
    n = len(Us)
    P = ctypes.c_void_p
    vp = vec_prec_of(ins[0]) if vec_prec is None else vec_prec
    ctx.check(ctx.lib.dslash_eo_multi(ctx.handle, n, (P * n)(*[g.handle.value for g in Us]),
                                      (P * n)(*[t.data_ptr() for t in ins]),
                                      (P * n)(*[t.data_ptr() for t in outs]), int(out_parity), int(nrhs),
                                      int(vp), _stream(stream)))


def paired_numel(Vh: int, nrhs: int) -> int:
    """float32 elements of a paired colour-planar field: ((nrhs + 1) // 2) pairs x 3 colours
    x Vh sites x 4 reals."""
    return ((int(nrhs) + 1) // 2) * 3 * int(Vh) * 4


def lq_vec_pair(ctx: Context, Vh: int, nrhs: int, inp, out, stream=None):
    """Canonical complex64 [nrhs][Vh][3] -> paired colour-planar float32 layout."""
    ctx.check(ctx.lib.lq_vec_pair(ctx.handle, int(Vh), int(nrhs), _ptr(inp), _ptr(out), _stream(stream)))


def lq_vec_unpair(ctx: Context, Vh: int, nrhs: int, inp, out, stream=None):
    """Paired colour-planar float32 layout -> canonical complex64 [nrhs][Vh][3]."""
    ctx.check(ctx.lib.lq_vec_unpair(ctx.handle, int(Vh), int(nrhs), _ptr(inp), _ptr(out), _stream(stream)))


def dslash_eo_paired(ctx: Context, U: Gauge, inp, out, out_parity: int, nrhs: int, stream=None):
    """out = D inp on parity ``out_parity`` for ``nrhs`` right-hand sides in the paired layout."""
    ctx.check(ctx.lib.dslash_eo_paired(ctx.handle, U.handle, _ptr(inp), _ptr(out), int(out_parity),
                                       int(nrhs), _stream(stream)))


def su3_mul_batch(ctx: Context, A, B, C, n=None, adjA=0, adjB=0, prec=None, stream=None):
    """C[i] = op(A[i]) op(B[i]) (Table 1: mult_su3_nn / _an / _na)."""
    n = A.shape[0] if n is None else n
    prec = vec_prec_of(A) if prec is None else prec
    ctx.check(ctx.lib.su3_mul_batch(ctx.handle, _ptr(A), _ptr(B), _ptr(C), int(n), int(adjA),
                                    int(adjB), int(prec), _stream(stream)))


def su3_scalar_mult_add_batch(ctx: Context, A, B, C, s: float, n=None, prec=None, stream=None):
    """C = A + s B per 3x3 matrix (Table 1: scalar_mult_add_su3_matrix)."""
    n = A.numel() // 9 if n is None else n
    prec = vec_prec_of(A) if prec is None else prec
    ctx.check(ctx.lib.su3_scalar_mult_add_batch(ctx.handle, _ptr(A), _ptr(B), _ptr(C), float(s), int(n),
                                                int(prec), _stream(stream)))


def su3_exp_mul_batch(ctx: Context, P, U, out, eps: float, n=None, prec=None, stream=None):
    """out = reunit(exp(eps P) U) per link (P traceless anti-Hermitian)."""
    n = U.numel() // 9 if n is None else n
    prec = vec_prec_of(U) if prec is None else prec
    ctx.check(ctx.lib.su3_exp_mul_batch(ctx.handle, _ptr(P), _ptr(U), _ptr(out), float(eps), int(n),
                                        int(prec), _stream(stream)))


def su3_matvec_batch(ctx: Context, A, b, c, n=None, adj=0, prec=None, stream=None):
    """c[i] = op(A[i]) b[i] (Table 1: mult_su3_mat_vec / mult_adj_su3_mat_vec)."""
    n = A.shape[0] if n is None else n
    prec = vec_prec_of(A) if prec is None else prec
    ctx.check(ctx.lib.su3_matvec_batch(ctx.handle, _ptr(A), _ptr(b), _ptr(c), int(n), int(adj),
                                       int(prec), _stream(stream)))


def su3_matvec_batch_ex(ctx: Context, A, b, c, n, adj=0, mat_prec=LQ_F32, recon=18, vec_prec=None,
                        stream=None):
    """c[i] = op(A[i]) b[i] with matrices of ``mat_prec`` and ``recon`` reals (12: rows 0 and
    1 stored, [n][2][3]) and vectors of ``vec_prec`` (default: the matrices' precision)."""
    mat_prec = PREC[mat_prec] if isinstance(mat_prec, str) else int(mat_prec)
    vec_prec = mat_prec if vec_prec is None else (PREC[vec_prec] if isinstance(vec_prec, str) else int(vec_prec))
    ctx.check(ctx.lib.su3_matvec_batch_ex(ctx.handle, _ptr(A), _ptr(b), _ptr(c), int(n), int(adj), mat_prec,
                                          int(recon), vec_prec, _stream(stream)))


def su3_mat_hwvec_batch(ctx: Context, A, h, c, n=None, adj=0, prec=None, stream=None):
    """c[i] = op(A[i]) h[i] for half Wilson vectors (Table 1: mult_su3_mat_hwvec /
    mult_adj_su3_mat_hwvec)."""
    n = A.shape[0] if n is None else n
    prec = vec_prec_of(A) if prec is None else prec
    ctx.check(ctx.lib.su3_mat_hwvec_batch(ctx.handle, _ptr(A), _ptr(h), _ptr(c), int(n), int(adj),
                                          int(prec), _stream(stream)))


def _cg_call(fn, ctx, U_hi, U_lo, mass, b, x, nrhs, tol, maxiter, reliable_every, delta,
             check_every, stream):
    params = lq_cg_params(float(tol), int(maxiter), int(reliable_every), float(delta), int(check_every))
    stats = (lq_cg_stats * int(nrhs))()
    st = fn(ctx.handle, U_hi.handle, None if U_lo is None else U_lo.handle,
            float(mass), _ptr(b), _ptr(x), int(nrhs), ctypes.byref(params), stats, _stream(stream))
    out = [dict(iters=s.iters, reliable_updates=s.reliable_updates,
                true_rel_resid=s.true_rel_resid, seconds=s.seconds) for s in stats]
    if st != 0:
        err = LQError(ctx.lib.lq_status_string(st).decode(), ctx.lib.lq_last_error(ctx.handle).decode())
        err.stats = out
        raise err
    return out


def cg_solve(ctx: Context, U_hi: Gauge, U_lo: Gauge | None, mass: float, b, x, nrhs: int = 1,
             tol=1e-10, maxiter=10000, reliable_every=100, delta=0.1, check_every=20, stream=None):
    """Solve (m^2 - D_eo D_oe) x = b on even sites; returns a list of per-rhs stats dicts.
    Raises LQError on failure (including LQ_ERR_NOT_CONVERGED)."""
    return _cg_call(ctx.lib.cg_solve, ctx, U_hi, U_lo, mass, b, x, nrhs, tol, maxiter,
                    reliable_every, delta, check_every, stream)


def cg_solve_noalloc(ctx: Context, U_hi: Gauge, U_lo: Gauge | None, mass: float, b, x,
                     nrhs: int = 1, tol=1e-10, maxiter=10000, reliable_every=100, delta=0.1,
                     check_every=20, stream=None):
    """cg_solve for callers that cannot allocate GPU memory when they solve: scratch in the
    library's fixed 32 MiB device array, no allocation, stream, event or graph creation.
    Calls whose GPU work overlaps share that array and race."""
    return _cg_call(ctx.lib.cg_solve_noalloc, ctx, U_hi, U_lo, mass, b, x, nrhs, tol, maxiter,
                    reliable_every, delta, check_every, stream)


def cg_solve_batched(ctx: Context, U_hi, U_lo, masses, bs, xs, nrhs: int = 1, tol=1e-10,
                     maxiter=10000, reliable_every=100, delta=0.1, check_every=20, stream=None):
    """Batched CG over several lattices (lists of Gauge / tensors, one per lattice; U_lo None
    for FP64).  Returns per-lattice lists of per-rhs stats dicts."""
    n = len(U_hi)
    P = ctypes.c_void_p
    hi = (P * n)(*[g.handle.value for g in U_hi])
    lo = None if U_lo is None else (P * n)(*[g.handle.value for g in U_lo])
    m = (ctypes.c_double * n)(*[float(v) for v in masses])
    bp = (P * n)(*[t.data_ptr() for t in bs])
    xp = (P * n)(*[t.data_ptr() for t in xs])
    params = lq_cg_params(float(tol), int(maxiter), int(reliable_every), float(delta), int(check_every))
    stats = (lq_cg_stats * (n * int(nrhs)))()
    st = ctx.lib.cg_solve_batched(ctx.handle, n, hi, lo, m, bp, xp, int(nrhs), ctypes.byref(params),
                                  stats, _stream(stream))
    flat = [dict(iters=s.iters, reliable_updates=s.reliable_updates,
                 true_rel_resid=s.true_rel_resid, seconds=s.seconds) for s in stats]
    out = [flat[l * nrhs:(l + 1) * nrhs] for l in range(n)]
    if st != 0:
        err = LQError(ctx.lib.lq_status_string(st).decode(), ctx.lib.lq_last_error(ctx.handle).decode())
        err.stats = out
        raise err
    return out


def dslash_force(ctx: Context, U: Gauge, mass: float, chi, dSdU=None, force_TA=None, dSdchi=None,
                 want_S: bool = False, stream=None):
    """Gradients of S = Re chi^dag (m^2 - D_eo D_oe) chi (see lqcd.h); returns S (float) when
    want_S, else None.  Outputs are written into the given tensors."""
    S = ctypes.c_double(0.0)
    ctx.check(ctx.lib.dslash_force(ctx.handle, U.handle, float(mass), _ptr(chi), _ptr(dSdU),
                                   _ptr(force_TA), _ptr(dSdchi), ctypes.byref(S) if want_S else None,
                                   _stream(stream)))
    return S.value if want_S else None


def lq_gauge_repack(ctx: Context, g: Gauge, U, stream=None):
    """Re-pack the canonical complex128 field U into the existing gauge object g (no
    allocation)."""
    ctx.check(ctx.lib.lq_gauge_repack(ctx.handle, g.handle, _ptr(U), _stream(stream)))


def lq_gauge_set_halo(ctx: Context, g: Gauge, Ut_ghost, stream=None):
    """Attach the ghost links of a t-split sub-domain: the previous sub-domain's U_t on its
    last slice, a contiguous complex128 CUDA tensor (Vs, 3, 3)."""
    ctx.check(ctx.lib.lq_gauge_set_halo(ctx.handle, g.handle, _ptr(Ut_ghost), _stream(stream)))


def dslash_eo_halo(ctx: Context, U: Gauge, inp, ghost_bwd, ghost_fwd, out, out_parity: int, nrhs: int = 1,
                   a1: float = 0.0, w1=None, c: float = 1.0, vec_prec=None, stream=None):
    """out = a1 w1 + c D inp on a t-split sub-domain, the t hops leaving it reading the ghost
    faces (complex [nrhs][Vs/2][3] tensors) and the gauge's ghost links."""
    vp = vec_prec_of(inp) if vec_prec is None else vec_prec
    ctx.check(ctx.lib.dslash_eo_halo(ctx.handle, U.handle, _ptr(inp), _ptr(ghost_bwd), _ptr(ghost_fwd), _ptr(out),
                                     int(out_parity), int(nrhs), int(vp), float(a1), _ptr(w1), float(c),
                                     _stream(stream)))


def lq_vec_axpby(ctx: Context, a: float, x, b: float, y, stream=None):
    """y = a x + b y over a whole complex tensor (complex128 or complex64)."""
    ctx.check(ctx.lib.lq_vec_axpby(ctx.handle, int(x.numel()), float(a), _ptr(x), float(b), _ptr(y),
                                   vec_prec_of(x), _stream(stream)))


def lq_vec_dot(ctx: Context, x, y, result, stream=None):
    """result (a float64 CUDA tensor of one element) = Re<x, y>, summed in FP64."""
    ctx.check(ctx.lib.lq_vec_dot(ctx.handle, int(x.numel()), _ptr(x), _ptr(y), vec_prec_of(x), _ptr(result),
                                 _stream(stream)))


def md_leapfrog(ctx: Context, dims, U, P, chi, mass: float, eps: float, nsteps: int, work: Gauge | None = None,
                F=None, stream=None):
    """Leapfrog molecular dynamics for H = -1/2 sum Tr(P^2) + Re chi^dag (m^2 - D^2) chi with
    chi held fixed (C entry point md_leapfrog): P += eps/2 F; (U = reunit(exp(eps P) U);
    P += eps F) ..., the last momentum half step eps/2.  U, P: canonical complex128 CUDA
    tensors (4, V, 3, 3), updated in place; chi: (Vh, 3) complex128.  ``work`` (an FP64
    18-real Gauge of the lattice) and ``F`` (a tensor like U) are reused across calls when
    given.  Returns the final action S."""
    import torch
    if work is None:
        work = lq_gauge_pack(ctx, dims, U, LQ_F64, 18, stream)
    if F is None:
        F = torch.empty_like(U)
    S = ctypes.c_double(0.0)
    ctx.check(ctx.lib.md_leapfrog(ctx.handle, work.handle, _ptr(U), _ptr(P), _ptr(chi), float(mass), float(eps),
                                  int(nsteps), _ptr(F), ctypes.byref(S), _stream(stream)))
    return S.value
