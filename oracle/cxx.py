"""ctypes binding of the FP64 C++ oracle (``oracle/cpp/oracle.cpp``) -- TEST INFRASTRUCTURE.

The same definitions as the numpy oracle (staggered Dslash, M = m^2 - D_eo D_oe, FP64 CG,
the Table 1 SU(3) routines), in plain C++ loops parallel over sites (OpenMP), so that the
oracle can also be timed on the host cores.  ``build()`` compiles it with g++ (no
architecture-specific flags); ``__graft_entry__.build()`` calls it.  Arrays are numpy
complex128 in the canonical layouts (gauge (4, V, 3, 3), vectors (Vh, 3)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpp", "oracle.cpp")
LIB = os.path.join(HERE, "_lib", "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp"
    cmd = ["g++", "-O3", "-std=c++17", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"g++ failed on {SRC}:\n{p.stderr}")
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        P, I, D, Lg = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
        L.ora_num_threads.restype = I
        L.ora_su3_mat_vec.argtypes = [Lg, P, P, P, I]
        L.ora_su3_mul.argtypes = [Lg, P, P, P, I, I]
        L.ora_dslash_eo.argtypes = [P, P, P, P, I, I]
        L.ora_normal_op.argtypes = [P, P, P, P, D, I]
        L.ora_cg.argtypes = [P, P, P, P, D, D, I, I, I, ctypes.POINTER(D)]
        L.ora_cg.restype = I
        _lib = L
    return _lib


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(dims):
    return (ctypes.c_int * 4)(*[int(d) for d in dims])


def max_threads() -> int:
    return int(lib().ora_num_threads())


def dslash_eo(U, chi_cb, dims, out_parity, threads=1):
    U, chi = _c(U), _c(chi_cb)
    out = np.empty_like(chi)
    lib().ora_dslash_eo(_dims(dims), _p(U), _p(chi), _p(out), int(out_parity), int(threads))
    return out


def normal_op(U, p_cb, mass, dims, threads=1):
    U, p = _c(U), _c(p_cb)
    out = np.empty_like(p)
    lib().ora_normal_op(_dims(dims), _p(U), _p(p), _p(out), float(mass), int(threads))
    return out


def cg(U, b, mass, dims, tol=1e-10, maxiter=10000, max_restarts=5, threads=1):
    U, b = _c(U), _c(b)
    x = np.empty_like(b)
    res = ctypes.c_double()
    it = lib().ora_cg(_dims(dims), _p(U), _p(b), _p(x), float(mass), float(tol), int(maxiter),
                      int(max_restarts), int(threads), ctypes.byref(res))
    return x, dict(iters=it, true_rel_resid=res.value)


def su3_mat_vec(A, b, adj=0):
    A, b = _c(A), _c(b)
    c = np.empty_like(b)
    lib().ora_su3_mat_vec(len(A), _p(A), _p(b), _p(c), int(adj))
    return c


def su3_mul(A, B, adjA=0, adjB=0):
    A, B = _c(A), _c(B)
    C = np.empty_like(A)
    lib().ora_su3_mul(len(A), _p(A), _p(B), _p(C), int(adjA), int(adjB))
    return C
