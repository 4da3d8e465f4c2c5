"""The C-ABI library builds, loads and exports every entry point declared in include/*.h;
host-side argument checks answer without touching a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "sizeof", "return"):
                names.add(name)
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1309_0551_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("su3_mul_batch", "su3_matvec_batch", "dslash_eo", "cg_solve", "lq_gauge_pack"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_null_context(lib):
    lib.lq_status_string.restype = ctypes.c_char_p
    assert lib.lq_status_string(0) == b"LQ_OK"
    assert lib.lq_status_string(3) == b"LQ_ERR_NOT_CONVERGED"
    # every entry point rejects a NULL context before touching the device
    assert lib.dslash_eo(None, None, None, None, 0, 1, 0, None) == 1
    assert lib.su3_mul_batch(None, None, None, None, ctypes.c_int64(1), 0, 0, 0, None) == 1
    assert lib.cg_solve(None, None, None, ctypes.c_double(0.1), None, None, 1, None, None, None) == 1
    assert lib.dslash_wilson_eo(None, None, None, None, 0, 1, 0, 1, None) == 1
    assert lib.su3_mat_hwvec_batch(None, None, None, None, ctypes.c_int64(1), 0, 0, None) == 1
