"""CPU-side checks of the C-ABI library: it loads, exports every declared entry
point, and rejects invalid input on the host before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(relaybp_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2607_27644_b300 import build
    lib = ctypes.CDLL(build.build())
    names = _declared()
    assert "relaybp_build" in names and "relaybp_decode_batch" in names and "relaybp_sample" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_2607_27644_b300 import relaybp
    for n in _declared():
        assert hasattr(relaybp, n), n


def _csr(rows, cols, indptr, indices):
    from paper_2607_27644_b300.relaybp import relaybp_csr
    ip = np.ascontiguousarray(indptr, dtype=np.int32)
    ix = np.ascontiguousarray(indices, dtype=np.int32)
    return relaybp_csr(rows, cols, ip.ctypes.data_as(ctypes.c_void_p), ix.ctypes.data_as(ctypes.c_void_p)), (ip, ix)


@pytest.mark.parametrize("case", ["col_range", "unsorted", "single", "prior", "params", "dtype"])
def test_build_rejects_invalid_input(case):
    from paper_2607_27644_b300 import relaybp as R
    indptr, indices, pri = [0, 2, 4], [0, 1, 1, 2], [0.1, 0.1, 0.1]
    p = R.Params(num_sets=3)
    if case == "col_range":
        indices = [0, 1, 1, 3]
    elif case == "unsorted":
        indices = [1, 0, 1, 2]
    elif case == "single":
        indptr, indices = [0, 1, 3], [0, 1, 2]
    elif case == "prior":
        pri = [0.1, 0.0, 0.1]
    elif case == "params":
        p = R.Params(stop_nconv=0)
    elif case == "dtype":
        p = R.Params()
        cp = p.c()
        cp.msg_dtype = 9
    H, keep = _csr(2, 3, indptr, indices)
    pr = np.asarray(pri, dtype=np.float64)
    out = ctypes.c_void_p()
    cp = p.c() if case != "dtype" else cp
    rc = R._lib.relaybp_build(ctypes.byref(H), pr.ctypes.data_as(ctypes.c_void_p), None, ctypes.byref(cp),
                              ctypes.byref(out))
    assert rc in (-1, -3)
    assert out.value is None
    assert R.relaybp_last_error()


def test_null_handle_calls_fail_cleanly():
    from paper_2607_27644_b300 import relaybp as R
    assert R._lib.relaybp_decode_batch(None, None, 0, 1, None, None, None, None) == -1
    assert R._lib.relaybp_sample(None, 0, 0, 1, None, None, None, None) == -1
    assert R._lib.relaybp_destroy(None) == 0
