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


@pytest.mark.parametrize("case", ["col_range", "unsorted", "single", "prior", "prior_nan", "prior_one", "params",
                                  "dtype"])
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
    elif case == "prior_nan":
        pri = [0.1, float("nan"), 0.1]
    elif case == "prior_one":
        pri = [0.1, 1.0, 0.1]
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


# Entry points whose first argument is a handle (or group): called with a NULL
# one and zero / NULL everywhere else, each returns a negative status (or -1
# for the size queries) and sets an error message -- no crash, no device work.
_HANDLE_CALLS = ["relaybp_set_params", "relaybp_set_learned", "relaybp_set_learned_rows", "relaybp_set_learned_legs",
                 "relaybp_sizes", "relaybp_sample", "relaybp_decode_batch", "relaybp_decode_timed",
                 "relaybp_decode_trace", "relaybp_decode_batch_noalloc", "relaybp_decode_host",
                 "relaybp_count_failures", "relaybp_learned_tape_bytes", "relaybp_learned_forward",
                 "relaybp_learned_backward", "relaybp_autotune", "relaybp_group_decode", "relaybp_windows_info",
                 "relaybp_set_tail_offload", "relaybp_sync",
                 "relaybp_windows_handle", "relaybp_windows_decode"]


@pytest.mark.parametrize("name", _HANDLE_CALLS)
def test_every_handle_call_rejects_a_null_handle(name):
    from paper_2607_27644_b300 import relaybp as R
    fn = getattr(R._lib, name)
    args = []
    for t in fn.argtypes:
        if t is ctypes.c_double:
            args.append(0.0)
        elif t in (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64):
            args.append(1 if t is ctypes.c_int64 else 0)          # one shot where a count is asked for
        else:
            args.append(None)
    assert fn(*args) < 0
    assert R.relaybp_last_error()


@pytest.mark.parametrize("case", ["window0", "negative_round", "no_rounds", "params"])
def test_windows_create_validates_before_any_device_work(case):
    from paper_2607_27644_b300 import relaybp as R
    H, keep = _csr(2, 3, [0, 2, 4], [0, 1, 1, 2])
    pr = np.full(3, 0.1)
    rounds = np.array([0, 1], dtype=np.int32)
    window, p = 1, R.Params(num_sets=3)
    if case == "window0":
        window = 0
    elif case == "negative_round":
        rounds = np.array([0, -1], dtype=np.int32)
    elif case == "no_rounds":
        H, keep = _csr(0, 3, [0], [])
        rounds = np.zeros(0, dtype=np.int32)
    elif case == "params":
        p = R.Params(pre_iter=0)
    out = ctypes.c_void_p()
    rc = R._lib.relaybp_windows_create(ctypes.byref(H), pr.ctypes.data_as(ctypes.c_void_p), None,
                                       rounds.ctypes.data_as(ctypes.c_void_p), window, ctypes.byref(p.c()),
                                       ctypes.byref(out))
    assert rc == -1 and out.value is None
    assert R.relaybp_last_error()


def test_group_create_rejects_empty_and_oversized_groups():
    from paper_2607_27644_b300 import relaybp as R
    out = ctypes.c_void_p()
    assert R._lib.relaybp_group_create(None, 0, ctypes.byref(out)) < 0 and out.value is None
    assert R._lib.relaybp_group_create(None, 17, ctypes.byref(out)) < 0 and out.value is None


@pytest.mark.parametrize("dtype,scale,ok", [("f32", 0.5, False), ("i8", -1.0, False), ("i8", float("inf"), False),
                                            ("f16", 0.0, True)])
def test_int8_scale_is_validated_before_any_device_work(dtype, scale, ok):
    """int8_scale must be 0 except for int8 storage, and finite and >= 0 there;
    a rejected parameter set fails before any CUDA call (so also here)."""
    from paper_2607_27644_b300 import relaybp as R
    cp = R.Params(msg_dtype=dtype, int8_scale=scale).c()
    H, keep = _csr(2, 3, [0, 2, 4], [0, 1, 1, 2])
    pr = np.full(3, 0.1)
    out = ctypes.c_void_p()
    rc = R._lib.relaybp_build(ctypes.byref(H), pr.ctypes.data_as(ctypes.c_void_p), None, ctypes.byref(cp),
                              ctypes.byref(out))
    msg = R.relaybp_last_error()
    if ok:
        assert rc == 0 or "int8_scale" not in msg
    else:
        assert rc == -1 and "int8_scale" in msg and out.value is None
    if rc == 0:
        R._lib.relaybp_destroy(out)


@pytest.mark.parametrize("priors,scale,ok", [([0.5, 0.5, 0.5], 0.0, False), ([0.5, 0.5, 0.5], 0.25, True),
                                             ([0.9, 0.95, 0.5], 0.0, True)])
def test_int8_automatic_step_needs_a_nonzero_prior_llr(priors, scale, ok):
    """The automatic int8 step is the largest |prior LLR| / 24: priors all 1/2
    make it 0, which is rejected before any device work; an explicit step, or
    priors above 1/2 (negative LLRs, counted by magnitude), are accepted."""
    from paper_2607_27644_b300 import relaybp as R
    cp = R.Params(msg_dtype="i8", int8_scale=scale).c()
    H, keep = _csr(2, 3, [0, 2, 4], [0, 1, 1, 2])
    pr = np.asarray(priors, dtype=np.float64)
    out = ctypes.c_void_p()
    rc = R._lib.relaybp_build(ctypes.byref(H), pr.ctypes.data_as(ctypes.c_void_p), None, ctypes.byref(cp),
                              ctypes.byref(out))
    msg = R.relaybp_last_error()
    if ok:
        assert rc == 0 or "automatic int8 step" not in msg
    else:
        assert rc == -1 and "automatic int8 step" in msg and out.value is None
    if rc == 0:
        R._lib.relaybp_destroy(out)
