"""Thin Python binding of the C ABI in include/relaybp.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
compute of its own: device buffers are torch tensors passed by data pointer,
streams are torch CUDA streams.  Importing this module loads the in-tree
``librelaybp.so``; if it is missing, the import fails -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librelaybp.so")

RELAYBP_MSG_F64 = 0
RELAYBP_MSG_F32 = 1
RELAYBP_MSG_F16 = 2
RELAYBP_MSG_BF16 = 3
RELAYBP_MSG_I8 = 4
_DTYPES = {"f64": RELAYBP_MSG_F64, "f32": RELAYBP_MSG_F32, "f16": RELAYBP_MSG_F16, "bf16": RELAYBP_MSG_BF16,
           "i8": RELAYBP_MSG_I8}


class relaybp_csr(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32),
                ("indptr", ctypes.c_void_p), ("indices", ctypes.c_void_p)]


class relaybp_params(ctypes.Structure):
    _fields_ = [("gamma0", ctypes.c_double), ("pre_iter", ctypes.c_int32), ("num_sets", ctypes.c_int32),
                ("max_iterations", ctypes.c_int32), ("stop_nconv", ctypes.c_int32),
                ("gamma_min", ctypes.c_double), ("gamma_max", ctypes.c_double),
                ("msg_dtype", ctypes.c_int32), ("stop_all", ctypes.c_int32),
                ("carry_messages", ctypes.c_int32), ("int8_scale", ctypes.c_float), ("seed", ctypes.c_uint64)]


STATS_BYTES = 24      # sizeof(relaybp_shot_stats)


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2607_27644_b300.build` "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "relaybp_build": ([ctypes.POINTER(relaybp_csr), P, ctypes.POINTER(relaybp_csr),
                           ctypes.POINTER(relaybp_params), ctypes.POINTER(P)], ctypes.c_int),
        "relaybp_set_params": ([P, ctypes.POINTER(relaybp_params)], ctypes.c_int),
        "relaybp_set_learned": ([P, P, I32, P, I32], ctypes.c_int),
        "relaybp_set_learned_rows": ([P, P, I32, P, I32], ctypes.c_int),
        "relaybp_set_learned_legs": ([P, I32], ctypes.c_int),
        "relaybp_set_pair_kernel": ([P, I32, I32], ctypes.c_int),
        "relaybp_sizes": ([P, P, P, P, P], ctypes.c_int),
        "relaybp_sample": ([P, U64, U64, I64, P, P, P, P], ctypes.c_int),
        "relaybp_decode_batch": ([P, P, U64, I64, P, P, P, P], ctypes.c_int),
        "relaybp_decode_timed": ([P, P, U64, I64, P, P, P, P, P], ctypes.c_int),
        "relaybp_decode_trace": ([P, P, U64, I64, I32, P, P, P], ctypes.c_int),
        "relaybp_decode_batch_noalloc": ([P, P, U64, I64, P, P, P, P], ctypes.c_int),
        "relaybp_decode_host": ([P, P, U64, I64, P, P, P], ctypes.c_int),
        "relaybp_decode_flagged": ([P, P, U64, I64, P, P, P, I64, P, P, P, P], ctypes.c_int),
        "relaybp_osd": ([P, P, P, P, I64, I32, P, P, P], ctypes.c_int),
        "relaybp_spa_create": ([ctypes.POINTER(relaybp_csr), ctypes.POINTER(P)], ctypes.c_int),
        "relaybp_spa_llr": ([P, I32, P, ctypes.c_double, ctypes.c_double, U64, U64, I64, P, P], ctypes.c_int),
        "relaybp_spa_decode": ([P, I32, P, I64, I32, ctypes.c_double, I32, P, P, P, P, P], ctypes.c_int),
        "relaybp_spa_destroy": ([P], ctypes.c_int),
        "relaybp_windows_create": ([ctypes.POINTER(relaybp_csr), P, ctypes.POINTER(relaybp_csr), P, I32,
                                    ctypes.POINTER(relaybp_params), ctypes.POINTER(P)], ctypes.c_int),
        "relaybp_windows_info": ([P, P, P], ctypes.c_int),
        "relaybp_windows_handle": ([P, I32, ctypes.POINTER(P)], ctypes.c_int),
        "relaybp_windows_decode": ([P, P, U64, I64, P, P, P, P, P], ctypes.c_int),
        "relaybp_windows_destroy": ([P], ctypes.c_int),
        "relaybp_set_cluster_kernel": ([P, I32], ctypes.c_int),
        "relaybp_set_tail_offload": ([P, I32, I32, I64], ctypes.c_int),
        "relaybp_count_failures": ([P, P, P, P, I64, P, P], ctypes.c_int),
        "relaybp_launch_count": ([P], I64),
        "relaybp_sync": ([P, P], ctypes.c_int),
        "relaybp_learned_tape_bytes": ([P, I32, I32, I64], I64),
        "relaybp_learned_forward": ([P, I32, I32, P, I32, P, U64, I32, P, P, U64, I64, P, P, P], ctypes.c_int),
        "relaybp_learned_backward": ([P, I32, I32, P, I32, P, U64, I32, P, P, U64, I64, P, ctypes.c_double, P, P,
                                      P], ctypes.c_int),
        "relaybp_autotune": ([P, P, U64, I64, P, P, P, P, P], ctypes.c_int),
        "relaybp_group_create": ([P, I32, ctypes.POINTER(P)], ctypes.c_int),
        "relaybp_group_decode": ([P, P, P, P, P, P, P, P], ctypes.c_int),
        "relaybp_group_launch_count": ([P], I64),
        "relaybp_group_destroy": ([P], ctypes.c_int),
        "relaybp_probe_smem_read": ([I32, P, P, P], ctypes.c_int),
        "relaybp_destroy": ([P], ctypes.c_int),
        "relaybp_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()

EXPORTED = ["relaybp_build", "relaybp_set_params", "relaybp_set_learned", "relaybp_set_learned_rows",
            "relaybp_set_learned_legs", "relaybp_set_pair_kernel", "relaybp_set_cluster_kernel", "relaybp_set_tail_offload", "relaybp_sizes", "relaybp_sample", "relaybp_decode_batch",
            "relaybp_decode_timed", "relaybp_decode_trace", "relaybp_decode_batch_noalloc", "relaybp_decode_host", "relaybp_decode_flagged", "relaybp_osd", "relaybp_spa_create", "relaybp_spa_llr",
            "relaybp_spa_decode", "relaybp_spa_destroy", "relaybp_windows_create", "relaybp_windows_info",
            "relaybp_windows_handle", "relaybp_windows_decode", "relaybp_windows_destroy", "relaybp_count_failures", "relaybp_launch_count", "relaybp_sync",
            "relaybp_probe_smem_read", "relaybp_learned_tape_bytes", "relaybp_learned_forward",
            "relaybp_learned_backward", "relaybp_autotune", "relaybp_group_create", "relaybp_group_decode", "relaybp_group_launch_count",
            "relaybp_group_destroy", "relaybp_destroy", "relaybp_last_error"]


class RelayBPError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise RelayBPError(f"{what} failed ({rc}): {_lib.relaybp_last_error().decode()}")


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


@dataclass
class Params:
    """Decoder parameters (Sec. 6.1 decoder configuration list; Table 9 intervals)."""
    gamma0: float = 0.125
    pre_iter: int = 80
    num_sets: int = 1000
    max_iterations: int = 60
    stop_nconv: int = 5
    gamma_min: float = -0.24
    gamma_max: float = 0.66
    msg_dtype: str = "f32"
    stop_all: bool = False
    carry_messages: bool = False
    seed: int = 0
    int8_scale: float = 0.0      # int8 storage: value of one step (0: largest prior LLR / 24)

    def c(self) -> relaybp_params:
        return relaybp_params(self.gamma0, self.pre_iter, self.num_sets, self.max_iterations, self.stop_nconv,
                              self.gamma_min, self.gamma_max, _DTYPES[self.msg_dtype], int(self.stop_all),
                              int(self.carry_messages), float(self.int8_scale), self.seed)


@dataclass
class Handle:
    ptr: ctypes.c_void_p
    n_det: int
    n_loc: int
    n_obs: int
    n_edges: int
    _keep: list = field(default_factory=list)

    @property
    def wc(self):
        return (self.n_det + 31) // 32

    @property
    def wv(self):
        return (self.n_loc + 31) // 32

    @property
    def wk(self):
        return max(1, (self.n_obs + 31) // 32)


def relaybp_build(H_indptr, H_indices, n_det: int, n_loc: int, priors, O_indptr=None, O_indices=None,
                  n_obs: int = 0, params: Params | None = None) -> Handle:
    params = params or Params()
    Hp = np.ascontiguousarray(H_indptr, dtype=np.int32)
    Hi = np.ascontiguousarray(H_indices, dtype=np.int32)
    pr = np.ascontiguousarray(priors, dtype=np.float64)
    H = relaybp_csr(n_det, n_loc, _ptr(Hp), _ptr(Hi))
    O = None
    keep = [Hp, Hi, pr]
    if O_indptr is not None and n_obs > 0:
        Op = np.ascontiguousarray(O_indptr, dtype=np.int32)
        Oi = np.ascontiguousarray(O_indices, dtype=np.int32)
        O = relaybp_csr(n_obs, n_loc, _ptr(Op), _ptr(Oi))
        keep += [Op, Oi]
    out = ctypes.c_void_p()
    cp = params.c()
    _check(_lib.relaybp_build(ctypes.byref(H), _ptr(pr), ctypes.byref(O) if O is not None else None,
                              ctypes.byref(cp), ctypes.byref(out)), "relaybp_build")
    h = Handle(out, 0, 0, 0, 0)
    h.n_det, h.n_loc, h.n_obs, h.n_edges = relaybp_sizes(h)
    return h


def relaybp_build_dem(dem, params: Params | None = None) -> Handle:
    """relaybp_build from a workloads.dem.DEM."""
    return relaybp_build(dem.H_indptr, dem.H_indices, dem.n_det, dem.n_loc, dem.priors, dem.O_indptr,
                         dem.O_indices, dem.n_obs, params)


def relaybp_sizes(h: Handle) -> tuple[int, int, int, int]:
    c, v, k, e = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(_lib.relaybp_sizes(h.ptr, ctypes.byref(c), ctypes.byref(v), ctypes.byref(k), ctypes.byref(e)),
           "relaybp_sizes")
    return c.value, v.value, k.value, e.value


def relaybp_set_params(h: Handle, params: Params):
    cp = params.c()
    _check(_lib.relaybp_set_params(h.ptr, ctypes.byref(cp)), "relaybp_set_params")


def relaybp_set_learned(h: Handle, d_w=None, d_knots=None):
    """Attach FP32 learned weights [T, E] and knots [K+1] (device tensors the
    caller keeps alive); None, None restores the plain method."""
    T = 0 if d_w is None else d_w.shape[0]
    K = 0 if d_knots is None else d_knots.shape[0] - 1
    _check(_lib.relaybp_set_learned(h.ptr, _ptr(d_w), T, _ptr(d_knots), K), "relaybp_set_learned")
    h._keep = [d_w, d_knots]


def relaybp_set_learned_rows(h: Handle, d_wrow=None, d_knots=None):
    """Attach FP32 row-tied weights [T, C] and knots [K+1] (device tensors kept
    alive by the caller)."""
    T = 0 if d_wrow is None else d_wrow.shape[0]
    K = 0 if d_knots is None else d_knots.shape[0] - 1
    _check(_lib.relaybp_set_learned_rows(h.ptr, _ptr(d_wrow), T, _ptr(d_knots), K), "relaybp_set_learned_rows")
    h._keep = [d_wrow, d_knots]


def relaybp_set_cluster_kernel(h: Handle, cluster: int):
    """Decode each shot with a cluster of `cluster` CTAs (0: off)."""
    _check(_lib.relaybp_set_cluster_kernel(h.ptr, cluster), "relaybp_set_cluster_kernel")


def relaybp_set_tail_offload(h: Handle, legs: int, cluster: int = 16, max_shots: int = 0):
    """Hand shots about to start relay leg `legs` over to `cluster`-CTA
    clusters (legs = 0: off); outputs unchanged bit for bit."""
    _check(_lib.relaybp_set_tail_offload(h.ptr, legs, cluster, max_shots), "relaybp_set_tail_offload")


def relaybp_set_learned_legs(h: Handle, legs: int):
    _check(_lib.relaybp_set_learned_legs(h.ptr, legs), "relaybp_set_learned_legs")


def relaybp_set_pair_kernel(h: Handle, enable: bool, warps: int = 0):
    """Select the two-shot FP32 kernel (default where it applies) or the
    general one-shot-per-block kernel; warps per block of the former (0: the
    library's choice)."""
    _check(_lib.relaybp_set_pair_kernel(h.ptr, int(bool(enable)), warps), "relaybp_set_pair_kernel")


def relaybp_sample(h: Handle, seed: int, shot0: int, shots: int, d_syndromes, d_obs=None, d_errors=None,
                   stream=None):
    _check(_lib.relaybp_sample(h.ptr, seed, shot0, shots, _ptr(d_syndromes), _ptr(d_obs), _ptr(d_errors),
                               _stream(stream)), "relaybp_sample")


def relaybp_decode_batch(h: Handle, d_syndromes, shot0: int, shots: int, d_corrections=None, d_pred_obs=None,
                         d_stats=None, stream=None):
    _check(_lib.relaybp_decode_batch(h.ptr, _ptr(d_syndromes), shot0, shots, _ptr(d_corrections),
                                     _ptr(d_pred_obs), _ptr(d_stats), _stream(stream)), "relaybp_decode_batch")


def relaybp_decode_timed(h: Handle, d_syndromes, shot0: int, shots: int, d_times, d_corrections=None,
                         d_pred_obs=None, d_stats=None, stream=None):
    """relaybp_decode_batch recording each shot's device clock at start and retire
    into d_times [shots][2] (int64 tensor, nanoseconds)."""
    _check(_lib.relaybp_decode_timed(h.ptr, _ptr(d_syndromes), shot0, shots, _ptr(d_corrections), _ptr(d_pred_obs),
                                     _ptr(d_stats), _ptr(d_times), _stream(stream)), "relaybp_decode_timed")


def relaybp_decode_flagged(h: Handle, d_syndromes, shot0: int, shots: int, max_flagged: int, d_flag_idx, d_flag_post,
                           d_flag_count, d_corrections=None, d_pred_obs=None, d_stats=None, stream=None):
    """relaybp_decode_batch plus the unresolved shots' indices (int64) and final
    posteriors (float64 [max_flagged, V]); d_flag_count (int32 [1], zeroed)
    counts them."""
    _check(_lib.relaybp_decode_flagged(h.ptr, _ptr(d_syndromes), shot0, shots, _ptr(d_corrections), _ptr(d_pred_obs),
                                       _ptr(d_stats), max_flagged, _ptr(d_flag_idx), _ptr(d_flag_post),
                                       _ptr(d_flag_count), _stream(stream)), "relaybp_decode_flagged")


def relaybp_osd(h: Handle, d_syndromes, d_post, d_idx, n: int, lam: int, d_out_e, d_out_valid, stream=None):
    """OSD-lam of n shots (syndrome rows d_idx of d_syndromes, posteriors d_post)."""
    _check(_lib.relaybp_osd(h.ptr, _ptr(d_syndromes), _ptr(d_post), _ptr(d_idx), n, lam, _ptr(d_out_e),
                            _ptr(d_out_valid), _stream(stream)), "relaybp_osd")


class Spa:
    """A classical code on the device for BPSK-AWGN sum-product decoding."""

    def __init__(self, indptr, indices, m: int, n: int):
        ip = np.ascontiguousarray(indptr, dtype=np.int32)
        ix = np.ascontiguousarray(indices, dtype=np.int32)
        H = relaybp_csr(m, n, _ptr(ip), _ptr(ix))
        out = ctypes.c_void_p()
        _check(_lib.relaybp_spa_create(ctypes.byref(H), ctypes.byref(out)), "relaybp_spa_create")
        self.ptr, self.m, self.n = out, m, n

    def llr(self, sigma: float, seed: int, shot0: int, shots: int, d_llr, llr_max: float = 20.0, d_codewords=None,
            stream=None):
        _check(_lib.relaybp_spa_llr(self.ptr, _prec(d_llr.dtype), _ptr(d_codewords), sigma, llr_max, seed, shot0, shots,
                                    _ptr(d_llr), _stream(stream)), "relaybp_spa_llr")

    def decode(self, d_llr, shots: int, d_bits, d_iters, d_valid, d_post=None, max_iter: int = 100,
               llr_max: float = 20.0, early_stop: bool = True, stream=None):
        _check(_lib.relaybp_spa_decode(self.ptr, _prec(d_llr.dtype), _ptr(d_llr), shots, max_iter, llr_max,
                                       int(early_stop), _ptr(d_bits), _ptr(d_iters), _ptr(d_valid), _ptr(d_post),
                                       _stream(stream)), "relaybp_spa_decode")

    def destroy(self):
        if self.ptr:
            _lib.relaybp_spa_destroy(self.ptr)
            self.ptr = None


def relaybp_spa_create(indptr, indices, m: int, n: int) -> Spa:
    return Spa(indptr, indices, m, n)


def relaybp_spa_llr(spa: Spa, *a, **k):
    spa.llr(*a, **k)


def relaybp_spa_decode(spa: Spa, *a, **k):
    spa.decode(*a, **k)


def relaybp_spa_destroy(spa: Spa):
    spa.destroy()


class Windows:
    """Sliding-window decoder with a commit region of one round: one device
    handle per window, built at construction."""

    def __init__(self, H_indptr, H_indices, n_det: int, n_loc: int, priors, det_round, window: int,
                 O_indptr=None, O_indices=None, n_obs: int = 0, params: Params | None = None):
        params = params or Params()
        Hp = np.ascontiguousarray(H_indptr, dtype=np.int32)
        Hi = np.ascontiguousarray(H_indices, dtype=np.int32)
        pr = np.ascontiguousarray(priors, dtype=np.float64)
        dr = np.ascontiguousarray(det_round, dtype=np.int32)
        if dr.shape != (n_det,):
            raise ValueError(f"det_round has shape {dr.shape}, expected ({n_det},)")
        H = relaybp_csr(n_det, n_loc, _ptr(Hp), _ptr(Hi))
        O = None
        if O_indptr is not None and n_obs > 0:
            Op = np.ascontiguousarray(O_indptr, dtype=np.int32)
            Oi = np.ascontiguousarray(O_indices, dtype=np.int32)
            O = relaybp_csr(n_obs, n_loc, _ptr(Op), _ptr(Oi))
        out = ctypes.c_void_p()
        cp = params.c()
        _check(_lib.relaybp_windows_create(ctypes.byref(H), _ptr(pr), ctypes.byref(O) if O is not None else None,
                                           _ptr(dr), window, ctypes.byref(cp), ctypes.byref(out)),
               "relaybp_windows_create")
        self.ptr = out
        self.n_det, self.n_loc, self.n_obs = n_det, n_loc, n_obs
        nw, nr = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.relaybp_windows_info(self.ptr, ctypes.byref(nw), ctypes.byref(nr)), "relaybp_windows_info")
        self.n_windows, self.n_rounds = nw.value, nr.value

    @property
    def wc(self):
        return (self.n_det + 31) // 32

    @property
    def wv(self):
        return (self.n_loc + 31) // 32

    @property
    def wk(self):
        return max(1, (self.n_obs + 31) // 32)

    def handle(self, t: int) -> Handle:
        """Window t's decoder (owned by this object: never relaybp_destroy it)."""
        out = ctypes.c_void_p()
        _check(_lib.relaybp_windows_handle(self.ptr, t, ctypes.byref(out)), "relaybp_windows_handle")
        h = Handle(out, 0, 0, 0, 0)
        h.n_det, h.n_loc, h.n_obs, h.n_edges = relaybp_sizes(h)
        return h

    def decode(self, d_syndromes, shot0: int, shots: int, d_corrections=None, d_pred_obs=None, d_residual=None,
               d_converged=None, stream=None):
        _check(_lib.relaybp_windows_decode(self.ptr, _ptr(d_syndromes), shot0, shots, _ptr(d_corrections),
                                           _ptr(d_pred_obs), _ptr(d_residual), _ptr(d_converged), _stream(stream)),
               "relaybp_windows_decode")

    def destroy(self):
        if self.ptr:
            _lib.relaybp_windows_destroy(self.ptr)
            self.ptr = None


def relaybp_windows_create(dem, det_round, window: int, params: Params | None = None) -> Windows:
    """relaybp_windows_create from a workloads.dem.DEM and its detector rounds."""
    return Windows(dem.H_indptr, dem.H_indices, dem.n_det, dem.n_loc, dem.priors, det_round, window, dem.O_indptr,
                   dem.O_indices, dem.n_obs, params)


def relaybp_windows_info(w: Windows) -> tuple[int, int]:
    """(windows, rounds)."""
    return w.n_windows, w.n_rounds


def relaybp_windows_handle(w: Windows, t: int) -> Handle:
    return w.handle(t)


def relaybp_windows_decode(w: Windows, *a, **k):
    w.decode(*a, **k)


def relaybp_windows_destroy(w: Windows):
    w.destroy()


def relaybp_decode_batch_noalloc(h: Handle, d_syndromes, shot0: int, shots: int, d_corrections=None,
                                 d_pred_obs=None, d_stats=None, stream=None):
    """relaybp_decode_batch without any device allocation (fixed in-library scratch);
    concurrent calls on one device race -- issue them on one stream."""
    _check(_lib.relaybp_decode_batch_noalloc(h.ptr, _ptr(d_syndromes), shot0, shots, _ptr(d_corrections),
                                             _ptr(d_pred_obs), _ptr(d_stats), _stream(stream)),
           "relaybp_decode_batch_noalloc")


def relaybp_decode_trace(h: Handle, d_syndromes, shot0: int, shots: int, trace_iters: int, d_trace, d_stats=None,
                         stream=None):
    _check(_lib.relaybp_decode_trace(h.ptr, _ptr(d_syndromes), shot0, shots, trace_iters, _ptr(d_trace),
                                     _ptr(d_stats), _stream(stream)), "relaybp_decode_trace")


def relaybp_decode_host(h: Handle, h_syndromes, shot0: int, shots: int, h_pred_obs=None, h_stats=None,
                        stream=None):
    _check(_lib.relaybp_decode_host(h.ptr, _ptr(h_syndromes), shot0, shots, _ptr(h_pred_obs), _ptr(h_stats),
                                    _stream(stream)), "relaybp_decode_host")


def relaybp_count_failures(h: Handle, d_pred_obs, d_true_obs, d_stats, shots: int, d_counters, stream=None):
    _check(_lib.relaybp_count_failures(h.ptr, _ptr(d_pred_obs), _ptr(d_true_obs), _ptr(d_stats), shots,
                                       _ptr(d_counters), _stream(stream)), "relaybp_count_failures")


def relaybp_launch_count(h: Handle) -> int:
    return int(_lib.relaybp_launch_count(h.ptr))


def relaybp_sync(h: Handle, stream=None):
    """Wait for the work queued on the stream; raise on an asynchronous CUDA
    failure there."""
    _check(_lib.relaybp_sync(h.ptr, _stream(stream)), "relaybp_sync")


def relaybp_probe_smem_read(reps: int, d_sink, stream=None) -> float:
    """Launch the shared-memory bandwidth probe; returns the bytes it reads."""
    b = ctypes.c_double()
    _check(_lib.relaybp_probe_smem_read(reps, _ptr(d_sink), ctypes.byref(b), _stream(stream)),
           "relaybp_probe_smem_read")
    return b.value


def _prec(dtype) -> int:
    import torch
    if dtype == torch.float64:
        return RELAYBP_MSG_F64
    if dtype == torch.float32:
        return RELAYBP_MSG_F32
    raise ValueError("learned training runs in float32 or float64")


def relaybp_learned_tape_bytes(h: Handle, precision: int, T: int, shots: int) -> int:
    n = int(_lib.relaybp_learned_tape_bytes(h.ptr, precision, T, shots))
    if n < 0:
        raise RelayBPError("relaybp_learned_tape_bytes: invalid arguments")
    return n


def relaybp_learned_forward(h: Handle, w, knots, gamma_seed: int, d_syndromes, d_errors, shot0: int, shots: int,
                            d_tape, d_loss, stream=None, objective: int = 0):
    T, K = w.shape[0], knots.shape[0] - 1
    _check(_lib.relaybp_learned_forward(h.ptr, _prec(w.dtype), T, _ptr(w), K, _ptr(knots), gamma_seed, objective,
                                        _ptr(d_syndromes), _ptr(d_errors), shot0, shots, _ptr(d_tape), _ptr(d_loss),
                                        _stream(stream)), "relaybp_learned_forward")


def relaybp_learned_backward(h: Handle, w, knots, gamma_seed: int, d_errors, shot0: int, shots: int, d_tape,
                             scale: float, d_grad_w, d_grad_knots, stream=None, objective: int = 0,
                             d_syndromes=None):
    T, K = w.shape[0], knots.shape[0] - 1
    _check(_lib.relaybp_learned_backward(h.ptr, _prec(w.dtype), T, _ptr(w), K, _ptr(knots), gamma_seed, objective,
                                         _ptr(d_syndromes), _ptr(d_errors), shot0, shots, _ptr(d_tape), scale,
                                         _ptr(d_grad_w), _ptr(d_grad_knots), _stream(stream)),
           "relaybp_learned_backward")


def relaybp_autotune(h: Handle, d_syndromes, shot0: int, shots: int, stream=None) -> dict:
    L, NB, T, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(_lib.relaybp_autotune(h.ptr, _ptr(d_syndromes), shot0, shots, ctypes.byref(L), ctypes.byref(NB),
                                 ctypes.byref(T), ctypes.byref(ms), _stream(stream)), "relaybp_autotune")
    return dict(L=L.value, NB=NB.value, threads=T.value, ms=ms.value)


@dataclass
class Group:
    ptr: ctypes.c_void_p
    handles: list


def relaybp_group_create(handles: list) -> Group:
    arr = (ctypes.c_void_p * len(handles))(*[h.ptr.value if hasattr(h.ptr, "value") else h.ptr for h in handles])
    out = ctypes.c_void_p()
    _check(_lib.relaybp_group_create(arr, len(handles), ctypes.byref(out)), "relaybp_group_create")
    return Group(out, list(handles))


def _ptr_array(ts):
    if ts is None:
        return None
    return (ctypes.c_void_p * len(ts))(*[None if t is None else t.data_ptr() for t in ts])


def relaybp_group_decode(grp: Group, d_syndromes: list, shot0: list, shots: list, d_corrections=None,
                         d_pred_obs=None, d_stats=None, stream=None):
    n = len(grp.handles)
    s0 = (ctypes.c_uint64 * n)(*shot0)
    ns = (ctypes.c_int64 * n)(*shots)
    _check(_lib.relaybp_group_decode(grp.ptr, _ptr_array(d_syndromes), s0, ns, _ptr_array(d_corrections),
                                     _ptr_array(d_pred_obs), _ptr_array(d_stats), _stream(stream)),
           "relaybp_group_decode")


def relaybp_group_launch_count(grp: Group) -> int:
    return int(_lib.relaybp_group_launch_count(grp.ptr))


def relaybp_group_destroy(grp: Group):
    if grp.ptr:
        _check(_lib.relaybp_group_destroy(grp.ptr), "relaybp_group_destroy")
        grp.ptr = ctypes.c_void_p()


def relaybp_destroy(h: Handle):
    if h.ptr:
        _check(_lib.relaybp_destroy(h.ptr), "relaybp_destroy")
        h.ptr = ctypes.c_void_p()


def relaybp_last_error() -> str:
    return _lib.relaybp_last_error().decode()


def stats_view(stats):
    """Split a [shots, 6] int32 stats tensor into its fields."""
    return dict(converged=stats[:, 0], nsol=stats[:, 1], legs=stats[:, 2], iters=stats[:, 3],
                weight=stats.view(dtype=__import__("torch").float64)[:, 2])
