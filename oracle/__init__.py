"""CPU oracle for the Relay-BP hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline / reference
legs may import this package.  It wraps ``relaybp_oracle.c`` (Relay-BP, the
fault sampler, the learned loss) and ``awgn_oracle.c`` (BPSK-AWGN sum-product
BP, OSD post-processing), plain C in FP64, through ctypes, and adds
``windows.py`` (sliding-window decoding over the Relay-BP oracle); each file
cites the passages of arXiv 2607.27644 it follows.  ``min_weight`` enumerates
codewords for the distance pins of the code builder.

Pins (tests/test_oracle.py, tests/test_awgn_oracle.py, tests/test_windows.py,
tests/test_workloads.py) tie it to things other than itself: published
Philox known-answer vectors, brute-force min-marginals and exact bitwise MAP
on cycle-free graphs, a closed-form memory recurrence, brute-force
minimum-weight decoding of the [[60,12,6]] and ZSZ-2BGA-64 codes, centre
automorphism equivariance, a stabilizer-tableau simulation of the circuits,
and invariants (H e^ = s on every claimed success); the minimum-weight
select against per-shot solution records (``solutions``) and brute-force
solution sets, and the leg carry-over against a hand-derived recurrence.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "relaybp_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "awgn_oracle.c")]
_LIB = os.path.join(_HERE, "librelaybp_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over shots)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp,
                               *_SRCS, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OracleParams(ctypes.Structure):
    _fields_ = [("gamma0", ctypes.c_double), ("pre_iter", ctypes.c_int32), ("num_sets", ctypes.c_int32),
                ("max_iterations", ctypes.c_int32), ("stop_nconv", ctypes.c_int32),
                ("gamma_min", ctypes.c_double), ("gamma_max", ctypes.c_double),
                ("stop_all", ctypes.c_int32), ("carry_messages", ctypes.c_int32), ("seed", ctypes.c_uint64)]


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.oracle_philox4x32_10.argtypes = [P, P, P]
        _lib.oracle_philox4x32_10.restype = None
        _lib.oracle_sample.argtypes = [ctypes.c_int32] * 3 + [P] * 5 + [ctypes.c_uint64, ctypes.c_uint64,
                                                                         ctypes.c_int64, P, P, P]
        _lib.oracle_sample.restype = ctypes.c_int
        _lib.oracle_relaybp_decode.argtypes = ([ctypes.c_int32] * 3 + [P] * 5 + [ctypes.POINTER(OracleParams), P,
                                               ctypes.c_uint64, ctypes.c_int64, P, P, P, P, ctypes.c_int32, P,
                                               ctypes.c_int32])
        _lib.oracle_relaybp_decode.restype = ctypes.c_int
        _lib.oracle_max_threads.restype = ctypes.c_int
        _lib.oracle_min_weight.argtypes = [ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32]
        _lib.oracle_min_weight.restype = ctypes.c_int
        _lib.oracle_awgn_llr.argtypes = [ctypes.c_int32, P, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_int64, P]
        _lib.oracle_awgn_llr.restype = ctypes.c_int
        _lib.oracle_sum_product.argtypes = ([ctypes.c_int32, ctypes.c_int32, P, P, P, ctypes.c_int64, ctypes.c_int32,
                                             ctypes.c_double, ctypes.c_int32, P, P, P, P, ctypes.c_int32])
        _lib.oracle_sum_product.restype = ctypes.c_int
        _lib.oracle_osd.argtypes = [ctypes.c_int32, ctypes.c_int32, P, P, P, P, P, ctypes.c_int32, ctypes.c_int64, P, P,
                                    ctypes.c_int32]
        _lib.oracle_osd.restype = ctypes.c_int
        _lib.oracle_relaybp_decode_post.argtypes = ([ctypes.c_int32] * 3 + [P] * 5 + [ctypes.POINTER(OracleParams), P,
                                                     ctypes.c_uint64, ctypes.c_int64, P, P, P, P, P, ctypes.c_int32])
        _lib.oracle_relaybp_decode_post.restype = ctypes.c_int
        _lib.oracle_learned_loss.argtypes = ([ctypes.c_int32] * 2 + [P] * 3 + [ctypes.c_int32, P, ctypes.c_int32, P,
                                             ctypes.c_uint64, P, P, ctypes.c_uint64, ctypes.c_int64,
                                             ctypes.c_int32, P, P, ctypes.c_int32])
        _lib.oracle_learned_loss.restype = ctypes.c_int
        _lib.oracle_relaybp_decode_learned.argtypes = ([ctypes.c_int32] * 3 + [P] * 5 +
                                                       [ctypes.POINTER(OracleParams), ctypes.c_int32, P,
                                                        ctypes.c_int32, P, ctypes.c_int32, P, ctypes.c_uint64,
                                                        ctypes.c_int64,
                                                        P, P, P, P, ctypes.c_int32, P, ctypes.c_int32])
        _lib.oracle_relaybp_decode_learned.restype = ctypes.c_int
        _lib.oracle_relaybp_solutions.argtypes = ([ctypes.c_int32] * 2 + [P] * 3 + [ctypes.POINTER(OracleParams), P,
                                                  ctypes.c_uint64, P, P, P, ctypes.c_int32, P, P, P, P, P])
        _lib.oracle_relaybp_solutions.restype = ctypes.c_int
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def min_weight(G: np.ndarray, n_threads: int = 0) -> int:
    """Minimum nonzero codeword weight of the row space of a binary k x n
    matrix G (k <= 63, n <= 64) by Gray-code enumeration of all codewords
    (test infrastructure for the Table 2 distance pin)."""
    G = np.asarray(G, dtype=np.uint8)
    k, n = G.shape
    rows = np.zeros(k, dtype=np.uint64)
    for c in range(n):
        rows |= G[:, c].astype(np.uint64) << np.uint64(c)
    d = _load().oracle_min_weight(k, n, rows.ctypes.data_as(ctypes.c_void_p), n_threads)
    if d < 0:
        raise ValueError("min_weight needs 1 <= k <= 63 and 1 <= n <= 64")
    return d


def awgn_sigma(ebn0_db: float, rate: float) -> float:
    """Noise deviation of BPSK over AWGN at E_b/N_0 (dB) for code rate R:
    E_b/N_0 = 1 / (2 R sigma^2) for unit-energy symbols (Sec. 6.2)."""
    return float(np.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))))


def awgn_llr(n: int, sigma: float, seed: int, shot0: int, shots: int, codewords=None,
             llr_max: float = 20.0) -> np.ndarray:
    """Channel LLRs [shots, n] of BPSK transmissions over AWGN (all-zero
    codeword unless packed `codewords` [shots, ceil(n/32)] are given)."""
    out = np.zeros((shots, n), dtype=np.float64)
    cw = None if codewords is None else np.ascontiguousarray(codewords, dtype=np.uint32)
    rc = _load().oracle_awgn_llr(n, None if cw is None else cw.ctypes.data_as(ctypes.c_void_p), sigma, llr_max,
                                 seed, shot0, shots, out.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise ValueError("oracle_awgn_llr rejected its arguments")
    return out


def sum_product(indptr, indices, m: int, n: int, llr: np.ndarray, max_iter: int = 100, llr_max: float = 20.0,
                early_stop: bool = True, posteriors: bool = False, n_threads: int = 0) -> dict:
    """Flooding sum-product BP (boxplus-phi check update) of LLR vectors
    llr [shots, n] for the m x n check matrix in CSR form (Sec. 6.2)."""
    llr = np.ascontiguousarray(llr, dtype=np.float64)
    shots = llr.shape[0]
    ip = np.ascontiguousarray(indptr, dtype=np.int32)
    ix = np.ascontiguousarray(indices, dtype=np.int32)
    bits = np.zeros((shots, (n + 31) // 32), dtype=np.uint32)
    iters = np.zeros(shots, dtype=np.int32)
    valid = np.zeros(shots, dtype=np.int32)
    post = np.zeros((shots, n), dtype=np.float64) if posteriors else None
    vp = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    rc = _load().oracle_sum_product(m, n, vp(ip), vp(ix), vp(llr), shots, max_iter, llr_max, int(early_stop), vp(bits),
                                    vp(iters), vp(valid), vp(post), n_threads)
    if rc != 0:
        raise ValueError("oracle_sum_product rejected its arguments")
    return dict(bits=bits, iters=iters, valid=valid.astype(bool), posteriors=post)


def osd(indptr, indices, m: int, n: int, syndromes: np.ndarray, soft: np.ndarray, order: int = 0,
        weights: np.ndarray | None = None, n_threads: int = 0) -> dict:
    """Ordered-statistics decoding: the solution of H e = s on the first rank(H)
    independent columns in ascending order of `soft` (posterior LLRs: the most
    likely errors first), OSD-0; with order > 0 also every flip of one or two
    of the first `order` columns outside that set, keeping the least sum of
    `weights` (prior LLRs).  syndromes [shots, ceil(m/32)] packed."""
    soft = np.ascontiguousarray(soft, dtype=np.float64)
    shots = soft.shape[0]
    syn = np.ascontiguousarray(syndromes, dtype=np.uint32)
    ip = np.ascontiguousarray(indptr, dtype=np.int32)
    ix = np.ascontiguousarray(indices, dtype=np.int32)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    e = np.zeros((shots, (n + 31) // 32), dtype=np.uint32)
    valid = np.zeros(shots, dtype=np.int32)
    vp = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)
    rc = _load().oracle_osd(m, n, vp(ip), vp(ix), vp(syn), vp(soft), vp(w), order, shots, vp(e), vp(valid),
                            n_threads)
    if rc != 0:
        raise ValueError("oracle_osd rejected its arguments")
    return dict(corrections=e, valid=valid.astype(bool))


def osd0(indptr, indices, m: int, n: int, syndromes: np.ndarray, soft: np.ndarray, n_threads: int = 0) -> dict:
    """OSD-0 (order 0 of `osd`)."""
    return osd(indptr, indices, m, n, syndromes, soft, 0, None, n_threads)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _dem_arrays(dem):
    return (np.ascontiguousarray(dem.H_indptr, dtype=np.int32), np.ascontiguousarray(dem.H_indices, dtype=np.int32),
            np.ascontiguousarray(dem.O_indptr, dtype=np.int32), np.ascontiguousarray(dem.O_indices, dtype=np.int32),
            np.ascontiguousarray(dem.priors, dtype=np.float64))


def sample(dem, seed: int, shot0: int, shots: int, want_errors: bool = False):
    """(syndromes [shots, ceil(C/32)] u32, obs [shots, ceil(k/32)] u32, errors or None)."""
    lib = _load()
    Hp, Hi, Op, Oi, pr = _dem_arrays(dem)
    syn = np.zeros((shots, (dem.n_det + 31) // 32), dtype=np.uint32)
    obs = np.zeros((shots, max(1, (dem.n_obs + 31) // 32)), dtype=np.uint32)
    err = np.zeros((shots, (dem.n_loc + 31) // 32), dtype=np.uint32) if want_errors else None
    rc = lib.oracle_sample(dem.n_det, dem.n_loc, dem.n_obs, _ptr(Hp), _ptr(Hi), _ptr(Op), _ptr(Oi), _ptr(pr),
                           seed, shot0, shots, _ptr(syn), _ptr(obs), _ptr(err))
    if rc != 0:
        raise ValueError("oracle_sample rejected its input")
    return syn, obs, err


@dataclass
class DecodeParams:
    """Relay-BP parameters (Sec. 6.1 decoder configuration list)."""
    gamma0: float = 0.125
    pre_iter: int = 80
    num_sets: int = 1000
    max_iterations: int = 60
    stop_nconv: int = 5
    gamma_min: float = -0.24
    gamma_max: float = 0.66
    stop_all: bool = False
    carry_messages: bool = False
    seed: int = 0

    def c(self) -> OracleParams:
        return OracleParams(self.gamma0, self.pre_iter, self.num_sets, self.max_iterations, self.stop_nconv,
                            self.gamma_min, self.gamma_max, int(self.stop_all), int(self.carry_messages),
                            self.seed)


def decode(dem, params: DecodeParams, syndromes: np.ndarray, shot0: int = 0, trace_iters: int = 0,
           n_threads: int = 0, w: np.ndarray | None = None, knots: np.ndarray | None = None,
           learned_legs: int = -1):
    """Relay-BP on every syndrome row.

    Returns dict(corrections, pred_obs, stats[shots,4], weights, trace or None).
    stats columns: converged, #solutions, legs run, total iterations.
    """
    lib = _load()
    Hp, Hi, Op, Oi, pr = _dem_arrays(dem)
    syn = np.ascontiguousarray(syndromes, dtype=np.uint32)
    shots = syn.shape[0]
    corr = np.zeros((shots, (dem.n_loc + 31) // 32), dtype=np.uint32)
    pobs = np.zeros((shots, max(1, (dem.n_obs + 31) // 32)), dtype=np.uint32)
    stats = np.zeros((shots, 4), dtype=np.int32)
    wts = np.zeros(shots, dtype=np.float64)
    trace = np.zeros((shots, trace_iters, dem.n_loc), dtype=np.float64) if trace_iters > 0 else None
    cp = params.c()
    if w is None and knots is None:
        rc = lib.oracle_relaybp_decode(dem.n_det, dem.n_loc, dem.n_obs, _ptr(Hp), _ptr(Hi), _ptr(Op), _ptr(Oi),
                                       _ptr(pr), ctypes.byref(cp), _ptr(syn), shot0, shots, _ptr(corr), _ptr(pobs),
                                       _ptr(stats), _ptr(wts), trace_iters, _ptr(trace), n_threads)
    else:
        lw = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        lk = None if knots is None else np.ascontiguousarray(knots, dtype=np.float64)
        rc = lib.oracle_relaybp_decode_learned(dem.n_det, dem.n_loc, dem.n_obs, _ptr(Hp), _ptr(Hi), _ptr(Op),
                                               _ptr(Oi), _ptr(pr), ctypes.byref(cp), 0 if lw is None else lw.shape[0],
                                               _ptr(lw), 0 if lk is None else lk.shape[0] - 1, _ptr(lk),
                                               learned_legs, _ptr(syn),
                                               shot0, shots, _ptr(corr), _ptr(pobs), _ptr(stats), _ptr(wts),
                                               trace_iters, _ptr(trace), n_threads)
    if rc != 0:
        raise ValueError("oracle_relaybp_decode rejected its input")
    return dict(corrections=corr, pred_obs=pobs, stats=stats, weights=wts, trace=trace)


def solutions(dem, params: DecodeParams, syndrome: np.ndarray, shot: int = 0, cap: int = 64) -> dict:
    """Decode one syndrome [ceil(C/32)] and record every solution found, in
    order: dict(correction, stats[4], weight, found, legs[n], iters[n],
    weights[n], bits[n, ceil(V/32)]) with n = min(found, cap); iters[r] is the
    shot's iteration count when solution r was found."""
    lib = _load()
    Hp, Hi, _, _, pr = _dem_arrays(dem)
    syn = np.ascontiguousarray(np.asarray(syndrome, dtype=np.uint32).reshape(-1))
    wv = (dem.n_loc + 31) // 32
    corr = np.zeros(wv, dtype=np.uint32)
    stats = np.zeros(4, dtype=np.int32)
    wt = np.zeros(1, dtype=np.float64)
    legs = np.zeros(max(1, cap), dtype=np.int32)
    iters = np.zeros(max(1, cap), dtype=np.int32)
    wts = np.zeros(max(1, cap), dtype=np.float64)
    bits = np.zeros((max(1, cap), wv), dtype=np.uint32)
    found = np.zeros(1, dtype=np.int32)
    cp = params.c()
    rc = lib.oracle_relaybp_solutions(dem.n_det, dem.n_loc, _ptr(Hp), _ptr(Hi), _ptr(pr), ctypes.byref(cp), _ptr(syn),
                                      shot, _ptr(corr), _ptr(stats), _ptr(wt), cap, _ptr(legs), _ptr(iters),
                                      _ptr(wts), _ptr(bits), _ptr(found))
    if rc != 0:
        raise ValueError("oracle_relaybp_solutions rejected its input")
    n = min(int(found[0]), cap)
    return dict(correction=corr, stats=stats, weight=float(wt[0]), found=int(found[0]), legs=legs[:n],
                iters=iters[:n], weights=wts[:n], bits=bits[:n])


def decode_with_posteriors(dem, params: DecodeParams, syndromes: np.ndarray, shot0: int = 0,
                           n_threads: int = 0) -> dict:
    """decode() plus each shot's marginals M after its last iteration
    (key "posteriors", [shots, n_loc]): the soft input of OSD post-processing."""
    lib = _load()
    Hp, Hi, Op, Oi, pr = _dem_arrays(dem)
    syn = np.ascontiguousarray(syndromes, dtype=np.uint32)
    shots = syn.shape[0]
    corr = np.zeros((shots, (dem.n_loc + 31) // 32), dtype=np.uint32)
    pobs = np.zeros((shots, max(1, (dem.n_obs + 31) // 32)), dtype=np.uint32)
    stats = np.zeros((shots, 4), dtype=np.int32)
    wts = np.zeros(shots, dtype=np.float64)
    post = np.zeros((shots, dem.n_loc), dtype=np.float64)
    cp = params.c()
    rc = lib.oracle_relaybp_decode_post(dem.n_det, dem.n_loc, dem.n_obs, _ptr(Hp), _ptr(Hi), _ptr(Op), _ptr(Oi),
                                        _ptr(pr), ctypes.byref(cp), _ptr(syn), shot0, shots, _ptr(corr), _ptr(pobs),
                                        _ptr(stats), _ptr(wts), _ptr(post), n_threads)
    if rc != 0:
        raise ValueError("oracle_relaybp_decode_post rejected its input")
    return dict(corrections=corr, pred_obs=pobs, stats=stats, weights=wts, posteriors=post)


def unpack_bits(words: np.ndarray, nbits: int) -> np.ndarray:
    """[..., W] u32 -> [..., nbits] uint8 (bit b in word b/32, position b%32)."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    b = np.unpackbits(w.view(np.uint8), axis=-1, bitorder="little")
    return b[..., :nbits]


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """[..., nbits] {0,1} -> [..., ceil(nbits/32)] u32."""
    bits = np.asarray(bits, dtype=np.uint8)
    nb = bits.shape[-1]
    pad = (-nb) % 32
    if pad:
        bits = np.concatenate([bits, np.zeros(bits.shape[:-1] + (pad,), dtype=np.uint8)], axis=-1)
    by = np.packbits(bits, axis=-1, bitorder="little")
    return np.ascontiguousarray(by).view(np.uint32)


def learned_loss(dem, w: np.ndarray, knots: np.ndarray, gamma_seed: int, syndromes: np.ndarray,
                 errors: np.ndarray, shot0: int = 0, trace: bool = False, n_threads: int = 0,
                 objective: int = 0):
    """Per-shot loss of the learned forward (T = w.shape[0] unrolled iterations).

    w: [T, E] message weights in row-major edge order; knots: [K+1] inverse CDF
    of the memory strengths; objective 0: cross-entropy of M against the
    sampled error, 1: soft syndrome (-log probability that each check holds
    its syndrome bit).  Returns (loss [shots], trace [shots, T, V] or None).
    """
    lib = _load()
    Hp, Hi, _, _, pr = _dem_arrays(dem)
    w = np.ascontiguousarray(w, dtype=np.float64)
    knots = np.ascontiguousarray(knots, dtype=np.float64)
    syn = np.ascontiguousarray(syndromes, dtype=np.uint32)
    err = np.ascontiguousarray(errors, dtype=np.uint32)
    shots = syn.shape[0]
    T, K = w.shape[0], knots.shape[0] - 1
    loss = np.zeros(shots, dtype=np.float64)
    tr = np.zeros((shots, T, dem.n_loc), dtype=np.float64) if trace else None
    rc = lib.oracle_learned_loss(dem.n_det, dem.n_loc, _ptr(Hp), _ptr(Hi), _ptr(pr), T, _ptr(w), K, _ptr(knots),
                                 gamma_seed, _ptr(syn), _ptr(err), shot0, shots, objective, _ptr(loss), _ptr(tr),
                                 n_threads)
    if rc != 0:
        raise ValueError("oracle_learned_loss rejected its input")
    return loss, tr
