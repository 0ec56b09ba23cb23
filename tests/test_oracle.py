"""Pins of the CPU oracle to things other than itself.

  * Philox4x32-10: published known-answer vectors (Random123 / SC'11).
  * Sampler: the fired faults are exactly the Philox words below floor(p 2^32);
    syndromes equal H e mod 2 by an independent dense product; frequencies.
  * Check + variable updates: on cycle-free Tanner graphs min-sum reaches the
    exact min-marginals, which brute force gives independently.
  * Memory term: a one-check, two-variable graph has a closed-form recurrence.
  * Minimum-weight decoding of single errors on the [[60,12,6]] code (Table 13).
  * Invariants on circuit-level DEMs: H e^ = s on every claimed success, the
    reported weight, solution counts and leg limits.
  * Minimum-weight select: every recorded solution against the brute-force
    solution set of tiny graphs, weights recomputed from the bits, the first
    record of least weight returned (ties to the earliest).
  * Leg carry-over (messages reset or carried, M carried): a hand-derived
    two-check, two-variable recurrence across leg boundaries.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from oracle import DecodeParams, unpack_bits, pack_bits
from workloads.dem import circuit_dem, code_capacity_dem, dem_from_dense

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_kat():
    n = 0
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert list(out) == v[6:10]
        n += 1
    assert n == 3


def test_sampler_definition_and_syndrome():
    D = circuit_dem("ZSZ-LP-60", 0.01, 2, "Z")
    seed, shot0, shots = 0x1234_5678_9ABC, 1000, 40
    syn, obs, err = oracle.sample(D, seed, shot0, shots, want_errors=True)
    e = unpack_bits(err, D.n_loc)
    thr = np.floor(D.priors * 2.0 ** 32)
    for s in range(0, shots, 7):
        shot = shot0 + s
        want = np.zeros(D.n_loc, dtype=np.uint8)
        for blk in range((D.n_loc + 3) // 4):
            w = oracle.philox4x32_10([blk, shot & 0xFFFFFFFF, shot >> 32, 0], [seed & 0xFFFFFFFF, seed >> 32])
            for t in range(4):
                j = 4 * blk + t
                if j < D.n_loc:
                    want[j] = w[t] < thr[j]
        assert np.array_equal(e[s], want)
    Hd, Od = D.dense_H().astype(np.int64), D.dense_O().astype(np.int64)
    assert np.array_equal(unpack_bits(syn, D.n_det), (e.astype(np.int64) @ Hd.T) % 2)
    assert np.array_equal(unpack_bits(obs, D.n_obs), (e.astype(np.int64) @ Od.T) % 2)


def test_sampler_frequencies():
    pr = np.array([0.5, 0.25, 0.01, 0.001, 0.3, 0.07, 0.0, 1.0])
    H = np.eye(len(pr), dtype=np.uint8)
    D = dem_from_dense(H, pr)
    n = 200_000
    _, _, err = oracle.sample(D, 99, 0, n, want_errors=True)
    f = unpack_bits(err, len(pr)).mean(0)
    sig = np.sqrt(pr * (1 - pr) / n)
    assert np.all(np.abs(f - pr) <= 5 * sig + 1e-12)


# ---------------------------------------------------------------------------
# min-sum on trees equals brute-force min-marginals
# ---------------------------------------------------------------------------
def _random_tree_graph(rng, n_checks):
    """Bipartite tree: every check has degree >= 2; returns dense H."""
    checks = [[0, 1]]
    nv = 2
    for c in range(1, n_checks):
        old = rng.integers(0, nv)                     # attach to an existing variable
        k = int(rng.integers(1, 3))                   # plus 1-2 fresh variables
        checks.append([old] + list(range(nv, nv + k)))
        nv += k
    H = np.zeros((n_checks, nv), dtype=np.uint8)
    for i, vs in enumerate(checks):
        H[i, vs] = 1
    return H


def _brute_min_marginals(H, L0, s):
    V = H.shape[1]
    best = {0: math.inf, 1: math.inf}
    best_j = np.full((V, 2), math.inf)
    Hi = H.astype(np.int64)
    for bits in itertools.product((0, 1), repeat=V):
        e = np.array(bits)
        if np.any((Hi @ e) % 2 != s):
            continue
        w = float(e @ L0)
        for j in range(V):
            best_j[j, bits[j]] = min(best_j[j, bits[j]], w)
    return best_j[:, 1] - best_j[:, 0]


@pytest.mark.parametrize("seed", range(6))
def test_minsum_tree_min_marginals(seed):
    rng = np.random.default_rng(seed)
    H = _random_tree_graph(rng, int(rng.integers(3, 7)))
    V = H.shape[1]
    assert V <= 14
    pr = rng.uniform(0.02, 0.45, V)
    L0 = np.log((1 - pr) / pr)
    e = (rng.random(V) < 0.3).astype(np.int64)
    s = (H.astype(np.int64) @ e) % 2
    # an extra check with no edges and syndrome 1 keeps the leg from stopping
    Hx = np.vstack([H, np.zeros((1, V), dtype=np.uint8)])
    sx = np.r_[s, 1]
    D = dem_from_dense(Hx, pr)
    T = 2 * Hx.shape[0] + 4
    P = DecodeParams(gamma0=0.0, pre_iter=T, num_sets=0, max_iterations=0, stop_nconv=1)
    r = oracle.decode(D, P, pack_bits(sx[None, :]), trace_iters=T)
    M = r["trace"][0, T - 1]
    want = _brute_min_marginals(H, L0, s)
    assert np.allclose(M, want, rtol=1e-12, atol=1e-12)
    assert r["stats"][0, 0] == 0 and r["stats"][0, 3] == T


def test_memory_recurrence_closed_form():
    """One check on two variables, syndrome 1, memory strength g.

    nu_{->1} = -L_2(t) and nu_{->2} = -L_1(t), so M_1(t) = L_1(t) - L_2(t) =
    -M_2(t).  With M(0) = L0 the first iteration has L(1) = L0 and
    M_1(1) = a - b; from then on L_k(t) = (1-g) L0_k + g M_k(t-1) gives
        M_1(t) = (1-g)(a-b) + 2g M_1(t-1),  t >= 2,
    i.e. M_1(t) = (a-b) [(1-g) sum_{u<t-1} (2g)^u + (2g)^(t-1)].
    Legs after the first use g = gamma_min = gamma_max and carry M, so the same
    recurrence continues across the leg boundary.
    """
    pa, pb = 0.1, 0.3
    a, b = math.log((1 - pa) / pa), math.log((1 - pb) / pb)
    H = np.array([[1, 1], [0, 0]], dtype=np.uint8)
    D = dem_from_dense(H, [pa, pb])
    for g in (0.0, 0.125, 0.3, -0.2):
        T0, T1 = 5, 4
        P = DecodeParams(gamma0=g, pre_iter=T0, num_sets=1, max_iterations=T1, stop_nconv=5,
                         gamma_min=g, gamma_max=g, seed=3)
        r = oracle.decode(D, P, pack_bits(np.array([[1, 1]])), trace_iters=T0 + T1)
        closed = [(a - b) * ((1 - g) * sum((2 * g) ** u for u in range(t - 1)) + (2 * g) ** (t - 1))
                  for t in range(1, T0 + T1 + 1)]
        tr = r["trace"][0]
        assert np.allclose(tr[:, 0], closed, rtol=1e-12, atol=1e-12)
        assert np.allclose(tr[:, 1], -np.array(closed), rtol=1e-12, atol=1e-12)
        assert r["stats"][0, 2] == 2 and r["stats"][0, 3] == T0 + T1


def test_gamma_draw_range_and_stream():
    """Legs >= 1 draw g_j from stream 1 of the decoder seed: with a single
    variable the first iteration of leg 1 gives M = (1-g) a + g M_prev exactly."""
    p = 0.2
    a = math.log((1 - p) / p)
    H = np.zeros((1, 1), dtype=np.uint8)              # one check with no edges, syndrome 1
    D = dem_from_dense(H, [p])
    P = DecodeParams(gamma0=0.5, pre_iter=1, num_sets=3, max_iterations=1, stop_nconv=9,
                     gamma_min=-0.24, gamma_max=0.66, seed=0xABCDEF)
    shot = 17
    r = oracle.decode(D, P, pack_bits(np.array([[1]])), shot0=shot, trace_iters=4)
    M = r["trace"][0, :, 0]
    assert np.isclose(M[0], a)                            # M(0) = a, so L(1) = a
    for leg in (1, 2, 3):
        w = oracle.philox4x32_10([leg * 1, shot, 0, 1], [0xABCDEF, 0])[0]
        g = -0.24 + 0.9 * ((int(w) >> 8) / 2.0 ** 24)
        assert -0.24 <= g <= 0.66
        assert np.isclose(M[leg], (1 - g) * a + g * M[leg - 1], rtol=1e-13)


def test_mw_single_errors_60():
    """[[60,12,6]] code capacity: no nonzero vector of ker H_X has weight <= 2,
    so each single Z error is the unique minimum-weight solution of its
    syndrome; Relay-BP must return it exactly."""
    D = code_capacity_dem("ZSZ-LP-60", 0.01)
    Hd = D.dense_H().astype(np.int64)
    V = D.n_loc
    for j1, j2 in itertools.combinations(range(V), 2):
        assert np.any(Hd[:, j1] ^ Hd[:, j2])
    assert np.all(Hd.sum(0) > 0)
    E = np.eye(V, dtype=np.uint8)
    syn = pack_bits((E.astype(np.int64) @ Hd.T) % 2)
    r = oracle.decode(D, DecodeParams(num_sets=20, seed=5), syn)
    assert np.all(r["stats"][:, 0] == 1)
    assert np.array_equal(unpack_bits(r["corrections"], V), E)


def test_mw_double_errors_60_weight_bound():
    """Weight-2 errors: every converged answer satisfies H e^ = s and has
    weight >= the brute-force minimum weight of its syndrome (<= 2)."""
    D = code_capacity_dem("ZSZ-LP-60", 0.01)
    Hd = D.dense_H().astype(np.int64)
    V = D.n_loc
    pairs = list(itertools.combinations(range(V), 2))[::11]
    E = np.zeros((len(pairs), V), dtype=np.uint8)
    for t, (a, b) in enumerate(pairs):
        E[t, [a, b]] = 1
    S = (E.astype(np.int64) @ Hd.T) % 2
    single = {tuple(Hd[:, j]) for j in range(V)}
    r = oracle.decode(D, DecodeParams(num_sets=20, seed=5), pack_bits(S))
    eh = unpack_bits(r["corrections"], V).astype(np.int64)
    conv = r["stats"][:, 0] == 1
    assert conv.mean() > 0.95
    assert np.array_equal((eh[conv] @ Hd.T) % 2, S[conv])
    for t in np.nonzero(conv)[0]:
        mw = 0 if not S[t].any() else (1 if tuple(S[t]) in single else 2)
        assert eh[t].sum() >= mw


def test_invariants_circuit_level():
    D = circuit_dem("ZSZ-LP-60", 0.004, 3, "Z")
    syn, obs, _ = oracle.sample(D, 11, 0, 300)
    P = DecodeParams(num_sets=30, stop_nconv=3, gamma_min=-0.15, gamma_max=0.61, seed=1)
    r = oracle.decode(D, P, syn)
    st = r["stats"]
    eh = unpack_bits(r["corrections"], D.n_loc).astype(np.int64)
    S = unpack_bits(syn, D.n_det).astype(np.int64)
    Hd = D.dense_H().astype(np.int64)
    conv = st[:, 0] == 1
    assert conv.mean() > 0.9
    assert np.array_equal((eh[conv] @ Hd.T) % 2, S[conv])
    L0 = np.log((1 - D.priors) / D.priors)
    assert np.allclose(r["weights"], eh @ L0, rtol=1e-12)
    assert np.all(st[:, 1] <= 3) and np.all(st[:, 2] <= 31)
    assert np.all(st[conv, 1] >= 1) and np.all(st[~conv, 1] == 0)
    assert np.all(st[:, 3] <= 80 + 30 * 60)
    # stop after stop_nconv solutions: a shot stops early only once it has them
    assert np.all((st[:, 2] == 31) | (st[:, 1] == 3))
    Od = D.dense_O().astype(np.int64)
    assert np.array_equal(unpack_bits(r["pred_obs"], D.n_obs), (eh @ Od.T) % 2)


def test_stop_all_runs_every_leg():
    D = circuit_dem("ZSZ-LP-60", 0.004, 2, "Z")
    syn, _, _ = oracle.sample(D, 12, 0, 20)
    P = DecodeParams(num_sets=4, stop_nconv=1, stop_all=True, seed=2)
    r = oracle.decode(D, P, syn)
    assert np.all(r["stats"][:, 2] == 5)


def test_deterministic_and_shard_invariant():
    """Counter-based draws: decoding shots [0,40) at once equals two shards."""
    D = circuit_dem("ZSZ-LP-60", 0.004, 2, "Z")
    syn, _, _ = oracle.sample(D, 13, 0, 40)
    P = DecodeParams(num_sets=10, seed=4)
    full = oracle.decode(D, P, syn, shot0=0)
    a = oracle.decode(D, P, syn[:25], shot0=0)
    b = oracle.decode(D, P, syn[25:], shot0=25)
    assert np.array_equal(full["corrections"], np.vstack([a["corrections"], b["corrections"]]))
    assert np.array_equal(full["stats"], np.vstack([a["stats"], b["stats"]]))


def test_iteration_map_amplifies_rounding():
    """Property of the method that sets the parity windows of the GPU tests:
    on a circuit-level DEM, perturbing every prior by one part in 2^50 grows
    to a relative posterior difference above 1e-9 within 40 iterations while
    staying below 1e-12 for the first 3 -- two correct evaluations whose
    rounding differs agree only in an early window."""
    D = circuit_dem("ZSZ-LP-160", 0.001, 10, "Z")
    P = DecodeParams(gamma0=0.125, pre_iter=80, num_sets=0, max_iterations=60, stop_nconv=1,
                     gamma_min=-0.15, gamma_max=0.61, seed=1)
    syn, _, _ = oracle.sample(D, 7, 1000, 8)
    T = 40
    a = oracle.decode(D, P, syn, shot0=1000, trace_iters=T)
    b = oracle.decode(D.with_priors(D.priors * (1 + 2.0 ** -50)), P, syn, shot0=1000, trace_iters=T)
    grew = 0
    for s in range(8):
        n = int(min(a["stats"][s, 3], b["stats"][s, 3], T))
        if n < 30:
            continue
        d = np.abs(a["trace"][s, :n] - b["trace"][s, :n]) / np.maximum(1, np.abs(a["trace"][s, :n]))
        assert d[:3].max() < 1e-12
        grew += int(d.max() > 1e-9)
    assert grew >= 1


# ---------------------------------------------------------------------------
# learned form (a10): pinned to the plain method and to a closed form
# ---------------------------------------------------------------------------
def test_learned_forward_reduces_to_plain_memory_bp():
    """w = 1 and constant knots g reproduce the plain oracle's leg 0 run at
    gamma0 = g bit for bit (an empty check with syndrome 1 keeps it going)."""
    D = circuit_dem("ZSZ-LP-60", 0.004, 3, "Z")
    Hd = D.dense_H()
    Hx = np.vstack([Hd, np.zeros((1, D.n_loc), dtype=np.uint8)])
    Dx = dem_from_dense(Hx, D.priors)
    syn, _, err = oracle.sample(D, 21, 0, 6, want_errors=True)
    S = np.hstack([unpack_bits(syn, D.n_det), np.ones((6, 1), dtype=np.uint8)])
    synx = pack_bits(S)
    T, g = 7, 0.3
    w = np.ones((T, Dx.n_edges))
    knots = np.full(17, g)
    loss, tr = oracle.learned_loss(Dx, w, knots, 5, synx, err, trace=True)
    P = DecodeParams(gamma0=g, pre_iter=T, num_sets=0, max_iterations=1, stop_nconv=1)
    r = oracle.decode(Dx, P, synx, trace_iters=T)
    assert np.array_equal(tr, r["trace"])
    E = unpack_bits(err, D.n_loc).astype(float)
    sp = lambda x: np.logaddexp(0.0, x)
    want = (E[:, None, :] * sp(tr) + (1 - E[:, None, :]) * sp(-tr)).sum(axis=(1, 2))
    assert np.allclose(loss, want, rtol=1e-12)


def test_learned_forward_closed_form_two_variables():
    """One check on two variables, syndrome 1, edge weights w1(t), w2(t) and
    memory strengths g1, g2 from the knot table:
        nu_1(t) = -w1(t) L_2(t),  nu_2(t) = -w2(t) L_1(t),
        L_k(t) = (1 - g_k) L0_k + g_k M_k(t-1),  M_k(0) = L0_k,
        M_1(t) = L_1(t) - w1(t) L_2(t),  M_2(t) = L_2(t) - w2(t) L_1(t)."""
    pa, pb = 0.1, 0.3
    a, b = math.log((1 - pa) / pa), math.log((1 - pb) / pb)
    H = np.array([[1, 1], [0, 0]], dtype=np.uint8)
    D = dem_from_dense(H, [pa, pb])
    T = 6
    rng = np.random.default_rng(3)
    w = rng.uniform(0.5, 1.5, (T, 2))
    knots = np.cumsum(np.r_[-0.2, rng.uniform(0.0, 0.08, 16)])
    seed, shot = 77, 9
    u = []
    for j in range(2):
        word = oracle.philox4x32_10([1 * 1 + j // 4, shot, 0, 1], [seed, 0])[j % 4]
        u.append((int(word) >> 8) / 2.0 ** 24)
    g = []
    for uj in u:
        k = min(int(np.floor(uj * 16)), 15)
        g.append(knots[k] + (knots[k + 1] - knots[k]) * (uj * 16 - k))
    M = [a, b]
    want = []
    for t in range(T):
        L1 = (1 - g[0]) * a + g[0] * M[0]
        L2 = (1 - g[1]) * b + g[1] * M[1]
        M = [L1 - w[t, 0] * L2, L2 - w[t, 1] * L1]
        want.append(list(M))
    syn = pack_bits(np.array([[1, 1]]))
    err = pack_bits(np.array([[1, 0]]))
    loss, tr = oracle.learned_loss(D, w, knots, seed, syn, err, shot0=shot, trace=True)
    assert np.allclose(tr[0], np.array(want), rtol=1e-12, atol=1e-12)


def test_learned_decode_leg0_matches_training_forward():
    """Leg 0 of the learned decode (weights by iteration, gamma0 = g) equals the
    training forward with constant knots g, which is pinned above."""
    D = circuit_dem("ZSZ-LP-60", 0.004, 3, "Z")
    Hx = np.vstack([D.dense_H(), np.zeros((1, D.n_loc), dtype=np.uint8)])
    Dx = dem_from_dense(Hx, D.priors)
    syn, _, err = oracle.sample(D, 22, 0, 5, want_errors=True)
    synx = pack_bits(np.hstack([unpack_bits(syn, D.n_det), np.ones((5, 1), dtype=np.uint8)]))
    T, g = 6, 0.2
    w = np.random.default_rng(8).uniform(0.7, 1.3, (T, Dx.n_edges))
    _, tr = oracle.learned_loss(Dx, w, np.full(17, g), 5, synx, err, trace=True)
    P = DecodeParams(gamma0=g, pre_iter=T, num_sets=0, max_iterations=1, stop_nconv=1)
    r = oracle.decode(Dx, P, synx, trace_iters=T, w=w, knots=np.full(17, 0.4))
    assert np.array_equal(tr, r["trace"])


def test_learned_decode_unit_weights_is_plain():
    D = circuit_dem("ZSZ-LP-60", 0.004, 3, "Z")
    syn, _, _ = oracle.sample(D, 23, 0, 40)
    P = DecodeParams(num_sets=8, seed=3)
    a = oracle.decode(D, P, syn)
    b = oracle.decode(D, P, syn, w=np.ones((5, D.n_edges)))
    assert np.array_equal(a["corrections"], b["corrections"]) and np.array_equal(a["stats"], b["stats"])
    Hd = D.dense_H().astype(np.int64)
    c = oracle.decode(D, P, syn, w=np.random.default_rng(2).uniform(0.8, 1.0, (5, D.n_edges)),
                      knots=np.linspace(-0.1, 0.5, 17))
    eh = unpack_bits(c["corrections"], D.n_loc).astype(np.int64)
    conv = c["stats"][:, 0] == 1
    assert np.array_equal((eh[conv] @ Hd.T) % 2, unpack_bits(syn, D.n_det)[conv])


def test_learned_legs_cutoff():
    """learned_legs = 0 is the plain method exactly; a cutoff of 2 agrees with
    the fully learned decode on shots settled in legs 0 and 1."""
    D = circuit_dem("ZSZ-LP-60", 0.004, 3, "Z")
    syn, _, _ = oracle.sample(D, 31, 0, 60)
    P = DecodeParams(num_sets=10, stop_nconv=2, seed=4)
    rng = np.random.default_rng(12)
    w = rng.uniform(0.7, 1.0, (5, D.n_edges))
    kn = np.linspace(-0.1, 0.5, 17)
    plain = oracle.decode(D, P, syn)
    cut0 = oracle.decode(D, P, syn, w=w, knots=kn, learned_legs=0)
    assert np.array_equal(plain["corrections"], cut0["corrections"]) and np.array_equal(plain["stats"], cut0["stats"])
    full = oracle.decode(D, P, syn, w=w, knots=kn)
    cut2 = oracle.decode(D, P, syn, w=w, knots=kn, learned_legs=2)
    early = full["stats"][:, 2] <= 2
    assert early.any()
    assert np.array_equal(full["corrections"][early], cut2["corrections"][early])


def test_mw_brute_force_weight_le4_60():
    """[[60,12,6]] code capacity (H_X, equal priors), errors of weight 3 and 4:
    the minimum weight of every syndrome of a weight <= 4 error, by enumerating
    all 523,686 patterns of weight <= 4; every converged Relay-BP answer
    satisfies H e^ = s and has Hamming weight >= that minimum, and nearly all
    reach it (measured on 2,000 shots: 99.8% at weight 3, 99.5% at weight 4)."""
    D = code_capacity_dem("ZSZ-LP-60", 0.01)
    Hd = D.dense_H().astype(np.int64)
    C, V = Hd.shape
    assert C <= 24
    col = (Hd * (1 << np.arange(C))[:, None]).sum(0)           # column j as a C-bit integer
    mw = np.full(1 << C, 127, dtype=np.int8)
    mw[0] = 0
    for w in range(1, 5):
        idx = np.array(list(itertools.combinations(range(V), w)), dtype=np.int64)
        syn = np.bitwise_xor.reduce(col[idx], axis=1)
        fresh = mw[syn] > w
        mw[syn[fresh]] = w
    rng = np.random.default_rng(11)
    E = np.zeros((240, V), dtype=np.uint8)
    for t in range(E.shape[0]):
        E[t, rng.choice(V, 3 + t % 2, replace=False)] = 1
    S = (E.astype(np.int64) @ Hd.T) % 2
    r = oracle.decode(D, DecodeParams(num_sets=50, gamma_min=-0.24, gamma_max=0.66, seed=9), pack_bits(S))
    eh = unpack_bits(r["corrections"], V).astype(np.int64)
    conv = r["stats"][:, 0] == 1
    assert conv.mean() > 0.9
    assert np.array_equal((eh[conv] @ Hd.T) % 2, S[conv])
    sid = (S * (1 << np.arange(C))).sum(1)
    best = mw[sid].astype(np.int64)
    assert np.all(best <= E.sum(1))
    got = eh.sum(1)
    assert np.all(got[conv] >= best[conv])
    assert (got[conv] == best[conv]).mean() > 0.95


def test_mw_brute_force_classical_zsz_2bga_64():
    """ZSZ-2BGA-64 (H_left of ZSZ-LP-160, [64, 32, 10]) under i.i.d. bit flips:
    the minimum weight of every syndrome of a weight <= 5 error, by tabulating
    all 8,303,633 patterns of weight <= 5 (<= d/2, so each such error is a
    minimum-weight solution of its syndrome, the only one below d/2); every
    converged Relay-BP answer to weight-4 and weight-5 errors satisfies
    H e^ = s, weighs at least that minimum, and here always reaches it."""
    from workloads.dem import dem_from_dense
    from workloads.zsz import load_code
    H = load_code("ZSZ-LP-160").H_left.astype(np.int64)
    m, n = H.shape
    col = (H * (1 << np.arange(m, dtype=np.int64))[:, None]).sum(0)
    syn_all, wt_all = [np.zeros(1, dtype=np.int64)], [np.zeros(1, dtype=np.int8)]
    for w in range(1, 6):
        idx = np.fromiter(itertools.chain.from_iterable(itertools.combinations(range(n), w)), dtype=np.int8)
        idx = idx.reshape(-1, w).astype(np.int64)
        syn_all.append(np.bitwise_xor.reduce(col[idx], axis=1))
        wt_all.append(np.full(idx.shape[0], w, dtype=np.int8))
    syn_all, wt_all = np.concatenate(syn_all), np.concatenate(wt_all)
    order = np.lexsort((wt_all, syn_all))
    syn_s, wt_s = syn_all[order], wt_all[order]
    first = np.r_[True, syn_s[1:] != syn_s[:-1]]
    keys, mw = syn_s[first], wt_s[first]
    # below half the distance every syndrome has a single pattern of that weight
    assert np.unique(syn_all[wt_all <= 4]).size == int((wt_all <= 4).sum())
    D = dem_from_dense(H.astype(np.uint8), np.full(n, 0.03))
    rng = np.random.default_rng(21)
    E = np.zeros((200, n), dtype=np.uint8)
    for t in range(E.shape[0]):
        E[t, rng.choice(n, 4 + t % 2, replace=False)] = 1
    S = (E.astype(np.int64) @ H.T) % 2
    r = oracle.decode(D, DecodeParams(num_sets=50, gamma_min=-0.24, gamma_max=0.66, seed=3), pack_bits(S))
    eh = unpack_bits(r["corrections"], n).astype(np.int64)
    conv = r["stats"][:, 0] == 1
    assert conv.mean() > 0.9
    assert np.array_equal((eh[conv] @ H.T) % 2, S[conv])
    sid = (S * (1 << np.arange(m, dtype=np.int64))).sum(1)
    best = mw[np.searchsorted(keys, sid)].astype(np.int64)
    assert np.array_equal(keys[np.searchsorted(keys, sid)], sid)
    assert np.all(best == E.sum(1))                 # weight <= d/2: the error itself is a minimum
    got = eh.sum(1)
    assert np.all(got[conv] >= best[conv])
    assert (got[conv] == best[conv]).mean() > 0.95


def test_center_automorphism_symmetry():
    """ZSZ-LP-160 H_X with random (generic) priors: for every centre element z,
    permuting the syndrome by P_z^{+2} and the priors by P_z^{+5} permutes the
    decoder's state by P_z^{+5} (H P_z^{+5} = P_z^{+2} H, App. D).  Leg 0
    only, so every memory strength is gamma0 and needs no permuting.  Min-sum's
    check update is a symmetric function of the other inputs, so only the order
    of the variable sums changes: the posteriors agree to rounding over the
    first iterations, and the decisions agree exactly on every shot that
    settles quickly (later, the iteration map amplifies the roundings, as for
    any two evaluation orders)."""
    from workloads.dem import dem_from_dense
    from workloads.zsz import L_mat, load_code
    code = load_code("ZSZ-LP-160")
    H = code.H_X.astype(np.int64)
    m, n = H.shape
    rng = np.random.default_rng(31)
    p = rng.uniform(0.005, 0.03, n)
    E = (rng.random((80, n)) < p).astype(np.int64)
    S = (E @ H.T) % 2
    prm = DecodeParams(num_sets=0, pre_iter=80, seed=1)
    r = oracle.decode(dem_from_dense(H.astype(np.uint8), p), prm, pack_bits(S), trace_iters=4)
    eh = unpack_bits(r["corrections"], n).astype(np.int64)
    quick = (r["stats"][:, 0] == 1) & (r["stats"][:, 3] <= 10)
    assert quick.sum() >= 40
    centre = [z for z in code.G.center() if z != code.G.elem(0, 0)]
    assert len(centre) == 7
    for z in centre:
        P = L_mat(code.G, [z]).astype(np.int64)
        P5, P2 = np.kron(np.eye(5, dtype=np.int64), P), np.kron(np.eye(2, dtype=np.int64), P)
        rz = oracle.decode(dem_from_dense(H.astype(np.uint8), P5 @ p), prm, pack_bits((S @ P2.T) % 2),
                           trace_iters=4)
        for s_ in range(S.shape[0]):
            t = min(4, int(r["stats"][s_, 3]), int(rz["stats"][s_, 3]))
            assert np.allclose(rz["trace"][s_, :t], r["trace"][s_, :t] @ P5.T, rtol=1e-12, atol=1e-12)
        ez = unpack_bits(rz["corrections"], n).astype(np.int64)
        assert np.array_equal(ez[quick], ((eh @ P5.T) % 2)[quick])
        assert np.array_equal(rz["stats"][quick], r["stats"][quick])


# ---------------------------------------------------------------------------
# a7 minimum-weight select and the leg carry-over, pinned independently
# (Sec. 6.1 decoder configuration list: collect up to stop_nconv solutions
# over the relay legs and keep the one of least weight).
# ---------------------------------------------------------------------------
def _all_solutions(H: np.ndarray, syn: np.ndarray) -> set:
    """Every e in {0,1}^V with H e = s, by enumeration (V <= 12)."""
    C, V = H.shape
    out = set()
    for bits in itertools.product((0, 1), repeat=V):
        e = np.array(bits, dtype=np.int64)
        if np.array_equal((H.astype(np.int64) @ e) % 2, syn):
            out.add(bits)
    return out


def _random_small_dem(rng, C, V):
    H = np.zeros((C, V), dtype=np.uint8)
    for j in range(V):
        H[rng.choice(C, size=int(rng.integers(1, 3)), replace=False), j] = 1
    for i in range(C):
        if H[i].sum() == 1:                          # rows need 0 or >= 2 entries
            H[i, rng.choice(np.nonzero(H[i] == 0)[0])] = 1
    return H


def test_select_returns_first_least_weight_solution():
    """Every solution a decode records is a true solution of H e = s (checked
    against the brute-force solution set), its weight is the sum of the prior
    LLRs log((1-p)/p) over its ones (recomputed here from the bits), and the
    returned correction is the FIRST record of least weight.  The sample must
    contain shots where the least weight is not the first solution and shots
    where a heavier solution follows the least one, so that a select keeping
    the first or the last solution fails; the tie case is the next test."""
    rng = np.random.default_rng(7)
    seen_later_best = seen_heavier_after = 0
    for trial in range(12):
        C, V = int(rng.integers(3, 6)), int(rng.integers(6, 11))
        H = _random_small_dem(rng, C, V)
        pr = rng.uniform(0.02, 0.3, size=V)
        L0 = np.log((1 - pr) / pr)
        D = dem_from_dense(H, pr)
        P = DecodeParams(gamma0=0.1, pre_iter=20, num_sets=40, max_iterations=15, stop_nconv=5,
                         gamma_min=-0.24, gamma_max=0.66, seed=trial)
        for s in range(20):
            e = (rng.random(V) < 0.25).astype(np.uint8)
            syn = (H.astype(np.int64) @ e) % 2
            sols = _all_solutions(H, syn)
            r = oracle.solutions(D, P, pack_bits(syn), shot=s, cap=64)
            n = len(r["weights"])
            assert n == r["found"] == r["stats"][1] <= P.stop_nconv
            assert r["stats"][0] == (1 if n else 0)
            bits = unpack_bits(r["bits"], V)
            for k in range(n):
                assert tuple(int(x) for x in bits[k]) in sols, "a recorded solution does not satisfy H e = s"
                assert math.isclose(r["weights"][k], float(np.sum(L0[bits[k] == 1])), rel_tol=1e-12, abs_tol=1e-12)
            assert list(r["legs"]) == sorted(r["legs"]) and len(set(r["legs"])) == n   # one per leg, in order
            if n == 0:
                continue
            w = r["weights"]
            b = int(np.argmin(w))                      # numpy: first index of the minimum
            assert np.array_equal(r["correction"], r["bits"][b])
            assert r["weight"] == w[b]
            seen_later_best += b > 0
            seen_heavier_after += any(w[k] > w[b] for k in range(b + 1, n))
    assert seen_later_best >= 5 and seen_heavier_after >= 5, (seen_later_best, seen_heavier_after)


def test_select_keeps_earliest_of_equal_weights():
    """One check on two variables with equal priors and syndrome 1: the
    solutions {1,0} and {0,1} weigh the same.  Leg 0 (uniform memory strength)
    stays symmetric and never settles; each later leg's random strengths pick
    one of the two.  The returned correction must be the first solution found
    even when a later leg finds the other one."""
    p = 0.1
    H = np.array([[1, 1]], dtype=np.uint8)
    D = dem_from_dense(H, [p, p])
    L0 = math.log((1 - p) / p)
    swaps = 0
    for shot in range(40):
        P = DecodeParams(gamma0=0.125, pre_iter=5, num_sets=12, max_iterations=5, stop_nconv=4,
                         gamma_min=-0.24, gamma_max=0.66, seed=99)
        r = oracle.solutions(D, P, pack_bits(np.array([1])), shot=shot, cap=16)
        assert r["found"] == 4 and 0 not in r["legs"]
        assert np.all(r["weights"] == L0)
        assert np.array_equal(r["correction"], r["bits"][0])
        swaps += any(not np.array_equal(r["bits"][k], r["bits"][0]) for k in range(1, 4))
    assert swaps >= 10                                 # a '<=' select would return a later, different one


def test_carry_messages_two_check_recurrence():
    """Two checks on the same two variables, syndrome (1, 0): unsatisfiable,
    so every leg runs to its cap.  Each check has degree 2, so its message to
    one variable is its syndrome sign times the other variable's message to
    it: with x_c = nu_{c->1}, y_c = nu_{c->2}, sigma_c = (-1)^{s_c},
        x_1(t) = sigma_1 (L_2(t) + y_2(t-1)),  x_2(t) = sigma_2 (L_2(t) + y_1(t-1)),
        y_1(t) = sigma_1 (L_1(t) + x_2(t-1)),  y_2(t) = sigma_2 (L_1(t) + x_1(t-1)),
        M_1 = L_1 + x_1 + x_2,  M_2 = L_2 + y_1 + y_2,  L_k(t) = (1-g) L0_k + g M_k(t-1).
    At a leg boundary the messages restart from 0 by default and continue
    with carry_messages = 1; M carries in both."""
    pa, pb = 0.1, 0.3
    a, b = math.log((1 - pa) / pa), math.log((1 - pb) / pb)
    H = np.array([[1, 1], [1, 1]], dtype=np.uint8)
    D = dem_from_dense(H, [pa, pb])
    s1, s2 = -1.0, 1.0
    for carry in (False, True):
        for g in (0.125, 0.4, -0.2):
            T0, T1, legs = 4, 3, 3
            P = DecodeParams(gamma0=g, pre_iter=T0, num_sets=legs - 1, max_iterations=T1, stop_nconv=1,
                             gamma_min=g, gamma_max=g, carry_messages=carry, seed=5)
            r = oracle.decode(D, P, pack_bits(np.array([[1, 0]])), trace_iters=T0 + (legs - 1) * T1)
            M1, M2 = a, b
            x1 = x2 = y1 = y2 = 0.0
            want = []
            for leg in range(legs):
                if leg > 0 and not carry:
                    x1 = x2 = y1 = y2 = 0.0
                for _ in range(T0 if leg == 0 else T1):
                    L1, L2 = (1 - g) * a + g * M1, (1 - g) * b + g * M2
                    x1, x2, y1, y2 = s1 * (L2 + y2), s2 * (L2 + y1), s1 * (L1 + x2), s2 * (L1 + x1)
                    M1, M2 = L1 + x1 + x2, L2 + y1 + y2
                    want.append((M1, M2))
            assert np.allclose(r["trace"][0], np.array(want), rtol=1e-12, atol=1e-12), (carry, g)
            assert r["stats"][0, 0] == 0 and r["stats"][0, 2] == legs


def test_soft_syndrome_objective_against_enumeration():
    """The soft-syndrome training objective (objective 1): for each iteration
    and check, the probability that independent bits, bit j in error with
    probability sigmoid(-M_j), have the row's syndrome parity -- computed here
    by enumerating every error pattern on the row's variables -- enters the
    loss as -log(eps + (1 - 2 eps) P); summed over checks and the T
    iterations of the forward (whose posteriors the trace gives)."""
    pr = [0.1, 0.3, 0.2, 0.05, 0.4]
    H = np.array([[1, 1, 0, 1, 0], [0, 1, 1, 0, 1], [1, 0, 1, 1, 1]], dtype=np.uint8)
    D = dem_from_dense(H, pr)
    T = 3
    w = np.random.default_rng(5).uniform(0.6, 1.2, (T, D.n_edges))
    knots = np.linspace(-0.1, 0.5, 9)
    syn = pack_bits(np.array([[1, 0, 1], [0, 0, 0], [1, 1, 0]]))
    err = pack_bits(np.zeros((3, 5), dtype=np.uint8))
    loss, tr = oracle.learned_loss(D, w, knots, 13, syn, err, trace=True, objective=1)
    eps = 1e-6
    S = unpack_bits(syn, 3)
    for s_ in range(3):
        want = 0.0
        for t in range(T):
            q = 1.0 / (1.0 + np.exp(tr[s_, t]))          # P(bit in error) = sigmoid(-M)
            for i in range(3):
                vars_ = np.nonzero(H[i])[0]
                P = 0.0
                for bits in itertools.product((0, 1), repeat=len(vars_)):
                    pb = np.prod([q[v] if b else 1 - q[v] for v, b in zip(vars_, bits)])
                    if sum(bits) % 2 == S[s_, i]:
                        P += pb
                want -= math.log(eps + (1 - 2 * eps) * P)
        assert math.isclose(loss[s_], want, rel_tol=1e-10), (s_, loss[s_], want)
    # the cross-entropy objective on the same run is a different number
    l0, _ = oracle.learned_loss(D, w, knots, 13, syn, err, objective=0)
    assert not np.allclose(l0, loss)


def test_learned_weights_end_at_the_trained_horizon():
    """Learned weights apply to the first T iterations of a leg; later
    iterations use unit weights: with w[T-1] = 0.5 and more iterations than T,
    the decode equals the one whose weight table is extended by ones, and
    differs from the one that repeats w[T-1]."""
    D = circuit_dem("ZSZ-LP-60", 0.006, 3, "Z")
    syn, _, _ = oracle.sample(D, 29, 0, 24)
    P = DecodeParams(num_sets=4, pre_iter=30, max_iterations=20, seed=4)
    T = 3
    w = np.random.default_rng(6).uniform(0.5, 0.9, (T, D.n_edges))
    a = oracle.decode(D, P, syn, w=w, trace_iters=12)
    b = oracle.decode(D, P, syn, w=np.vstack([w, np.ones((40, D.n_edges))]), trace_iters=12)
    c = oracle.decode(D, P, syn, w=np.vstack([w, np.repeat(w[-1:], 40, axis=0)]), trace_iters=12)
    assert np.array_equal(a["trace"], b["trace"], equal_nan=True) and np.array_equal(a["stats"], b["stats"])
    assert not np.array_equal(a["trace"], c["trace"])
