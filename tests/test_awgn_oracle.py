"""Pins of the classical channel-coding oracle (BPSK over AWGN, sum-product
BP; arXiv 2607.27644 Sec. 6.2) and of the OSD-0 post-processing oracle
(Sec. 7, improved decoding) to what the mathematics fixes."""
import itertools

import numpy as np
import pytest
from scipy import stats

import oracle
from workloads.zsz import gf2_nullspace, load_code


def _csr(H):
    H = np.asarray(H, dtype=np.uint8)
    indptr = np.r_[0, np.cumsum(H.sum(1))].astype(np.int32)
    indices = np.concatenate([np.nonzero(r)[0] for r in H]).astype(np.int32)
    return indptr, indices


def _random_tree_code(rng, n_checks):
    """A parity-check matrix whose Tanner graph is a tree: each new check
    attaches to one existing variable and brings 1-3 new ones."""
    rows, n = [], 1
    for _ in range(n_checks):
        old = int(rng.integers(n))
        new = list(range(n, n + int(rng.integers(1, 4))))
        n += len(new)
        rows.append([old] + new)
    H = np.zeros((n_checks, n), dtype=np.uint8)
    for i, r in enumerate(rows):
        H[i, r] = 1
    return H


def test_degree_two_check_passes_the_other_llr():
    """A single parity check on two bits: the check message to one bit is the
    other bit's LLR exactly (phi(phi(x)) = x), so after one iteration the
    posteriors are L1 + L2 for both bits."""
    H = np.array([[1, 1]])
    ip, ix = _csr(H)
    L = np.array([[0.3, -1.7], [4.0, 2.5], [-0.01, 7.25]])
    r = oracle.sum_product(ip, ix, 1, 2, L, max_iter=1, early_stop=False, posteriors=True)
    want = L.sum(1, keepdims=True) * np.ones((1, 2))
    assert np.allclose(r["posteriors"], want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_tree_codes_reach_exact_bitwise_map(seed):
    """On a cycle-free Tanner graph sum-product BP reaches the exact bitwise
    MAP log-likelihood ratios, here computed by summing over every codeword."""
    rng = np.random.default_rng(seed)
    H = _random_tree_code(rng, int(rng.integers(3, 7)))
    m, n = H.shape
    G = gf2_nullspace(H)
    words = np.array([(np.array(c) @ G) % 2 for c in itertools.product((0, 1), repeat=G.shape[0])])
    L = rng.uniform(-2.0, 2.0, (4, n))
    ip, ix = _csr(H)
    r = oracle.sum_product(ip, ix, m, n, L, max_iter=2 * n + 2, early_stop=False, posteriors=True)
    for s in range(L.shape[0]):
        logp = ((1 - 2 * words) * L[s]).sum(1) / 2.0            # log P(c | y) up to a constant
        for j in range(n):
            a = np.logaddexp.reduce(logp[words[:, j] == 0])
            b = np.logaddexp.reduce(logp[words[:, j] == 1])
            assert r["posteriors"][s, j] == pytest.approx(a - b, abs=1e-9)


def test_decoder_symmetry_under_codeword_flips():
    """BPSK-AWGN with a linear code: flipping the LLR signs on the support of a
    codeword c flips the decision by exactly c (sum-product treats signs and
    magnitudes separately), at any noise level."""
    code = load_code("ZSZ-LP-160")
    H = code.H_left
    m, n = H.shape
    G = gf2_nullspace(H)
    ip, ix = _csr(H)
    L0 = oracle.awgn_llr(n, oracle.awgn_sigma(1.5, 0.5), 7, 0, 40)
    rng = np.random.default_rng(2)
    c = (rng.integers(0, 2, (40, G.shape[0])) @ G) % 2
    Lc = np.where(c == 1, -L0, L0)
    r0 = oracle.sum_product(ip, ix, m, n, L0)
    rc = oracle.sum_product(ip, ix, m, n, Lc)
    h0 = oracle.unpack_bits(r0["bits"], n)
    hc = oracle.unpack_bits(rc["bits"], n)
    assert np.array_equal(hc, h0 ^ c)
    assert np.array_equal(rc["iters"], r0["iters"]) and np.array_equal(rc["valid"], r0["valid"])


def test_awgn_llr_distribution():
    """All-zero codeword: L = 2 y / sigma^2 with y ~ N(1, sigma^2), i.e.
    L ~ N(2/sigma^2, 4/sigma^2) (Sec. 6.2); codeword bits flip the mean; the
    underlying draws pass a Kolmogorov-Smirnov test against N(0, 1)."""
    sigma = oracle.awgn_sigma(1.0, 0.5)
    n, shots = 500, 200
    L = oracle.awgn_llr(n, sigma, 11, 0, shots, llr_max=1e9)
    z = (L * sigma ** 2 / 2.0 - 1.0) / sigma
    assert abs(z.mean()) < 5 / np.sqrt(z.size) and abs(z.std() - 1.0) < 5 / np.sqrt(2 * z.size)
    assert stats.kstest(z.ravel(), "norm").pvalue > 1e-3
    cw = np.full((shots, (n + 31) // 32), 0xffffffff, dtype=np.uint32)
    L1 = oracle.awgn_llr(n, sigma, 11, 0, shots, codewords=cw, llr_max=1e9)
    assert np.allclose(L1, L - 4.0 / sigma ** 2)
    Lc = oracle.awgn_llr(n, sigma, 11, 0, shots)                  # default clip at +-20
    assert np.abs(Lc).max() <= 20.0 and np.array_equal(Lc, np.clip(L, -20, 20))


def test_shannon_limit_of_rate_half_bpsk():
    """The BPSK-AWGN capacity 1 - E[log2(1 + e^-L)], L ~ N(2/s^2, 4/s^2),
    equals 1/2 at E_b/N_0 = 0.19 dB for R = 1/2 (Sec. 6.2): pins the E_b/N_0
    to sigma conversion the sampler uses."""
    x, w = np.polynomial.hermite_e.hermegauss(200)
    w = w / w.sum()

    def capacity(sigma):
        L = 2 / sigma ** 2 + (2 / sigma) * x
        return 1.0 - float((w * np.logaddexp(0.0, -L) / np.log(2.0)).sum())

    lo, hi = -2.0, 3.0
    for _ in range(60):
        mid = (lo + hi) / 2
        if capacity(oracle.awgn_sigma(mid, 0.5)) < 0.5:
            lo = mid
        else:
            hi = mid
    assert abs(lo - 0.19) < 0.01


def test_zsz_2bga_64_decoding_regimes():
    """ZSZ-2BGA-64 (the left seed code of ZSZ-LP-160, [64, 32, 10]): at 6 dB
    every transmission decodes to the sent codeword within a few iterations;
    at 0.5 dB some fail; every decision flagged valid satisfies H c^ = 0."""
    H = load_code("ZSZ-LP-160").H_left
    m, n = H.shape
    ip, ix = _csr(H)
    for ebn0, all_ok in ((6.0, True), (0.5, False)):
        L = oracle.awgn_llr(n, oracle.awgn_sigma(ebn0, 0.5), 5, 0, 300)
        r = oracle.sum_product(ip, ix, m, n, L, max_iter=100)
        h = oracle.unpack_bits(r["bits"], n).astype(np.int64)
        assert np.all(((h[r["valid"]] @ H.T) % 2) == 0)
        ok = r["valid"] & ~h.any(1)
        if all_ok:
            assert ok.all() and r["iters"].max() <= 10
        else:
            assert 0 < (~ok).sum() < 300


def _info_set(H, order):
    """First rank(H) columns of `order` that are independent over GF(2)
    (greedy, by rank of the growing prefix)."""
    from workloads.zsz import gf2_rank
    chosen = []
    for c in order:
        if gf2_rank(H[:, chosen + [c]]) > len(chosen):
            chosen.append(c)
    return chosen


def test_osd0_solution_lives_on_the_information_set():
    """[[60,12,6]] code capacity (H_X): for random errors and random soft
    values, OSD-0 returns a solution of H e = s supported on the information
    set (computed here independently by growing ranks) -- unique there."""
    from workloads.dem import code_capacity_dem
    D = code_capacity_dem("ZSZ-LP-60", 0.05)
    H = D.dense_H().astype(np.uint8)
    m, n = H.shape
    rng = np.random.default_rng(4)
    E = (rng.random((20, n)) < 0.06).astype(np.uint8)
    S = (E.astype(np.int64) @ H.T) % 2
    soft = rng.normal(0.0, 3.0, (20, n))
    r = oracle.osd0(D.H_indptr, D.H_indices, m, n, oracle.pack_bits(S), soft)
    e = oracle.unpack_bits(r["corrections"], n).astype(np.int64)
    assert r["valid"].all()
    assert np.array_equal((e @ H.T) % 2, S)
    for s in range(20):
        order = sorted(range(n), key=lambda j: (soft[s, j], j))
        info = set(_info_set(H, order))
        assert set(np.nonzero(e[s])[0]) <= info


def test_osd0_recovers_errors_ranked_first():
    """When the soft values rank the true error's support first and that
    support is independent (weight < the code distance 6), OSD-0 returns the
    error itself."""
    from workloads.dem import code_capacity_dem
    D = code_capacity_dem("ZSZ-LP-60", 0.05)
    H = D.dense_H().astype(np.uint8)
    m, n = H.shape
    rng = np.random.default_rng(5)
    E = np.zeros((30, n), dtype=np.uint8)
    for t in range(30):
        E[t, rng.choice(n, 1 + t % 5, replace=False)] = 1
    S = (E.astype(np.int64) @ H.T) % 2
    soft = np.where(E == 1, -8.0, 4.0) + rng.uniform(-1, 1, E.shape)
    r = oracle.osd0(D.H_indptr, D.H_indices, m, n, oracle.pack_bits(S), soft)
    assert np.array_equal(oracle.unpack_bits(r["corrections"], n), E)


def test_osd0_flags_syndromes_outside_the_column_space():
    """A rank-deficient check matrix (a repeated row): syndromes that break
    the row dependency are flagged invalid, the others solved."""
    H = np.array([[1, 1, 0, 1], [0, 1, 1, 1], [1, 1, 0, 1]], dtype=np.uint8)
    ip, ix = _csr(H)
    S = np.array([[1, 0, 1], [1, 0, 0], [0, 1, 0]])
    r = oracle.osd0(ip, ix, 3, 4, oracle.pack_bits(S), np.zeros((3, 4)))
    assert list(r["valid"]) == [True, False, True]
    e = oracle.unpack_bits(r["corrections"], 4).astype(np.int64)
    for s in (0, 2):
        assert np.array_equal((e[s] @ H.T) % 2, S[s])


def _gf2_solve(A, b):
    """x with A x = b over GF(2) for A of full column rank (plain elimination)."""
    A = (np.asarray(A, dtype=np.uint8) % 2).copy()
    b = (np.asarray(b, dtype=np.uint8) % 2).copy()
    m, k = A.shape
    row, piv = 0, []
    for c in range(k):
        p = next((i for i in range(row, m) if A[i, c]), None)
        assert p is not None
        A[[row, p]] = A[[p, row]]
        b[[row, p]] = b[[p, row]]
        for i in range(m):
            if i != row and A[i, c]:
                A[i] ^= A[row]
                b[i] ^= b[row]
        piv.append(c)
        row += 1
    assert not b[row:].any()
    return b[:k]


def test_osd_combination_sweep_minimises_weight():
    """OSD with order 8: independently, for the information set and each flip
    of one or two of the first 8 other columns, solve H e = s and weigh e by
    the prior LLRs; the oracle's answer attains the least weight, is valid,
    and never weighs more than its OSD-0 answer."""
    from workloads.dem import circuit_dem
    D = circuit_dem("ZSZ-LP-60", 0.01, 1, "Z")
    H = D.dense_H().astype(np.uint8)
    m, n = H.shape
    w = np.log((1 - D.priors) / D.priors)
    rng = np.random.default_rng(8)
    E = (rng.random((8, n)) < 0.01).astype(np.uint8)
    S = (E.astype(np.int64) @ H.T) % 2
    soft = rng.normal(2.0, 3.0, (8, n))
    lam = 8
    r = oracle.osd(D.H_indptr, D.H_indices, m, n, oracle.pack_bits(S), soft, order=lam, weights=w)
    r0 = oracle.osd0(D.H_indptr, D.H_indices, m, n, oracle.pack_bits(S), soft)
    e = oracle.unpack_bits(r["corrections"], n).astype(np.int64)
    e0 = oracle.unpack_bits(r0["corrections"], n).astype(np.int64)
    assert np.array_equal((e @ H.T) % 2, S)
    for s in range(S.shape[0]):
        order = sorted(range(n), key=lambda j: (soft[s, j], j))
        info = _info_set(H, order)
        rest = [c for c in order if c not in set(info)][:lam]
        best = None
        for T in [()] + [(a,) for a in rest] + [(a, b) for i, a in enumerate(rest) for b in rest[i + 1:]]:
            rhs = S[s].copy()
            for c in T:
                rhs ^= H[:, c]
            x = _gf2_solve(H[:, info], rhs)
            cand = np.zeros(n, dtype=np.int64)
            cand[info] = x
            cand[list(T)] = 1
            cw = float(w[cand == 1].sum())
            best = cw if best is None else min(best, cw)
        assert float(w[e[s] == 1].sum()) == pytest.approx(best, rel=1e-12)
        assert float(w[e[s] == 1].sum()) <= float(w[e0[s] == 1].sum()) + 1e-12
