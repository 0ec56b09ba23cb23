"""Pins of the input generators (ZSZ-LP codes, circuit DEMs) to the paper's tables."""
import os

import numpy as np
import pytest

from workloads.zsz import load_code, gf2_rank, ZSZGroup
from workloads.dem import circuit_dem, code_capacity_dem, memory_circuit

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def _girth(H):
    """Tanner-graph girth by BFS from every vertex (plain)."""
    m, n = H.shape
    adj = [[] for _ in range(m + n)]
    for i, j in zip(*np.nonzero(H)):
        adj[i].append(m + j)
        adj[m + j].append(i)
    best = 10 ** 9
    for s in range(m + n):
        dist = {s: 0}
        par = {s: -1}
        q = [s]
        for u in q:
            for w in adj[u]:
                if w not in dist:
                    dist[w] = dist[u] + 1
                    par[w] = u
                    q.append(w)
                elif par[u] != w:
                    best = min(best, dist[u] + dist[w] + 1)
    return best


def _cycles46(H):
    """Exact simple 4- and 6-cycle counts of a Tanner graph.

    4-cycles: check pairs sharing o variables give C(o,2).  6-cycles: for each
    unordered check triple with pairwise overlaps o12,o23,o13 and common
    variables T, choose one variable per pair, all distinct:
    o12*o23*o13 - T*(o12+o23+o13-2) (inclusion-exclusion).
    """
    H = H.astype(np.int64)
    O = H @ H.T
    m = H.shape[0]
    np.fill_diagonal(O, 0)
    c4 = int((O * (O - 1) // 2)[np.triu_indices(m, 1)].sum())
    c6 = 0
    nbr = [np.nonzero(O[i])[0] for i in range(m)]
    for i in range(m):
        for j in nbr[i]:
            if j <= i:
                continue
            for k in nbr[j]:
                if k <= j or O[i, k] == 0:
                    continue
                T = int((H[i] & H[j] & H[k]).sum())
                o1, o2, o3 = O[i, j], O[j, k], O[i, k]
                c6 += int(o1 * o2 * o3 - T * (o1 + o2 + o3 - 2))
    return c4, c6


@pytest.mark.parametrize("row", _table("zsz_lp_tables.txt"), ids=lambda r: r[0])
def test_code_tables(row):
    name, n, k, gl, gr, c4, c6, zc, nu2, nu3 = row[0], *map(int, row[1:])
    code = load_code(name)
    G = code.G
    assert pow(code.q, code.l2, code.l1) == 1
    assert code.n == n
    # CSS orthogonality H_X H_Z^T = 0 (Eq. 5-block CSS orth)
    assert not np.any((code.H_X.astype(np.int64) @ code.H_Z.T.astype(np.int64)) % 2)
    # full-rank seeds give k = l (Sec. 2.4) and match Table 1
    assert gf2_rank(code.H_left) == code.ell and gf2_rank(code.H_right) == code.ell
    assert code.k == k == code.ell
    # weight-9 checks; qubit degrees 3 on Q1..Q4 and 6 on Q5
    for H in (code.H_X, code.H_Z):
        assert set(H.sum(1).tolist()) == {9}
        cw = H.sum(0)
        assert set(cw[:4 * code.ell].tolist()) == {3} and set(cw[4 * code.ell:].tolist()) == {6}
    # Table 8: cycle counts summed over H_X and H_Z
    a, b = _cycles46(code.H_X), _cycles46(code.H_Z)
    assert a[0] + b[0] == c4 and a[1] + b[1] == c6
    # Table 11: center size; Table 6: element-order census
    assert len(G.center()) == zc
    orders = [G.element_order(g) for g in range(G.order)]
    assert orders.count(2) == nu2 and orders.count(3) == nu3
    # Table 2: classical girths (small codes only; BFS is quadratic)
    if code.ell <= 64:
        assert _girth(code.H_left) == gl and _girth(code.H_right) == gr


def test_equivariance_and_center():
    """R[g] H_left = H_left R[g]^{+2} (Eq. H_left symmetry) and H P_z^{+5} = P_z^{+2} H (App. D)."""
    code = load_code("ZSZ-LP-160")
    G = code.G
    from workloads.zsz import R_mat, L_mat
    for g in range(G.order):
        Rg = R_mat(G, [g])
        lhs = (Rg.astype(int) @ code.H_left) % 2
        rhs = (code.H_left.astype(int) @ np.kron(np.eye(2, dtype=int), Rg)) % 2
        assert np.array_equal(lhs, rhs)
    for z in G.center():
        P = L_mat(G, [z]).astype(int)
        for H in (code.H_X, code.H_Z):
            assert np.array_equal((H @ np.kron(np.eye(5, dtype=int), P)) % 2, (np.kron(np.eye(2, dtype=int), P) @ H) % 2)


def test_ogm_generators_160():
    """Table 7 generators satisfy u_L a~ + v_L b~ = 0 and c~ u_R + d~ v_R = 0 (Eq. generator validity)."""
    code = load_code("ZSZ-LP-160")
    G = code.G

    def alg(terms):
        v = np.zeros(G.order, dtype=np.uint8)
        for (a, b) in terms:
            v[G.elem(a, b)] ^= 1
        return v

    def mul(u, v):
        out = np.zeros(G.order, dtype=np.uint8)
        for g in np.nonzero(u)[0]:
            for h in np.nonzero(v)[0]:
                out[G.mul[g, h]] ^= 1
        return out

    def bar(u):
        out = np.zeros_like(u)
        out[G.inv[np.nonzero(u)[0]]] = 1
        return out

    uL = alg([(8, 0), (11, 0), (4, 1), (8, 1), (13, 1)])
    vL = alg([(0, 0), (10, 0), (15, 0), (3, 1), (11, 1)])
    uR = alg([(3, 0), (8, 0), (13, 0), (3, 1), (5, 1), (7, 1), (10, 1)])
    vR = alg([(5, 0), (8, 0), (10, 1)])
    a, b = alg(code.a_terms), alg(code.b_terms)
    c, d = alg(code.c_terms), alg(code.d_terms)
    assert not np.any(mul(uL, bar(a)) ^ mul(vL, bar(b)))
    assert not np.any(mul(bar(c), uR) ^ mul(bar(d), vR))
    assert uL.sum() + vL.sum() == code.d and uR.sum() + vR.sum() == code.d


def test_dem_160_structure():
    d = 10
    D = circuit_dem("ZSZ-LP-160", 0.001, d, "Z")
    code = load_code("ZSZ-LP-160")
    assert D.n_det == 2 * code.ell * (d + 1)            # Table 5: N_det = 2 l (d+1)
    assert D.n_obs == code.k
    assert np.all(np.diff(D.H_indptr) >= 2)             # every detector sees >= 2 mechanisms
    assert np.all((D.priors > 0) & (D.priors < 0.01))
    Dx = circuit_dem("ZSZ-LP-160", 0.001, d, "X")
    assert Dx.n_det == D.n_det and Dx.n_obs == D.n_obs


def test_dem_noiseless_limit_and_scaling():
    """Fault probabilities scale with p and the structure does not depend on p."""
    a = circuit_dem("ZSZ-LP-60", 0.001, 3, "Z")
    b = circuit_dem("ZSZ-LP-60", 0.002, 3, "Z")
    assert np.array_equal(a.H_indices, b.H_indices) and np.array_equal(a.H_indptr, b.H_indptr)
    r = b.priors / a.priors
    assert np.all((r > 1.9) & (r <= 2.0 + 1e-12))


@pytest.mark.parametrize("row", _table("dem_sizes.txt"), ids=lambda r: r[0])
def test_dem_sizes_table5(row):
    """(N_det, N_loc) of Table 5: 1920/28992, 2652/40326, 4180/63910."""
    name, rounds, ndet, nloc = row[0], *map(int, row[1:])
    D = circuit_dem(name, 0.001, rounds, "Z")
    assert (D.n_det, D.n_loc) == (ndet, nloc)


def test_dem_single_fault_consistency():
    """A tiny circuit: every column's detector set is what one fault propagates to.

    Cross-check by an independent dense GF(2) propagation of a single X error on
    a data qubit before round 1: it must flip exactly the Z-checks touching it
    in round 1 (time-like pair) -- i.e. the column equals H_Z[:, q] in round 0.
    """
    code = load_code("ZSZ-LP-60")
    D = circuit_dem("ZSZ-LP-60", 0.001, 2, "Z")
    Hd = D.dense_H()
    cols = {tuple(np.nonzero(Hd[:, j])[0]) for j in range(D.n_loc)}
    for q in range(code.n):
        want = tuple(np.nonzero(code.H_Z[:, q])[0])           # detectors of round 1
        assert want in cols
    # a measurement flip of Z-ancilla i in round 1 flips detectors (1,i) and (2,i)
    l2 = 2 * code.ell
    for i in range(l2):
        assert (i, l2 + i) in cols


def test_code_capacity_dem():
    D = code_capacity_dem("ZSZ-LP-160", 0.05)
    assert (D.n_det, D.n_loc, D.n_obs) == (64, 160, 32)
    assert D.n_edges == 576


def test_multi_p_builder_matches_single():
    from workloads.dem import circuit_dems
    many = circuit_dems("ZSZ-LP-60", [0.001, 0.0025, 0.004], 3, "Z")
    for D in many:
        one = circuit_dem("ZSZ-LP-60", D.meta["p"], 3, "Z")
        assert np.array_equal(D.H_indices, one.H_indices) and np.array_equal(D.priors, one.priors)


@pytest.mark.parametrize("basis,n_single,n_cx", [("Z", None, 200), ("X", 120, 60)])
def test_dem_faults_match_tableau_simulation(basis, n_single, n_cx):
    """The DEM builder's per-fault detector and observable flips against an
    independent stabilizer-tableau simulation of the same circuit (CHP,
    Aaronson-Gottesman 2004), on the [[60,12,6]] code with 2 rounds: the
    noiseless circuit gives all detectors and observables 0 under random
    measurement outcomes; every reset and measurement fault and a seeded
    sample of the CNOT Pauli components flip exactly what the Pauli-frame
    propagation says; and each such flip pattern is a column of the DEM."""
    from chp import run_memory_circuit
    from workloads.dem import _count_faults, _frame_sim, _set_bits_by_fault
    code = load_code("ZSZ-LP-60")
    circ, info = memory_circuit(code, 2, basis)
    for seed in range(3):
        d, o = run_memory_circuit(circ, info, None, seed)
        assert not d.any() and not o.any()
    nf = _count_faults(circ)
    rec, _ = _frame_sim(circ, 0.001, 0, nf)
    fa, row = _set_bits_by_fault(rec, nf)
    R = np.zeros((nf, circ.n_kept), dtype=np.int64)
    R[fa, row] = 1
    Dm = np.zeros((circ.n_kept, len(info["detectors"])), dtype=np.int64)
    for k, rows in enumerate(info["detectors"]):
        Dm[rows, k] = 1
    Om = np.zeros((circ.n_kept, len(info["observables"])), dtype=np.int64)
    for k, rows in enumerate(info["observables"]):
        Om[rows, k] = 1
    FD, FO = (R @ Dm) % 2, (R @ Om) % 2
    # fault ids: resets and measurements by op, CNOT components sampled
    single, cx = [], []
    base = 0
    for op in circ.ops:
        n_op = len(op[1]) * (15 if op[0] == "CX" else 1)
        (cx if op[0] == "CX" else single).extend(range(base, base + n_op))
        base += n_op
    assert base == nf
    rng = np.random.default_rng(7)
    if n_single is not None:
        single = list(rng.choice(single, n_single, replace=False))
    pick = list(single) + list(rng.choice(cx, n_cx, replace=False))
    D = circuit_dem("ZSZ-LP-60", 0.001, 2, basis)
    Hd, Od = D.dense_H(), D.dense_O()
    cols = {(tuple(np.nonzero(Hd[:, j])[0]), tuple(np.nonzero(Od[:, j])[0])) for j in range(D.n_loc)}
    for f in pick:
        d, o = run_memory_circuit(circ, info, int(f), int(f))
        assert np.array_equal(d, FD[f]) and np.array_equal(o, FO[f]), f
        if d.any() or o.any():
            assert (tuple(np.nonzero(d)[0]), tuple(np.nonzero(o)[0])) in cols, f


def test_min_weight_enumerator_small_codes():
    """The Gray-code enumerator against direct enumeration of every message on
    small random codes, and the [7,4,3] Hamming code."""
    import itertools
    import oracle
    ham = np.array([[1, 0, 0, 0, 0, 1, 1], [0, 1, 0, 0, 1, 0, 1], [0, 0, 1, 0, 1, 1, 0], [0, 0, 0, 1, 1, 1, 1]])
    assert oracle.min_weight(ham) == 3
    rng = np.random.default_rng(3)
    for k, n in ((5, 12), (9, 20), (10, 64)):
        G = rng.integers(0, 2, (k, n))
        best = min(int(((np.array(m) @ G) % 2).sum()) for m in itertools.product((0, 1), repeat=k) if any(m)
                   if ((np.array(m) @ G) % 2).any())
        assert oracle.min_weight(G) == best


@pytest.mark.parametrize("row", _table("zsz_2bga_distances.txt"), ids=lambda r: r[0])
def test_classical_seed_distance_brute_force(row):
    """Table 2: the seed codes H_left and H_right of ZSZ-LP-160 are [64, 32, 10],
    checked by enumerating all 2^32 codewords of each."""
    import oracle
    from workloads.zsz import gf2_nullspace
    name, n, k, dl, dr = row[0], *map(int, row[1:])
    code = load_code(name)
    for H, d in ((code.H_left, dl), (code.H_right, dr)):
        G = gf2_nullspace(H)
        assert H.shape[1] == n and G.shape[0] == k
        assert not ((G.astype(np.int64) @ H.T.astype(np.int64)) % 2).any()
        assert oracle.min_weight(G) == d


def _ogs_rows():
    rows = []
    for r in _table("ogs_generators.txt"):
        terms = [(int(a), int(g.split(":")[0])) for g in r[3:] for a in g.split(":")[1].split(",")]
        rows.append((r[0], r[1], int(r[2]), terms))
    return rows


@pytest.mark.parametrize("row", _ogs_rows(), ids=lambda r: f"{r[0]}-{r[1]}")
def test_ogs_generators(row):
    """Table 8: with u = 1 the generator validity conditions u_L a~ + v_L b~ = 0
    and c~ u_R + d~ v_R = 0 become v_L b~ = a~ and d~ v_R = c~; the printed
    systematic polynomials satisfy them, have the printed weights, and are the
    unique solutions (b and d are units: L[b], L[d] have full rank)."""
    name, side, weight, terms = row
    code = load_code(name)
    G = code.G

    def alg(ts):
        v = np.zeros(G.order, dtype=np.uint8)
        for (a, b) in ts:
            v[G.elem(a, b)] ^= 1
        return v

    def mul(u, v):
        out = np.zeros(G.order, dtype=np.uint8)
        for g in np.nonzero(u)[0]:
            for h in np.nonzero(v)[0]:
                out[G.mul[g, h]] ^= 1
        return out

    def bar(u):
        out = np.zeros_like(u)
        out[G.inv[np.nonzero(u)[0]]] = 1
        return out

    def left_matrix(u):                     # column h = u * h
        M = np.zeros((G.order, G.order), dtype=np.uint8)
        for h in range(G.order):
            for g in np.nonzero(u)[0]:
                M[G.mul[g, h], h] ^= 1
        return M

    v = alg(terms)
    assert len(terms) == weight and v.sum() == weight
    if side == "L":
        a, b = alg(code.a_terms), alg(code.b_terms)
        assert np.array_equal(mul(v, bar(b)), bar(a))
        assert gf2_rank(left_matrix(b)) == G.order
    else:
        c, d = alg(code.c_terms), alg(code.d_terms)
        assert np.array_equal(mul(bar(d), v), bar(c))
        assert gf2_rank(left_matrix(d)) == G.order


def test_ogm_orbits_give_full_rank_logical_bases_160():
    """Sec. 3.2 and Table 7: the OGM seed codewords (bar u, bar v) of H_left and
    H_right (weight d = 10) generate, under the group action that commutes
    with each seed code (right multiplication for H_left = (L[a] L[b]), left
    for H_right = (R[c] R[d])), orbits of rank l = 32; embedded as
    z1 = (c1, 0, c2, 0, 0), z2 = (0, c1, 0, c2, 0) they lie in ker H_X, as
    x1 = (c1, c2, 0, 0, 0), x2 = (0, 0, c1, c2, 0) in ker H_Z, and span a
    full k = 32 dimensional logical space outside rs H_Z (rs H_X); z1 has
    weight 10, so d_Z <= 10."""
    code = load_code("ZSZ-LP-160")
    G, ell = code.G, code.ell

    def alg(ts):
        v = np.zeros(G.order, dtype=np.uint8)
        for (a, b) in ts:
            v[G.elem(a, b)] ^= 1
        return v

    def bar(u):
        out = np.zeros_like(u)
        out[G.inv[np.nonzero(u)[0]]] = 1
        return out

    def right(x, g):                       # R[g]: basis element h -> h g
        out = np.zeros_like(x)
        out[G.mul[np.nonzero(x)[0], g]] = 1
        return out

    def left(x, g):                        # L[g]: basis element h -> g h
        out = np.zeros_like(x)
        out[G.mul[g, np.nonzero(x)[0]]] = 1
        return out

    cl = (bar(alg([(8, 0), (11, 0), (4, 1), (8, 1), (13, 1)])), bar(alg([(0, 0), (10, 0), (15, 0), (3, 1), (11, 1)])))
    cr = (bar(alg([(3, 0), (8, 0), (13, 0), (3, 1), (5, 1), (7, 1), (10, 1)])), bar(alg([(5, 0), (8, 0), (10, 1)])))
    z0 = np.zeros(ell, dtype=np.uint8)
    orb_l = np.array([np.r_[right(cl[0], g), right(cl[1], g)] for g in range(ell)])
    orb_r = np.array([np.r_[left(cr[0], g), left(cr[1], g)] for g in range(ell)])
    assert not ((orb_l.astype(int) @ code.H_left.T.astype(int)) % 2).any()
    assert not ((orb_r.astype(int) @ code.H_right.T.astype(int)) % 2).any()
    assert gf2_rank(orb_l) == ell and gf2_rank(orb_r) == ell
    Z = np.array([np.r_[c[:ell], z0, c[ell:], z0, z0] for c in orb_l] +
                 [np.r_[z0, c[:ell], z0, c[ell:], z0] for c in orb_l])
    X = np.array([np.r_[c[:ell], c[ell:], z0, z0, z0] for c in orb_r] +
                 [np.r_[z0, z0, c[:ell], c[ell:], z0] for c in orb_r])
    assert not ((Z.astype(int) @ code.H_X.T.astype(int)) % 2).any()
    assert not ((X.astype(int) @ code.H_Z.T.astype(int)) % 2).any()
    assert gf2_rank(np.r_[code.H_Z, Z]) - gf2_rank(code.H_Z) == code.k
    assert gf2_rank(np.r_[code.H_X, X]) - gf2_rank(code.H_X) == code.k
    assert Z[0].sum() == code.d and gf2_rank(np.r_[code.H_Z, Z[:1]]) > gf2_rank(code.H_Z)
