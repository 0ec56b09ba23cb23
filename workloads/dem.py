"""Syndrome-extraction circuits and detector error models (seeded input generator).

Builds the detector error model (DEM) that the decoder consumes: a sparse
detector x fault matrix H, fault probabilities p_j and an observable x fault
matrix O.  It is an input generator shared by the CUDA path and the oracle and
holds none of the decoder's arithmetic.

Paper references (arXiv 2607.27644):
  * Sec. 5 and App. E, Table 10: sequential X-then-Z syndrome extraction with
    the greedy monomial gate order; X-check CNOTs point ancilla -> data, Z-check
    CNOTs data -> ancilla.  A table entry (check block, data block, term) applies
    the CNOTs of every Tanner edge that term contributes to that block.
  * Sec. 6.1, noise model: depolarising noise of strength p after every
    two-qubit gate, preparation flips with probability p, measurement flips with
    probability p; no idle or single-qubit noise.
  * Sec. 6.1, memory experiments: X- (Z-) memory prepares |+> (|0>), runs d
    rounds of X+Z extraction and measures the data in X (Z).
  * Table 5: N_det = 2*l*(d+1) detectors for a d-round memory experiment.

Readings where the paper is silent (stated again in the design notes):
  * each of the 15 two-qubit Pauli components is an independent mechanism with
    probability p/15;
  * only detectors of the memory type are kept (Z checks for Z-memory);
  * mechanisms with identical (detector set, observable set) merge by
    p <- p1 + p2 - 2 p1 p2; mechanisms that flip nothing are dropped.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .zsz import ZSZLPCode, load_code

# ---------------------------------------------------------------------------
# Table 10 (App. E): CNOT layers.  Token "CQt<i>": check block C (1|2), data
# block Q (1..5), trinomial letter t and term index i (1-based, in the order the
# trinomials are printed in Table 3).  The Z-check table prints inverse
# monomials as frame labels; the edges are those of the named term.
# ---------------------------------------------------------------------------
X_LAYERS = {
    "ZSZ-LP-160": ["11a1 22a1", "13b1 24b1", "15c1", "11a2 25d1", "22a2", "15c2 22a3", "15c3 24b2",
                   "24b3", "11a3", "13b2 25d2", "13b3 25d3"],
    "ZSZ-LP-240": ["11a1 22a1", "13b1 24b1", "13b2 24b2", "13b3 24b3", "11a3 22a3", "11a2 22a2",
                   "15c1", "15c2", "15c3", "25d1", "25d3", "25d2"],
    "ZSZ-LP-320": ["11a1 22a1", "13b1 24b1", "15c1", "11a3 25d1", "13b2 22a3", "11a2 24b2",
                   "13b3 22a2", "24b3", "15c2", "15c3", "25d2", "25d3"],
    "ZSZ-LP-390": ["11a1 22a1", "13b1 24b1", "15c1", "13b3 25d1", "11a2 24b3", "11a3 22a2",
                   "13b2 22a3", "24b2", "15c2", "15c3", "25d2", "25d3"],
    "ZSZ-LP-550": ["11a1 22a1", "13b1 24b1", "15c1", "11a3 25d1", "13b3 22a3", "11a2 24b3",
                   "13b2 22a2", "24b2", "15c3", "15c2", "25d3", "25d2"],
}
Z_LAYERS = {
    "ZSZ-LP-160": ["11c1 23c1", "12d1 24d1", "15a1", "11c2 25b1", "11c3 23c2", "12d3 23c3",
                   "12d2 24d3", "24d2", "15a2", "15a3", "25b2", "25b3"],
    "ZSZ-LP-240": ["11c1 23c1", "12d1 24d1", "15a1", "12d3 25b1", "11c2 24d3", "11c3 23c2",
                   "12d2 23c3", "24d2", "15a3", "15a2", "25b2", "25b3"],
    "ZSZ-LP-320": ["11c1 23c1", "12d1 24d1", "15a1", "15a3", "25b1", "12d2 25b2", "11c3",
                   "11c2 24d2", "12d3 23c3", "23c2", "15a2 24d3", "25b3"],
    "ZSZ-LP-390": ["11c1 23c1", "12d1 24d1", "15a1", "12d2 25b1", "11c3 24d2", "12d3",
                   "11c2 25b3", "25b2", "15a2", "15a3 23c2", "24d3", "23c3"],
    "ZSZ-LP-550": ["11c1 23c1", "12d1 24d1", "15a1", "15a3", "15a2", "25b1", "11c3 25b3",
                   "12d3 25b2", "11c2", "12d2 23c3", "24d3", "23c2", "24d2"],
}

# Codes without a Table 10 entry (the small test codes) use a plain order: one
# term per layer, check block 2 deferring its Q5 terms by three layers so that
# no layer touches a data qubit twice.  Not from the paper.
_DEFAULT_X = ["11a1 22a1", "11a2 22a2", "11a3 22a3", "13b1 24b1", "13b2 24b2", "13b3 24b3",
              "15c1", "15c2", "15c3", "25d1", "25d2", "25d3"]
_DEFAULT_Z = ["11c1 23c1", "11c2 23c2", "11c3 23c3", "12d1 24d1", "12d2 24d2", "12d3 24d3",
              "15a1", "15a2", "15a3", "25b1", "25b2", "25b3"]

# Which matrix block sits at (check block, data block) -- Eq. (5-block H_X, H_Z).
_X_BLOCK = {(1, 1): "A", (2, 2): "A", (1, 3): "B", (2, 4): "B", (1, 5): "CT", (2, 5): "DT"}
_Z_BLOCK = {(1, 1): "C", (1, 2): "D", (2, 3): "C", (2, 4): "D", (1, 5): "AT", (2, 5): "BT"}


def _layer_pairs(code: ZSZLPCode, tokens: str, kind: str):
    """(check qubit index within the check type, data qubit index) pairs."""
    l = code.ell
    blockmap = _X_BLOCK if kind == "X" else _Z_BLOCK
    checks, datas = [], []
    for tok in tokens.split():
        cb, qb, letter, ti = int(tok[0]), int(tok[1]), tok[2], int(tok[3:]) - 1
        blk = blockmap[(cb, qb)]
        if blk[0].lower() != letter:
            raise ValueError(f"token {tok} does not match block {blk}")
        c, dq = code.term_edges(blk, ti)
        checks.append(c + (cb - 1) * l)
        datas.append(dq + (qb - 1) * l)
    return np.concatenate(checks), np.concatenate(datas)


# ---------------------------------------------------------------------------
# Circuit representation
# ---------------------------------------------------------------------------
@dataclass
class Circuit:
    """Ops: ("R", qubits, basis), ("CX", ctrl, tgt), ("M", qubits, basis, keep)."""
    n_qubits: int
    ops: list = field(default_factory=list)
    n_kept: int = 0


def memory_circuit(code: ZSZLPCode, rounds: int, basis: str) -> tuple[Circuit, dict]:
    """d-round memory experiment (Sec. 6.1) with the Table 10 gate order."""
    name = code.name
    l, n = code.ell, code.n
    data = np.arange(n)
    anc_x = n + np.arange(2 * l)
    anc_z = n + 2 * l + np.arange(2 * l)
    circ = Circuit(n_qubits=n + 4 * l)
    xl = [_layer_pairs(code, t, "X") for t in X_LAYERS.get(name, _DEFAULT_X)]
    zl = [_layer_pairs(code, t, "Z") for t in Z_LAYERS.get(name, _DEFAULT_Z)]
    for c, dq in xl + zl:
        if len(np.unique(c)) != len(c) or len(np.unique(dq)) != len(dq):
            raise ValueError("a CNOT layer touches a qubit twice")
    keep_rounds = []   # kept record index of each memory-type ancilla measurement
    circ.ops.append(("R", data, basis))
    for _ in range(rounds):
        circ.ops.append(("R", anc_x, "X"))
        for c, dq in xl:
            circ.ops.append(("CX", anc_x[c], data[dq]))
        circ.ops.append(("M", anc_x, "X", basis == "X"))
        if basis == "X":
            keep_rounds.append(circ.n_kept + np.arange(2 * l))
            circ.n_kept += 2 * l
        circ.ops.append(("R", anc_z, "Z"))
        for c, dq in zl:
            circ.ops.append(("CX", data[dq], anc_z[c]))
        circ.ops.append(("M", anc_z, "Z", basis == "Z"))
        if basis == "Z":
            keep_rounds.append(circ.n_kept + np.arange(2 * l))
            circ.n_kept += 2 * l
    circ.ops.append(("M", data, basis, True))
    final = circ.n_kept + np.arange(n)
    circ.n_kept += n
    H = code.H_Z if basis == "Z" else code.H_X
    logical = code.logicals_Z if basis == "Z" else code.logicals_X
    det = []
    for r in range(rounds):
        for i in range(2 * l):
            det.append([keep_rounds[r][i]] if r == 0 else [keep_rounds[r][i], keep_rounds[r - 1][i]])
    for i in range(2 * l):
        det.append([keep_rounds[-1][i]] + list(final[np.nonzero(H[i])[0]]))
    obs = [list(final[np.nonzero(row)[0]]) for row in logical]
    return circ, dict(detectors=det, observables=obs)


def _count_faults(circ: Circuit) -> int:
    nf = 0
    for op in circ.ops:
        if op[0] == "R" or op[0] == "M":
            nf += len(op[1])
        else:
            nf += 15 * len(op[1])
    return nf


# The 15 non-identity two-qubit Paulis as (x_c, z_c, x_t, z_t) bits.
_PAULI2 = [(xc, zc, xt, zt) for xc in (0, 1) for zc in (0, 1) for xt in (0, 1) for zt in (0, 1)
           if (xc, zc, xt, zt) != (0, 0, 0, 0)]


def _frame_sim(circ: Circuit, p: float, f0: int, f1: int):
    """Propagate one Pauli frame per fault component in [f0, f1).

    Returns (kept measurement flip records [n_kept, W] uint64, fault probs).
    Bit f-f0 of a record row is set iff fault f flips that measurement.
    """
    nf = f1 - f0
    W = (nf + 63) // 64
    nq = circ.n_qubits
    X = np.zeros((nq, W), dtype=np.uint64)
    Z = np.zeros((nq, W), dtype=np.uint64)
    rec = np.zeros((circ.n_kept, W), dtype=np.uint64)
    probs = np.zeros(nf, dtype=np.float64)
    base = 0
    kept = 0

    def in_chunk(ids):
        m = (ids >= f0) & (ids < f1)
        return m, ids[m] - f0

    def flip(arr, qubits, local):
        words = (local // 64).astype(np.int64)
        bits = np.left_shift(np.uint64(1), (local % 64).astype(np.uint64))
        np.bitwise_xor.at(arr, (qubits, words), bits)

    for op in circ.ops:
        kind = op[0]
        if kind == "R":
            q = op[1]
            X[q] = 0
            Z[q] = 0
            ids = base + np.arange(len(q))
            m, local = in_chunk(ids)
            flip(X if op[2] == "Z" else Z, q[m], local)      # |1> for |0>, |-> for |+>
            probs[local] = p
            base += len(q)
        elif kind == "CX":
            c, t = op[1], op[2]
            X[t] ^= X[c]
            Z[c] ^= Z[t]
            npair = len(c)
            for k, (xc, zc, xt, zt) in enumerate(_PAULI2):
                ids = base + k * npair + np.arange(npair)
                m, local = in_chunk(ids)
                if not m.any():
                    continue
                if xc:
                    flip(X, c[m], local)
                if zc:
                    flip(Z, c[m], local)
                if xt:
                    flip(X, t[m], local)
                if zt:
                    flip(Z, t[m], local)
                probs[local] = p / 15.0
            base += 15 * npair
        else:  # "M"
            q, mb, keep = op[1], op[2], op[3]
            ids = base + np.arange(len(q))
            m, local = in_chunk(ids)
            probs[local] = p
            if keep:
                rows = kept + np.arange(len(q))
                rec[rows] = X[q] if mb == "Z" else Z[q]
                flip(rec, rows[m], local)
                kept += len(q)
            base += len(q)
    return rec, probs


@dataclass
class DEM:
    """Detector error model in the layouts the decoder takes.

    H_indptr/H_indices: CSR of the detector x fault matrix (rows = detectors).
    O_indptr/O_indices: CSR of the observable x fault matrix.
    priors: fault probabilities (float64), one per column.
    """
    name: str
    n_det: int
    n_loc: int
    n_obs: int
    H_indptr: np.ndarray
    H_indices: np.ndarray
    O_indptr: np.ndarray
    O_indices: np.ndarray
    priors: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.H_indices.size)

    def dense_H(self) -> np.ndarray:
        M = np.zeros((self.n_det, self.n_loc), dtype=np.uint8)
        for i in range(self.n_det):
            M[i, self.H_indices[self.H_indptr[i]:self.H_indptr[i + 1]]] = 1
        return M

    def dense_O(self) -> np.ndarray:
        M = np.zeros((self.n_obs, self.n_loc), dtype=np.uint8)
        for i in range(self.n_obs):
            M[i, self.O_indices[self.O_indptr[i]:self.O_indptr[i + 1]]] = 1
        return M

    def with_priors(self, priors: np.ndarray) -> "DEM":
        return DEM(self.name, self.n_det, self.n_loc, self.n_obs, self.H_indptr, self.H_indices,
                   self.O_indptr, self.O_indices, np.asarray(priors, dtype=np.float64), dict(self.meta))


def _csr_from_cols(cols: list[tuple], nrows: int) -> tuple[np.ndarray, np.ndarray]:
    """CSR (rows x len(cols)) from per-column sorted row lists."""
    rr, cc = [], []
    for j, rows in enumerate(cols):
        rr.extend(rows)
        cc.extend([j] * len(rows))
    rr = np.asarray(rr, dtype=np.int64)
    cc = np.asarray(cc, dtype=np.int64)
    order = np.lexsort((cc, rr))
    rr, cc = rr[order], cc[order]
    indptr = np.zeros(nrows + 1, dtype=np.int64)
    np.add.at(indptr, rr + 1, 1)
    indptr = np.cumsum(indptr)
    return indptr.astype(np.int32), cc.astype(np.int32)


def _set_bits_by_fault(R: np.ndarray, nloc: int) -> tuple[np.ndarray, np.ndarray]:
    """(fault, row) pairs of the set bits of a [rows, words] bit matrix whose bit
    f of a row means fault f flips it, sorted by fault then row."""
    rows, wi = np.nonzero(R)
    if rows.size == 0:
        return np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.int64)
    bits = np.unpackbits(np.ascontiguousarray(R[rows, wi]).view(np.uint8).reshape(-1, 8), axis=1,
                         bitorder="little")
    k, b = np.nonzero(bits)
    fault = wi[k].astype(np.int64) * 64 + b
    row = rows[k].astype(np.int64)
    keep = fault < nloc
    fault, row = fault[keep], row[keep]
    order = np.lexsort((row, fault))
    return fault[order], row[order]


def detector_rounds(dem) -> np.ndarray:
    """Round of each detector of a d-round memory DEM: the 2l detectors of
    round r (0 <= r < d) come r-th, the final data-readout detectors form round
    d (Table 5: N_det = 2 l (d + 1))."""
    rounds = int(dem.meta["rounds"])
    per, rem = divmod(dem.n_det, rounds + 1)
    if rem:
        raise ValueError(f"{dem.n_det} detectors do not split into {rounds + 1} equal rounds")
    return (np.arange(dem.n_det) // per).astype(np.int32)


def circuit_dem(code_name: str, p: float, rounds: int | None = None, basis: str = "Z",
                chunk: int = 1 << 17) -> DEM:
    """Circuit-level DEM of a d-round memory experiment (Sec. 6.1, App. E).

    Columns appear in the order of the first fault component that produces
    them; merged probabilities accumulate in that order.
    """
    return circuit_dems(code_name, [p], rounds, basis, chunk)[0]


def circuit_dems(code_name: str, ps, rounds: int | None = None, basis: str = "Z",
                 chunk: int = 1 << 17) -> list[DEM]:
    """circuit_dem for several noise strengths p, sharing one frame simulation
    (the detector structure does not depend on p; only the merged
    probabilities do)."""
    code = load_code(code_name)
    rounds = code.d if rounds is None else rounds
    circ, info = memory_circuit(code, rounds, basis)
    nf = _count_faults(circ)
    det_rows, obs_rows = info["detectors"], info["observables"]
    n_det, n_obs = len(det_rows), len(obs_rows)
    # two independent 64-bit random keys per detector / observable: a fault's
    # 128-bit signature is the XOR of its keys (set identity with collision
    # probability ~ n^2 / 2^128)
    rng = np.random.default_rng(0x5EED_DE11)
    kd = rng.integers(0, 2 ** 63, size=(2, n_det), dtype=np.int64).astype(np.uint64) * np.uint64(2) + np.uint64(1)
    ko = rng.integers(0, 2 ** 63, size=(2, max(1, n_obs)), dtype=np.int64).astype(np.uint64) * np.uint64(2)
    sig_all, first_dets, first_obs, probs_all = [], [], [], []
    for f0 in range(0, nf, chunk):
        f1 = min(nf, f0 + chunk)
        rec, probs = _frame_sim(circ, 1.0, f0, f1)     # unit strength: scaled per p below
        D = np.zeros((n_det, rec.shape[1]), dtype=np.uint64)
        for i, rows in enumerate(det_rows):
            D[i] = np.bitwise_xor.reduce(rec[rows], axis=0)
        O = np.zeros((n_obs, rec.shape[1]), dtype=np.uint64)
        for i, rows in enumerate(obs_rows):
            O[i] = np.bitwise_xor.reduce(rec[rows], axis=0)
        nloc = f1 - f0
        fd, dd = _set_bits_by_fault(D, nloc)
        fo, oo = _set_bits_by_fault(O, nloc)
        sig = np.zeros((nloc, 2), dtype=np.uint64)
        for t in range(2):
            np.bitwise_xor.at(sig[:, t], fd, kd[t][dd])
            if n_obs:
                np.bitwise_xor.at(sig[:, t], fo, ko[t][oo])
        hit = np.zeros(nloc, dtype=bool)
        hit[fd] = True
        hit[fo] = True
        nz = np.nonzero(hit)[0]
        dstart = np.searchsorted(fd, np.arange(nloc + 1))
        ostart = np.searchsorted(fo, np.arange(nloc + 1))
        sig_all.append(sig[nz])
        probs_all.append(probs[nz])
        first_dets.append([(dd[dstart[f]:dstart[f + 1]], oo[ostart[f]:ostart[f + 1]]) for f in nz])
    sig = np.concatenate(sig_all)
    probs = np.concatenate(probs_all)
    sets = [x for chunk_sets in first_dets for x in chunk_sets]
    _, first, inv = np.unique(sig, axis=0, return_index=True, return_inverse=True)
    inv = inv.reshape(-1)
    order = np.argsort(first, kind="stable")          # groups by first occurrence
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    col = rank[inv]
    ncol = order.size
    reps = first[order]
    col_dets = [tuple(sets[r][0].tolist()) for r in reps]
    col_obs = [tuple(sets[r][1].tolist()) for r in reps]
    for f in range(0, col.size, max(1, col.size // 2000)):   # spot-check set identity within groups
        r = reps[col[f]]
        if not (np.array_equal(sets[f][0], sets[r][0]) and np.array_equal(sets[f][1], sets[r][1])):
            raise RuntimeError("signature collision while merging fault mechanisms")
    Hp, Hi = _csr_from_cols(col_dets, n_det)
    Op, Oi = _csr_from_cols(col_obs, n_obs)
    out = []
    for p in ps:
        # component probabilities at strength p: p for resets and measurements,
        # p/15 for each two-qubit Pauli (the unit-strength values times p)
        pr = np.where(probs == 1.0, p, p / 15.0)     # unit strength marks p (1.0) or p/15 (1/15)
        col_p = np.zeros(ncol, dtype=np.float64)
        seen = np.zeros(ncol, dtype=bool)
        for f in range(col.size):                     # p <- p1 + p2 - 2 p1 p2, in fault order
            j = col[f]
            if seen[j]:
                q = col_p[j]
                col_p[j] = q + pr[f] - 2.0 * q * pr[f]
            else:
                col_p[j] = pr[f]
                seen[j] = True
        out.append(DEM(f"{code_name}/circuit/d{rounds}/{basis}/p{p:g}", n_det, ncol, n_obs, Hp, Hi, Op, Oi, col_p,
                       dict(code=code_name, rounds=rounds, basis=basis, p=p, n_fault_components=nf)))
    return out


def code_capacity_dem(code_name: str, p: float) -> DEM:
    """Code-capacity model: i.i.d. Z errors on the data, syndrome H_X e.

    Failure is judged by the X-type logicals (ker H_Z modulo rs H_X).
    """
    code = load_code(code_name)
    H = code.H_X
    L = code.logicals_X
    Hp, Hi = _dense_to_csr(H)
    Op, Oi = _dense_to_csr(L)
    return DEM(f"{code_name}/code-capacity/p{p:g}", H.shape[0], H.shape[1], L.shape[0], Hp, Hi, Op, Oi,
               np.full(H.shape[1], p, dtype=np.float64), dict(code=code_name, p=p))


def _dense_to_csr(M: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    indptr = np.zeros(M.shape[0] + 1, dtype=np.int32)
    idx = []
    for i in range(M.shape[0]):
        nz = np.nonzero(M[i])[0]
        idx.append(nz)
        indptr[i + 1] = indptr[i] + nz.size
    return indptr, (np.concatenate(idx) if idx else np.zeros(0)).astype(np.int32)


def dem_from_dense(H: np.ndarray, priors: np.ndarray, O: np.ndarray | None = None, name: str = "dense") -> DEM:
    """DEM from dense matrices (small synthetic instances)."""
    if O is None:
        O = np.zeros((0, H.shape[1]), dtype=np.uint8)
    Hp, Hi = _dense_to_csr(H)
    Op, Oi = _dense_to_csr(O)
    return DEM(name, H.shape[0], H.shape[1], O.shape[0], Hp, Hi, Op, Oi, np.asarray(priors, dtype=np.float64))
