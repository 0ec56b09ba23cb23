"""ZSZ group algebra and the five-block ZSZ-LP codes (seeded input generator).

This module builds the parity-check matrices that every decoding workload
starts from.  It holds none of the decoder's arithmetic: the CUDA path and the
CPU oracle both take its matrices as plain inputs.

Paper references (arXiv 2607.27644):
  * Sec. 2.2, Eq. (ZSZ presentation) and the push-through relations: the group
    Z_l1 x|_q Z_l2 with canonical elements x^a y^b and
    (x^i y^j)(x^a y^b) = x^(i + q^j a) y^(j + b).
  * App. B, Eq. (regular representation): L[g]|h> = |gh>, R[g]|h> = |hg>;
    element x^a y^b is indexed a*l2 + b (App. C, "Equivariant codewords").
  * Sec. 2.3, Eq. (H_left, H_right): H_left = (L[a] L[b]), H_right = (R[c] R[d]).
  * Sec. 2.1 / 2.4, Eq. (5-block H_X, H_Z) with A=L[a], B=L[b], C=R[c], D=R[d].
  * Table 3 (trinomials per code), Table 13 (additional frontier codes),
    Table 1 (n, k, d).
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import cached_property

import numpy as np


# ---------------------------------------------------------------------------
# Group arithmetic (Sec. 2.2)
# ---------------------------------------------------------------------------
class ZSZGroup:
    """Z_{l1} x|_q Z_{l2}: elements x^a y^b stored as index a*l2 + b."""

    def __init__(self, l1: int, l2: int, q: int):
        if pow(q, l2, l1) != 1 % l1:
            raise ValueError(f"q^l2 != 1 mod l1 for (l1,l2,q)=({l1},{l2},{q})")
        self.l1, self.l2, self.q = l1, l2, q
        self.order = l1 * l2
        n = self.order
        a = np.arange(n) // l2
        b = np.arange(n) % l2
        qpow = np.array([pow(q, j, l1) for j in range(l2)], dtype=np.int64)
        # (x^i y^j)(x^al y^be) = x^(i + q^j al) y^(j + be)
        i, j = a[:, None], b[:, None]
        al, be = a[None, :], b[None, :]
        ra = (i + qpow[j] * al) % l1
        rb = (j + be) % l2
        self.mul = (ra * l2 + rb).astype(np.int64)          # mul[g, h] = g*h
        ident = 0
        self.inv = np.argmax(self.mul == ident, axis=1).astype(np.int64)
        assert np.all(self.mul[np.arange(n), self.inv] == ident)

    def elem(self, a: int, b: int) -> int:
        return (a % self.l1) * self.l2 + (b % self.l2)

    def exps(self, g: int) -> tuple[int, int]:
        return g // self.l2, g % self.l2

    def element_order(self, g: int) -> int:
        h, k = g, 1
        while h != 0:
            h = int(self.mul[h, g])
            k += 1
        return k

    def center(self) -> list[int]:
        n = self.order
        return [g for g in range(n) if np.array_equal(self.mul[g, :], self.mul[:, g])]


# ---------------------------------------------------------------------------
# Group-algebra elements and regular representations (App. B)
# ---------------------------------------------------------------------------
def monomials(G: ZSZGroup, terms) -> list[int]:
    """Parse a list of (a, b) exponent pairs into group-element indices."""
    return [G.elem(a, b) for (a, b) in terms]


def L_mat(G: ZSZGroup, poly: list[int]) -> np.ndarray:
    """Left-regular representation: column h has a 1 at row g*h per monomial g."""
    n = G.order
    M = np.zeros((n, n), dtype=np.uint8)
    h = np.arange(n)
    for g in poly:
        M[G.mul[g, h], h] ^= 1
    return M


def R_mat(G: ZSZGroup, poly: list[int]) -> np.ndarray:
    """Right-regular representation: column h has a 1 at row h*g per monomial g."""
    n = G.order
    M = np.zeros((n, n), dtype=np.uint8)
    h = np.arange(n)
    for g in poly:
        M[G.mul[h, g], h] ^= 1
    return M


# ---------------------------------------------------------------------------
# GF(2) linear algebra (plain Gaussian elimination)
# ---------------------------------------------------------------------------
def gf2_rref(M: np.ndarray) -> tuple[np.ndarray, list[int]]:
    A = (np.array(M, dtype=np.uint8) & 1).copy()
    rows, cols = A.shape
    piv = []
    r = 0
    for c in range(cols):
        if r >= rows:
            break
        nz = np.nonzero(A[r:, c])[0]
        if nz.size == 0:
            continue
        p = r + nz[0]
        if p != r:
            A[[r, p]] = A[[p, r]]
        others = np.nonzero(A[:, c])[0]
        others = others[others != r]
        A[others] ^= A[r]
        piv.append(c)
        r += 1
    return A[:r], piv


def gf2_rank(M: np.ndarray) -> int:
    return len(gf2_rref(M)[1])


def gf2_nullspace(M: np.ndarray) -> np.ndarray:
    """Basis (rows) of {v : M v = 0} over GF(2)."""
    R, piv = gf2_rref(M)
    n = M.shape[1]
    free = [c for c in range(n) if c not in set(piv)]
    basis = np.zeros((len(free), n), dtype=np.uint8)
    for t, f in enumerate(free):
        basis[t, f] = 1
        for r, p in enumerate(piv):
            if R[r, f]:
                basis[t, p] = 1
    return basis


def logical_basis(H_comm: np.ndarray, H_stab: np.ndarray) -> np.ndarray:
    """Rows spanning ker(H_comm) modulo rs(H_stab).

    Z-type logicals: H_comm = H_X, H_stab = H_Z (Sec. 3, codeword embedding:
    logicals live in ker H minus the row space of the same-type checks).
    """
    K = gf2_nullspace(H_comm)
    base_rank = gf2_rank(H_stab)
    out = []
    cur = H_stab.copy()
    r = base_rank
    for v in K:
        trial = np.vstack([cur, v[None, :]])
        rt = gf2_rank(trial)
        if rt > r:
            out.append(v)
            cur, r = trial, rt
    return np.array(out, dtype=np.uint8).reshape(len(out), H_comm.shape[1])


# ---------------------------------------------------------------------------
# Code table (Table 3 and Table 13)
# ---------------------------------------------------------------------------
# Each trinomial as a list of (x exponent, y exponent) pairs, in the order the
# paper prints it (the order defines a_1, a_2, a_3 used by the gate schedule).
CODES = {
    "ZSZ-LP-160": dict(l1=16, l2=2, q=9, d=10,
                       a=[(0, 0), (13, 0), (14, 1)], b=[(0, 0), (3, 1), (13, 1)],
                       c=[(0, 0), (14, 0), (12, 1)], d_=[(0, 0), (7, 0), (11, 0)]),
    "ZSZ-LP-240": dict(l1=12, l2=4, q=7, d=12,
                       a=[(0, 0), (8, 1), (7, 2)], b=[(0, 0), (2, 0), (5, 1)],
                       c=[(0, 0), (4, 1), (2, 3)], d_=[(0, 0), (4, 0), (9, 0)]),
    "ZSZ-LP-320": dict(l1=16, l2=4, q=3, d=14,
                       a=[(0, 0), (1, 0), (0, 1)], b=[(0, 0), (2, 0), (13, 3)],
                       c=[(0, 0), (12, 1), (2, 3)], d_=[(0, 0), (12, 0), (11, 2)]),
    "ZSZ-LP-390": dict(l1=26, l2=3, q=3, d=16,
                       a=[(0, 0), (17, 1), (14, 2)], b=[(0, 0), (16, 0), (3, 1)],
                       c=[(0, 0), (24, 0), (8, 1)], d_=[(0, 0), (21, 0), (0, 1)]),
    "ZSZ-LP-550": dict(l1=22, l2=5, q=3, d=18,
                       a=[(0, 0), (10, 0), (5, 2)], b=[(0, 0), (8, 0), (2, 3)],
                       c=[(0, 0), (7, 0), (16, 1)], d_=[(0, 0), (1, 0), (6, 4)]),
    "ZSZ-LP-775": dict(l1=31, l2=5, q=2, d=22,
                       a=[(0, 0), (26, 2), (18, 3)], b=[(0, 0), (13, 2), (7, 4)],
                       c=[(0, 0), (1, 1), (28, 4)], d_=[(0, 0), (0, 1), (22, 2)]),
    # Table 13, first row: [[60,12,6]] over ZSZ_{3,4,2}; small enough for
    # brute-force checks.
    "ZSZ-LP-60": dict(l1=3, l2=4, q=2, d=6,
                      a=[(0, 0), (0, 3), (2, 3)], b=[(0, 0), (1, 0), (1, 2)],
                      c=[(0, 0), (0, 1), (1, 3)], d_=[(0, 0), (0, 2), (0, 3)]),
}


@dataclass
class ZSZLPCode:
    name: str
    l1: int
    l2: int
    q: int
    d: int
    a_terms: list
    b_terms: list
    c_terms: list
    d_terms: list

    @classmethod
    def from_table(cls, name: str) -> "ZSZLPCode":
        e = CODES[name]
        return cls(name, e["l1"], e["l2"], e["q"], e["d"], e["a"], e["b"], e["c"], e["d_"])

    @cached_property
    def G(self) -> ZSZGroup:
        return ZSZGroup(self.l1, self.l2, self.q)

    @property
    def ell(self) -> int:
        return self.l1 * self.l2

    @property
    def n(self) -> int:
        return 5 * self.ell

    def poly(self, which: str) -> list[int]:
        terms = {"a": self.a_terms, "b": self.b_terms, "c": self.c_terms, "d": self.d_terms}[which]
        return monomials(self.G, terms)

    @cached_property
    def A(self):
        return L_mat(self.G, self.poly("a"))

    @cached_property
    def B(self):
        return L_mat(self.G, self.poly("b"))

    @cached_property
    def C(self):
        return R_mat(self.G, self.poly("c"))

    @cached_property
    def D(self):
        return R_mat(self.G, self.poly("d"))

    @cached_property
    def H_left(self):
        return np.hstack([self.A, self.B])

    @cached_property
    def H_right(self):
        return np.hstack([self.C, self.D])

    @cached_property
    def H_X(self):
        l = self.ell
        Z = np.zeros((l, l), dtype=np.uint8)
        return np.block([[self.A, Z, self.B, Z, self.C.T], [Z, self.A, Z, self.B, self.D.T]]).astype(np.uint8)

    @cached_property
    def H_Z(self):
        l = self.ell
        Z = np.zeros((l, l), dtype=np.uint8)
        return np.block([[self.C, self.D, Z, Z, self.A.T], [Z, Z, self.C, self.D, self.B.T]]).astype(np.uint8)

    @cached_property
    def k(self) -> int:
        return self.n - gf2_rank(self.H_X) - gf2_rank(self.H_Z)

    @cached_property
    def logicals_Z(self) -> np.ndarray:
        """Z-type logical supports: ker H_X modulo rs H_Z (k rows)."""
        return logical_basis(self.H_X, self.H_Z)

    @cached_property
    def logicals_X(self) -> np.ndarray:
        """X-type logical supports: ker H_Z modulo rs H_X (k rows)."""
        return logical_basis(self.H_Z, self.H_X)

    # Tanner edges contributed by one monomial term of one block, used by the
    # syndrome-extraction schedule (App. E, Table 10).  Returns (check, data)
    # index pairs within the check block and data block, over all h in G.
    def term_edges(self, block: str, t: int) -> tuple[np.ndarray, np.ndarray]:
        G = self.G
        h = np.arange(self.ell)
        poly = self.poly(block[0].lower())
        g = poly[t]
        if block == "A" or block == "B":        # L[p]: data h -> check g h
            return G.mul[g, h], h
        if block == "C" or block == "D":        # R[p]: data h -> check h g
            return G.mul[h, g], h
        if block == "AT" or block == "BT":      # L[p]^T: check h -> data g h
            return h, G.mul[g, h]
        if block == "CT" or block == "DT":      # R[p]^T: check h -> data h g
            return h, G.mul[h, g]
        raise ValueError(block)


def load_code(name: str) -> ZSZLPCode:
    return ZSZLPCode.from_table(name)
