"""Stabilizer-tableau simulator for test cross-checks.

Written from the published CHP algorithm (S. Aaronson and D. Gottesman,
"Improved simulation of stabilizer circuits", Phys. Rev. A 70, 052328 (2004)):
a tableau of n destabilizer rows, n stabilizer rows and one scratch row, each
an n-qubit Pauli (x bits, z bits) with a sign bit; Hadamard and CNOT update
columns, Pauli gates flip the signs of anticommuting rows, and a Z measurement
is random when some stabilizer anticommutes with Z_q (then the tableau is
updated by row products) and deterministic otherwise (the outcome is the sign
of the product of the stabilizers whose destabilizers anticommute with Z_q).

It simulates the memory circuits of workloads/dem.py gate by gate, a
computation independent of the Pauli-frame propagation that builds the DEMs.
"""
from __future__ import annotations

import numpy as np


class Tableau:
    def __init__(self, n: int, rng: np.random.Generator):
        self.n = n
        self.x = np.zeros((2 * n + 1, n), dtype=np.uint8)
        self.z = np.zeros((2 * n + 1, n), dtype=np.uint8)
        self.r = np.zeros(2 * n + 1, dtype=np.uint8)
        idx = np.arange(n)
        self.x[idx, idx] = 1            # destabilizer i = X_i
        self.z[n + idx, idx] = 1        # stabilizer i = Z_i: the state |0...0>
        self.rng = rng

    # -- gates (q, c, t: index arrays of distinct qubits) --------------------
    def h(self, q):
        x, z = self.x, self.z
        self.r ^= np.bitwise_xor.reduce(x[:, q] & z[:, q], axis=1)
        xq = x[:, q].copy()
        x[:, q] = z[:, q]
        z[:, q] = xq

    def cx(self, c, t):
        x, z = self.x, self.z
        self.r ^= np.bitwise_xor.reduce(x[:, c] & z[:, t] & (x[:, t] ^ z[:, c] ^ 1), axis=1)
        x[:, t] ^= x[:, c]
        z[:, c] ^= z[:, t]

    def pauli(self, q: int, px: int, pz: int):
        """Apply X^px Z^pz to qubit q: rows that anticommute change sign."""
        if px:
            self.r ^= self.z[:, q]
        if pz:
            self.r ^= self.x[:, q]

    # -- row products ------------------------------------------------------------
    def _rowsum(self, hs, i: int):
        """Rows hs <- rows hs times row i, with the phase of the product."""
        x1 = self.x[i].astype(np.int64)
        z1 = self.z[i].astype(np.int64)
        x2 = self.x[hs].astype(np.int64)
        z2 = self.z[hs].astype(np.int64)
        g = np.where((x1 == 1) & (z1 == 1), z2 - x2,
                     np.where((x1 == 1) & (z1 == 0), z2 * (2 * x2 - 1),
                              np.where((x1 == 0) & (z1 == 1), x2 * (1 - 2 * z2), 0)))
        tot = 2 * self.r[hs].astype(np.int64) + 2 * int(self.r[i]) + g.sum(axis=1)
        self.r[hs] = ((tot % 4) // 2).astype(np.uint8)
        self.x[hs] ^= self.x[i]
        self.z[hs] ^= self.z[i]

    # -- measurement and reset ---------------------------------------------------
    def measure_z(self, q: int) -> int:
        n = self.n
        anti = np.nonzero(self.x[n:2 * n, q])[0]
        if anti.size:                                   # random outcome
            p = n + int(anti[0])
            rows = np.nonzero(self.x[:2 * n, q])[0]
            rows = rows[rows != p]
            if rows.size:
                self._rowsum(rows, p)
            self.x[p - n] = self.x[p]
            self.z[p - n] = self.z[p]
            self.r[p - n] = self.r[p]
            self.x[p] = 0
            self.z[p] = 0
            self.z[p, q] = 1
            m = int(self.rng.integers(2))
            self.r[p] = m
            return m
        s = 2 * n                                       # deterministic: scratch row
        self.x[s] = 0
        self.z[s] = 0
        self.r[s] = 0
        for i in np.nonzero(self.x[:n, q])[0]:
            self._rowsum(np.array([s]), n + int(i))
        return int(self.r[s])

    def measure(self, q: int, basis: str) -> int:
        if basis == "Z":
            return self.measure_z(q)
        self.h(np.array([q]))
        m = self.measure_z(q)
        self.h(np.array([q]))
        return m

    def reset(self, q: int, basis: str):
        if self.measure_z(q):
            self.pauli(q, 1, 0)
        if basis == "X":
            self.h(np.array([q]))


# The 15 non-identity two-qubit Paulis (x_c, z_c, x_t, z_t) in the order the
# DEM builder numbers a CNOT layer's fault components.
PAULI2 = [(xc, zc, xt, zt) for xc in (0, 1) for zc in (0, 1) for xt in (0, 1) for zt in (0, 1)
          if (xc, zc, xt, zt) != (0, 0, 0, 0)]


def run_memory_circuit(circ, info, fault: int | None, seed: int):
    """Simulate a workloads.dem memory circuit with at most one fault component
    (numbered like the DEM builder: resets, then the 15 components of each
    CNOT pair after its layer, then measurement flips, in op order).
    Returns (detector bits, observable bits)."""
    rng = np.random.default_rng(seed)
    tab = Tableau(circ.n_qubits, rng)
    rec = []
    base = 0
    for op in circ.ops:
        kind = op[0]
        if kind == "R":
            q, basis = op[1], op[2]
            for qq in q:
                tab.reset(int(qq), basis)
            if fault is not None and base <= fault < base + len(q):
                qq = int(q[fault - base])
                tab.pauli(qq, 1, 0) if basis == "Z" else tab.pauli(qq, 0, 1)
            base += len(q)
        elif kind == "CX":
            c, t = op[1], op[2]
            tab.cx(c, t)
            npair = len(c)
            if fault is not None and base <= fault < base + 15 * npair:
                k, j = divmod(fault - base, npair)
                xc, zc, xt, zt = PAULI2[k]
                tab.pauli(int(c[j]), xc, zc)
                tab.pauli(int(t[j]), xt, zt)
            base += 15 * npair
        else:
            q, basis, keep = op[1], op[2], op[3]
            out = [tab.measure(int(qq), basis) for qq in q]
            if fault is not None and base <= fault < base + len(q):
                out[fault - base] ^= 1
            if keep:
                rec.extend(out)
            base += len(q)
    rec = np.array(rec, dtype=np.uint8)
    det = np.array([int(np.bitwise_xor.reduce(rec[d])) for d in info["detectors"]], dtype=np.uint8)
    obs = np.array([int(np.bitwise_xor.reduce(rec[o])) for o in info["observables"]], dtype=np.uint8)
    return det, obs
