"""Relay-BP tuning and logical-error-rate sweeps over the decode path.

arXiv 2607.27644 tunes the memory-strength interval [gamma_min, gamma_max] of
Relay-BP per code by a grid search at one noise strength p_sweep, keeping the
interval with the lowest logical error rate (Sec. 6.1, Table 9), and reports
block LERs averaged over X- and Z-memory experiments, converted per round and
per qubit-round, with 95% Clopper-Pearson intervals (Sec. 6.1, Figs. 5-6).

This module orchestrates those experiments; the decoding itself runs in the
library's kernels through `GpuDecoder`.  Any object with the same `run`
method can stand in (the tests use one that calls the CPU oracle on small
codes).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

from .stats import clopper_pearson, per_qubit_round, per_round


@dataclass
class Tally:
    shots: int = 0
    failures: int = 0          # nonconverged or undetected logical error
    nonconverged: int = 0
    logical: int = 0

    def __add__(self, o: "Tally") -> "Tally":
        return Tally(self.shots + o.shots, self.failures + o.failures, self.nonconverged + o.nonconverged,
                     self.logical + o.logical)


class GpuDecoder:
    """Samples and decodes on the current CUDA device in batches through the
    C ABI (relaybp_sample, relaybp_decode_batch, relaybp_count_failures)."""

    def __init__(self, batch: int = 1 << 16, sample_seed: int = 2):
        self.batch = batch
        self.sample_seed = sample_seed

    def run(self, dem, params, shots: int, shot0: int = 0) -> Tally:
        import torch
        from . import relaybp as R
        h = R.relaybp_build_dem(dem, params)
        try:
            B = max(1, min(self.batch, shots))
            syn = torch.empty((B, h.wc), dtype=torch.int32, device="cuda")
            obs = torch.empty((B, h.wk), dtype=torch.int32, device="cuda")
            pobs = torch.empty((B, h.wk), dtype=torch.int32, device="cuda")
            stats = torch.empty((B, 6), dtype=torch.int32, device="cuda")
            cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
            done = 0
            while done < shots:
                n = min(B, shots - done)
                s0 = shot0 + done
                R.relaybp_sample(h, self.sample_seed, s0, n, syn, obs)
                R.relaybp_decode_batch(h, syn, s0, n, None, pobs, stats)
                R.relaybp_count_failures(h, pobs, obs, stats, n, cnt)
                done += n
            c = cnt.cpu().tolist()
        finally:
            R.relaybp_destroy(h)
        return Tally(int(c[0]), int(c[3]), int(c[1]), int(c[2]))


@dataclass
class LerPoint:
    """XZ-averaged logical error rates of one (code, p, decoder setting)."""
    p: float
    rounds: int
    k: int
    per_basis: dict = field(default_factory=dict)      # basis -> Tally
    gamma: tuple = (0.0, 0.0)

    @property
    def block(self) -> float:
        """Block LER averaged over the bases (equal shot counts)."""
        return sum(t.failures / t.shots for t in self.per_basis.values()) / len(self.per_basis)

    @property
    def pooled(self) -> Tally:
        out = Tally()
        for t in self.per_basis.values():
            out = out + t
        return out

    def block_ci(self, level: float = 0.95) -> tuple[float, float]:
        t = self.pooled
        return clopper_pearson(t.failures, t.shots, level)

    @property
    def per_round(self) -> float:
        return per_round(self.block, self.rounds)

    @property
    def per_qubit_round(self) -> float:
        return per_qubit_round(self.block, self.rounds, self.k)

    def per_qubit_round_ci(self, level: float = 0.95) -> tuple[float, float]:
        lo, hi = self.block_ci(level)
        return per_qubit_round(lo, self.rounds, self.k), per_qubit_round(hi, self.rounds, self.k)

    def as_dict(self) -> dict:
        lo, hi = self.per_qubit_round_ci()
        return {"p": self.p, "gamma": list(self.gamma), "rounds": self.rounds, "k": self.k,
                "per_basis": {b: vars(t) for b, t in self.per_basis.items()},
                "block_ler": self.block, "per_round": self.per_round, "per_qubit_round": self.per_qubit_round,
                "per_qubit_round_95": [lo, hi]}


def ler_point(decoder, dems: dict, params, shots: int, p: float, rounds: int, k: int,
              shot0: int = 0) -> LerPoint:
    """Decode `shots` shots of each basis' DEM (dems: basis -> DEM) with one
    parameter set; the bases use the same shot indices."""
    pt = LerPoint(p=p, rounds=rounds, k=k, gamma=(params.gamma_min, params.gamma_max))
    for basis, dem in sorted(dems.items()):
        pt.per_basis[basis] = decoder.run(dem, params, shots, shot0)
    return pt


def gamma_grid_search(decoder, dems: dict, params, gamma_mins, gamma_maxs, shots: int, p: float, rounds: int,
                      k: int, shot0: int = 0) -> tuple[LerPoint, list[LerPoint]]:
    """Table 9's tuning step: every interval [gmin, gmax] of the grid with
    gmin < gmax decodes the same shots of both memory experiments; returns the
    interval with the fewest pooled failures (the first in grid order on a
    tie) and every grid point."""
    points = []
    for gmin in gamma_mins:
        for gmax in gamma_maxs:
            if not gmin < gmax:
                continue
            pr = replace(params, gamma_min=float(gmin), gamma_max=float(gmax))
            points.append(ler_point(decoder, dems, pr, shots, p, rounds, k, shot0))
    if not points:
        raise ValueError("the grid holds no interval with gamma_min < gamma_max")
    best = min(points, key=lambda q: q.pooled.failures)
    return best, points


def ler_curve(decoder, dems_by_p: dict, params, shots: int, rounds: int, k: int, shot0: int = 0) -> list[LerPoint]:
    """XZ-averaged LER per qubit-round at each noise strength (dems_by_p:
    p -> {basis: DEM}), one decoder setting."""
    return [ler_point(decoder, dems_by_p[p], params, shots, p, rounds, k, shot0) for p in sorted(dems_by_p)]
