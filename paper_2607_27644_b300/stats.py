"""Logical-error-rate statistics (host side).

arXiv 2607.27644, Sec. 6.1: for a raw block LER p over T rounds the per-round
rate is 1 - (1 - p)^(1/T), and the per-qubit-round rate replaces T by T*k;
error bars are 95% Clopper-Pearson intervals (Fig. 6 caption).
"""
from __future__ import annotations

import math

from scipy.stats import beta


def per_round(p_block: float, rounds: int) -> float:
    return 1.0 - (1.0 - p_block) ** (1.0 / rounds)


def per_qubit_round(p_block: float, rounds: int, k: int) -> float:
    return per_round(p_block, rounds * k)


def clopper_pearson(failures: int, shots: int, level: float = 0.95) -> tuple[float, float]:
    a = 1.0 - level
    lo = 0.0 if failures == 0 else float(beta.ppf(a / 2, failures, shots - failures + 1))
    hi = 1.0 if failures == shots else float(beta.ppf(1 - a / 2, failures + 1, shots - failures))
    return lo, hi


def binomial_sigma(failures: int, shots: int) -> float:
    p = failures / shots
    return math.sqrt(max(p * (1 - p), 1.0 / shots) / shots)


def agree_within(f1: int, n1: int, f2: int, n2: int, nsigma: float = 2.0) -> bool:
    """Two binomial rates agree within nsigma combined standard errors."""
    s = math.hypot(binomial_sigma(f1, n1), binomial_sigma(f2, n2))
    return abs(f1 / n1 - f2 / n2) <= nsigma * s
