"""Host logic of the gamma-interval grid search and LER sweeps, run end to end
on the CPU with the oracle standing in for the GPU decoder (small code)."""
import numpy as np
import pytest

import oracle
from oracle import DecodeParams
from paper_2607_27644_b300.stats import clopper_pearson, per_qubit_round
from paper_2607_27644_b300.sweep import Tally, gamma_grid_search, ler_curve, ler_point
from workloads.dem import circuit_dems
from workloads.zsz import load_code


class OracleDecoder:
    """The sweep's decoder interface over the FP64 oracle."""

    def __init__(self):
        self.calls = 0

    def run(self, dem, params, shots, shot0=0):
        self.calls += 1
        syn, obs, _ = oracle.sample(dem, 2, shot0, shots)
        r = oracle.decode(dem, params, syn, shot0=shot0)
        conv = r["stats"][:, 0] == 1
        wrong = np.any(r["pred_obs"][:, :obs.shape[1]] != obs, axis=1)
        return Tally(shots, int((~conv).sum() + (conv & wrong).sum()), int((~conv).sum()), int((conv & wrong).sum()))


P_LO, P_HI = 0.003, 0.01
KW = dict(gamma0=0.125, pre_iter=30, num_sets=4, max_iterations=20, stop_nconv=2, seed=5)
N = 150


@pytest.fixture(scope="module")
def dems60():
    zs = circuit_dems("ZSZ-LP-60", [P_LO, P_HI], 2, "Z")
    xs = circuit_dems("ZSZ-LP-60", [P_LO, P_HI], 2, "X")
    return {P_LO: {"Z": zs[0], "X": xs[0]}, P_HI: {"Z": zs[1], "X": xs[1]}}


def test_ler_point_statistics(dems60):
    k = load_code("ZSZ-LP-60").k
    pt = ler_point(OracleDecoder(), dems60[P_LO], DecodeParams(gamma_min=-0.24, gamma_max=0.66, **KW), N,
                   P_LO, 2, k)
    z, x = pt.per_basis["Z"], pt.per_basis["X"]
    assert z.shots == x.shots == N and z.failures == z.nonconverged + z.logical
    assert pt.block == pytest.approx((z.failures + x.failures) / (2 * N))
    assert pt.per_qubit_round == pytest.approx(per_qubit_round(pt.block, 2, k))
    lo, hi = clopper_pearson(z.failures + x.failures, 2 * N)
    assert pt.block_ci() == (lo, hi) and lo <= pt.block <= hi
    qlo, qhi = pt.per_qubit_round_ci()
    assert qlo <= pt.per_qubit_round <= qhi
    assert pt.as_dict()["per_basis"]["Z"]["failures"] == z.failures


def test_gamma_grid_search_picks_the_fewest_failures(dems60):
    dec = OracleDecoder()
    k = load_code("ZSZ-LP-60").k
    base = DecodeParams(**KW)
    best, pts = gamma_grid_search(dec, dems60[P_LO], base, [-0.24, 0.0, 0.5], [0.3, 0.66], N, P_LO, 2, k)
    grid = [(a, b) for a in (-0.24, 0.0, 0.5) for b in (0.3, 0.66) if a < b]
    assert [p.gamma for p in pts] == grid and dec.calls == 2 * len(grid)
    assert best.pooled.failures == min(p.pooled.failures for p in pts)
    assert best is next(p for p in pts if p.pooled.failures == best.pooled.failures)
    assert any(p.pooled.failures > 0 for p in pts)
    # the same shots decode to the same tally (counter-based draws)
    again = ler_point(OracleDecoder(), dems60[P_LO], DecodeParams(gamma_min=best.gamma[0], gamma_max=best.gamma[1],
                                                                   **KW), N, P_LO, 2, k)
    assert vars(again.pooled) == vars(best.pooled)
    with pytest.raises(ValueError):
        gamma_grid_search(dec, dems60[P_LO], base, [0.5], [0.3], 10, P_LO, 2, k)


def test_ler_curve_grows_with_p(dems60):
    k = load_code("ZSZ-LP-60").k
    pts = ler_curve(OracleDecoder(), dems60, DecodeParams(gamma_min=-0.24, gamma_max=0.66, **KW), N, 2, k)
    assert [p.p for p in pts] == [P_LO, P_HI]
    assert pts[1].pooled.failures > pts[0].pooled.failures
    assert pts[1].per_qubit_round > pts[0].per_qubit_round
