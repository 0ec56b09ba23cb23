"""Sliding-window decoding (commit region 1) over the FP64 oracle: the
procedure's own invariants, on the [[60,12,6]] circuit DEM."""
import numpy as np
import pytest

import oracle
from oracle import DecodeParams, unpack_bits
from oracle.windows import column_rounds, sliding_window_decode
from workloads.dem import circuit_dem
from workloads.zsz import load_code

ROUNDS = 3
KW = dict(gamma0=0.125, pre_iter=60, num_sets=10, max_iterations=40, stop_nconv=2, gamma_min=-0.24,
          gamma_max=0.66, seed=7)


@pytest.fixture(scope="module")
def setup():
    code = load_code("ZSZ-LP-60")
    dem = circuit_dem("ZSZ-LP-60", 0.004, ROUNDS, "Z")
    det_round = np.arange(dem.n_det) // (2 * code.ell)        # rounds 0..d-1, then the final readout
    assert det_round.max() == ROUNDS
    syn, obs, _ = oracle.sample(dem, 5, 0, 120)
    return dem, det_round, syn, obs


def test_columns_have_one_or_two_consecutive_rounds(setup):
    dem, det_round, _, _ = setup
    Hd = dem.dense_H().astype(bool)
    cr = column_rounds(dem, det_round)
    assert cr.max() <= ROUNDS
    for j in range(dem.n_loc):
        rs = np.unique(det_round[Hd[:, j]])
        assert rs.size and rs.min() == cr[j] and rs.max() - rs.min() <= 1


def test_one_window_over_all_rounds_is_the_block_decode(setup):
    dem, det_round, syn, _ = setup
    p = DecodeParams(**KW)
    w = sliding_window_decode(dem, det_round, ROUNDS + 1, p, syn)
    r = oracle.decode(dem, p, syn)
    assert w["windows"] == 1
    assert np.array_equal(w["corrections"], unpack_bits(r["corrections"], dem.n_loc))
    assert np.array_equal(w["converged"], r["stats"][:, 0] == 1)


@pytest.mark.parametrize("window", [1, 2, 3])
def test_converged_windows_leave_no_residual(setup, window):
    """Each window's decision satisfies its rows, so committing round t clears
    round t: a shot whose windows all converge ends with H e = s."""
    dem, det_round, syn, obs = setup
    w = sliding_window_decode(dem, det_round, window, DecodeParams(**KW), syn)
    assert w["windows"] == ROUNDS + 2 - window
    assert w["converged"].mean() > 0.8
    assert not w["residual"][w["converged"]].any()
    Hd = dem.dense_H().astype(np.int64)
    S = unpack_bits(syn, dem.n_det).astype(np.int64)
    assert np.array_equal((w["corrections"].astype(np.int64) @ Hd.T + S) % 2, w["residual"])


def test_look_ahead_pays(setup):
    """A one-round window decides without seeing the next round's detectors;
    the whole-block decode does better on the same shots (measured on 400
    shots: 65% correct for one-round windows, 78% for two or three rounds,
    83% for the whole block)."""
    dem, det_round, syn, obs = setup
    truth = unpack_bits(obs, dem.n_obs)
    rate = {}
    for window in (1, ROUNDS + 1):
        w = sliding_window_decode(dem, det_round, window, DecodeParams(**KW), syn)
        rate[window] = (w["converged"] & np.all(w["pred_obs"] == truth, axis=1)).mean()
    assert rate[1] < rate[ROUNDS + 1]
