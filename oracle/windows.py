"""Sliding-window Relay-BP decoding with a commit region of one round, plain
numpy over the FP64 oracle decoder (test infrastructure only).

arXiv 2607.27644, Sec. 6.1 (decoding latency) argues that its decoder is fast
enough for sliding-window decoding with a commit region of 1, where about d
rounds of syndromes are decoded every syndrome-extraction round; the paper
does not spell the procedure out.  The reading implemented here:

  * every detector has a round r (0 .. R-1; a memory experiment's final
    data-readout detectors form the last round), every fault column the round
    of its earliest detector (columns that touch no detector are never
    decoded, as in a whole-block decode where their posterior keeps the prior
    sign);
  * window t holds the columns whose round lies in [t, t + w) and the rows of
    those rounds; it decodes the residual syndrome on those rows with the
    handle's Relay-BP parameters and the same shot indices as a whole-block
    decode;
  * the columns of round t are committed (the last window, t + w >= R,
    commits all of its columns): their bits join the correction and their
    detector sets are XORed into the residual syndrome, which clears round t
    whenever the window converged; then t advances by one.
"""
from __future__ import annotations

import numpy as np

from . import DecodeParams, decode, pack_bits, unpack_bits


def column_rounds(dem, det_round: np.ndarray) -> np.ndarray:
    """Round of each fault column: the least round of its detectors (R + 1,
    past every window, for a column with no detector; R = number of rounds)."""
    Hd = dem.dense_H().astype(bool)
    R = int(det_round.max()) + 1
    rounds = np.where(Hd, det_round[:, None], R + 1).min(axis=0)
    return rounds


def _sub_dem(dem, rows: np.ndarray, cols: np.ndarray):
    from workloads.dem import dem_from_dense
    H = dem.dense_H()[np.ix_(rows, cols)]
    O = dem.dense_O()[:, cols]
    return dem_from_dense(H, dem.priors[cols], O, name=f"{dem.name}/window")


def sliding_window_decode(dem, det_round: np.ndarray, window: int, params: DecodeParams, syndromes: np.ndarray,
                          shot0: int = 0) -> dict:
    """Decode packed syndromes [shots, ceil(C/32)] window by window.  Returns
    dict(corrections [shots, V] uint8, pred_obs [shots, K] uint8,
    residual [shots, C] uint8 (H e + s: zero when every window converged),
    converged [shots] bool (every window converged), windows int)."""
    if window < 1:
        raise ValueError("window must be >= 1 round")
    C, V = dem.n_det, dem.n_loc
    det_round = np.asarray(det_round, dtype=np.int64)
    R = int(det_round.max()) + 1
    col_round = column_rounds(dem, det_round)
    Hd = dem.dense_H().astype(np.int64)
    S = unpack_bits(syndromes, C).astype(np.int64)
    shots = S.shape[0]
    resid = S.copy()
    corr = np.zeros((shots, V), dtype=np.int64)
    conv = np.ones(shots, dtype=bool)
    n_win = 0
    for t in range(R):
        last = t + window >= R
        rows = np.nonzero((det_round >= t) & (det_round < t + window))[0]
        cols = np.nonzero((col_round >= t) & (col_round < t + window))[0]
        sub = _sub_dem(dem, rows, cols)
        r = decode(sub, params, pack_bits(resid[:, rows]), shot0=shot0)
        n_win += 1
        conv &= r["stats"][:, 0] == 1
        e = unpack_bits(r["corrections"], len(cols)).astype(np.int64)
        commit = np.ones(len(cols), dtype=bool) if last else (col_round[cols] == t)
        cc = cols[commit]
        corr[:, cc] ^= e[:, commit]
        resid = (resid + e[:, commit] @ Hd[:, cc].T) % 2
        if last:
            break
    pred = (corr @ dem.dense_O().astype(np.int64).T) % 2
    return dict(corrections=corr.astype(np.uint8), pred_obs=pred.astype(np.uint8), residual=resid.astype(np.uint8),
                converged=conv, windows=n_win)
