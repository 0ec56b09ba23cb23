"""Sliding-window decoding with a commit region of one round (Sec. 6.1,
decoding-latency paragraph) through the C ABI, against the window oracle.

FP64 windows decode with the literal-order kernel, so corrections, predicted
observables, residuals and convergence flags equal the oracle's bit for bit
on the [[60,12,6]] 3-round circuit DEM for every window length.  FP32 windows
of the ZSZ-LP-160 d = 10 circuit DEM agree with the FP64 oracle on the answer
(convergence and predicted observables) of >= 99% of shots; at any precision
one window over all rounds is the whole-DEM decode, bit for bit, and the
residual equals H e^ + s with e^ the committed correction."""
import numpy as np
import pytest
import torch

import oracle
from oracle import DecodeParams, unpack_bits
from oracle.windows import sliding_window_decode
from workloads.dem import circuit_dem, detector_rounds

pytestmark = pytest.mark.gpu

KW60 = dict(gamma0=0.125, pre_iter=60, num_sets=10, max_iterations=40, stop_nconv=2, gamma_min=-0.24,
            gamma_max=0.66, seed=7)
KW160 = dict(gamma0=0.125, pre_iter=80, num_sets=1000, max_iterations=60, stop_nconv=5, gamma_min=-0.15,
             gamma_max=0.61, seed=202)


def _gpu_windows(R, wins, syn, shot0):
    n = syn.shape[0]
    d_syn = torch.from_numpy(syn.view(np.int32)).cuda()
    corr = torch.full((n, wins.wv), -1, dtype=torch.int32, device="cuda")
    pobs = torch.full((n, wins.wk), -1, dtype=torch.int32, device="cuda")
    res = torch.full((n, wins.wc), -1, dtype=torch.int32, device="cuda")
    conv = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    wins.decode(d_syn, shot0, n, corr, pobs, res, conv)
    torch.cuda.synchronize()
    return dict(corrections=corr.cpu().numpy().view(np.uint32), pred_obs=pobs.cpu().numpy().view(np.uint32),
                residual=res.cpu().numpy().view(np.uint32), converged=conv.cpu().numpy())


@pytest.fixture(scope="module")
def dem60():
    dem = circuit_dem("ZSZ-LP-60", 0.004, 3, "Z")
    return dem, detector_rounds(dem)


@pytest.mark.parametrize("window", [1, 2, 3, 4])
def test_fp64_windows_equal_the_oracle(dem60, window):
    from paper_2607_27644_b300 import relaybp as R
    dem, dr = dem60
    shots, shot0 = 400, 1000
    syn, _, _ = oracle.sample(dem, 5, shot0, shots)
    ref = sliding_window_decode(dem, dr, window, DecodeParams(**KW60), syn, shot0=shot0)
    wins = R.relaybp_windows_create(dem, dr, window, R.Params(msg_dtype="f64", **KW60))
    assert wins.n_windows == ref["windows"] == max(4 - window, 0) + 1
    got = _gpu_windows(R, wins, syn, shot0)
    wins.destroy()
    assert np.array_equal(unpack_bits(got["corrections"], dem.n_loc), ref["corrections"])
    assert np.array_equal(unpack_bits(got["pred_obs"], dem.n_obs), ref["pred_obs"])
    assert np.array_equal(unpack_bits(got["residual"], dem.n_det), ref["residual"])
    assert np.array_equal(got["converged"] == 1, ref["converged"])
    assert ref["converged"].mean() > 0.8


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16"])
def test_one_window_is_the_whole_dem_decode(dem60, dtype):
    from paper_2607_27644_b300 import relaybp as R
    dem, dr = dem60
    shots = 3000
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype=dtype, **KW60))
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 3, 0, shots, syn)
    corr = torch.zeros((shots, h.wv), dtype=torch.int32, device="cuda")
    pobs = torch.zeros((shots, h.wk), dtype=torch.int32, device="cuda")
    stats = torch.zeros((shots, 6), dtype=torch.int32, device="cuda")
    R.relaybp_decode_batch(h, syn, 0, shots, corr, pobs, stats)
    wins = R.relaybp_windows_create(dem, dr, 9, R.Params(msg_dtype=dtype, **KW60))
    assert wins.n_windows == 1
    got = _gpu_windows(R, wins, syn.cpu().numpy().view(np.uint32), 0)
    wins.destroy()
    assert np.array_equal(got["corrections"], corr.cpu().numpy().view(np.uint32))
    assert np.array_equal(got["pred_obs"], pobs.cpu().numpy().view(np.uint32))
    assert np.array_equal(got["converged"], stats.cpu().numpy()[:, 0])
    R.relaybp_destroy(h)


def test_fp32_windows_answer_the_oracle_zsz160():
    """ZSZ-LP-160, d = 10, p = 0.1%, three-round windows (9 windows) at the
    paper's decoder settings; 300 shots for the oracle.  The GPU side also
    decodes 20,000 shots whose residuals are checked against H e^ + s."""
    from paper_2607_27644_b300 import relaybp as R
    dem = circuit_dem("ZSZ-LP-160", 0.001, 10, "Z")
    dr = detector_rounds(dem)
    wins = R.relaybp_windows_create(dem, dr, 3, R.Params(msg_dtype="f32", **KW160))
    assert wins.n_windows == 9
    shots = 300
    syn, obs, _ = oracle.sample(dem, 21, 0, shots)
    ref = sliding_window_decode(dem, dr, 3, DecodeParams(**KW160), syn)
    got = _gpu_windows(R, wins, syn, 0)
    same = (got["converged"] == 1) == ref["converged"]
    same &= np.all(unpack_bits(got["pred_obs"], dem.n_obs) == ref["pred_obs"], axis=1)
    assert (~same).sum() <= 3, int((~same).sum())
    truth = unpack_bits(obs, dem.n_obs)
    assert (ref["converged"] & np.all(ref["pred_obs"] == truth, axis=1)).mean() > 0.95

    big = 20000
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", **KW160))
    d_syn = torch.zeros((big, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 22, 0, big, d_syn)
    g = _gpu_windows(R, wins, d_syn.cpu().numpy().view(np.uint32), 0)
    e = unpack_bits(g["corrections"], dem.n_loc).astype(np.int64)
    S = unpack_bits(d_syn.cpu().numpy().view(np.uint32), dem.n_det).astype(np.int64)
    Hd = dem.dense_H().astype(np.int64)
    assert np.array_equal((e @ Hd.T + S) % 2, unpack_bits(g["residual"], dem.n_det))
    assert not unpack_bits(g["residual"], dem.n_det)[g["converged"] == 1].any()
    assert g["converged"].mean() > 0.99
    wins.destroy()
    R.relaybp_destroy(h)
