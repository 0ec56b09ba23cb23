"""OSD post-processing of the shots Relay-BP leaves unresolved (the paper's
outlook, Sec. 7), through the C ABI: relaybp_decode_flagged hands over the
flagged shots' final posteriors, relaybp_osd solves them.  Against the FP64
oracle: with the literal-order FP64 kernel the flagged set and the posteriors
are bit-exact, and OSD-0 / OSD-lambda give the oracle's corrections bit for
bit from the same posteriors; at p = 0.4% on the ZSZ-LP-160 circuit DEM the
failures left after OSD are counted."""
import numpy as np
import pytest

import oracle
from oracle import unpack_bits
from workloads.dem import circuit_dem, circuit_dems

pytestmark = pytest.mark.gpu

KW = dict(gamma0=0.125, pre_iter=30, num_sets=3, max_iterations=20, stop_nconv=1, gamma_min=-0.24, gamma_max=0.66,
          seed=5)


def _flagged(R, h, syn_t, shots, maxf):
    import torch
    idx = torch.full((maxf,), -1, dtype=torch.int64, device="cuda")
    post = torch.zeros((maxf, h.n_loc), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    stats = torch.zeros((shots, 6), dtype=torch.int32, device="cuda")
    pobs = torch.zeros((shots, h.wk), dtype=torch.int32, device="cuda")
    R.relaybp_decode_flagged(h, syn_t, 0, shots, maxf, idx, post, cnt, d_pred_obs=pobs, d_stats=stats)
    torch.cuda.synchronize()
    n = int(cnt.item())
    return n, idx, post, stats.cpu().numpy(), pobs.cpu().numpy().view(np.uint32)


def _osd(R, h, syn_t, post, idx, n, lam):
    import torch
    e = torch.zeros((n, h.wv), dtype=torch.int32, device="cuda")
    valid = torch.zeros(n, dtype=torch.int32, device="cuda")
    R.relaybp_osd(h, syn_t, post, idx, n, lam, e, valid)
    torch.cuda.synchronize()
    return e.cpu().numpy().view(np.uint32), valid.cpu().numpy()


def test_flagged_posteriors_and_osd_bit_exact():
    import torch
    from paper_2607_27644_b300 import relaybp as R
    dem = circuit_dems("ZSZ-LP-60", [0.01], 2, "Z")[0]
    shots = 400
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f64", **KW))
    syn, _, _ = oracle.sample(dem, 31, 0, shots)
    syn_t = torch.from_numpy(syn.view(np.int32)).cuda()
    n, idx, post, stats, _ = _flagged(R, h, syn_t, shots, shots)
    ro = oracle.decode_with_posteriors(dem, oracle.DecodeParams(**KW), syn)
    flagged_o = np.nonzero(ro["stats"][:, 0] == 0)[0]
    assert 40 <= n == len(flagged_o)
    ix = idx[:n].cpu().numpy()
    order = np.argsort(ix)
    assert np.array_equal(ix[order], flagged_o)
    P = post[:n].cpu().numpy()[order]
    assert np.array_equal(P, ro["posteriors"][flagged_o])           # bit for bit: the literal-order kernel
    L0 = np.log((1 - dem.priors) / dem.priors)
    srt = torch.from_numpy(ix[order].astype(np.int64)).cuda()
    Pt = torch.from_numpy(P).cuda()
    for lam in (0, 8):
        eg, vg = _osd(R, h, syn_t, Pt, srt, n, lam)
        oo = oracle.osd(dem.H_indptr, dem.H_indices, dem.n_det, dem.n_loc, syn[flagged_o], P, order=lam,
                        weights=L0)
        assert np.array_equal(eg, oo["corrections"]), lam
        assert np.array_equal(vg.astype(bool), oo["valid"]), lam
        Hd = dem.dense_H().astype(np.int64)
        eh = unpack_bits(eg, dem.n_loc).astype(np.int64)
        S = unpack_bits(syn[flagged_o], dem.n_det)
        assert np.array_equal((eh[vg == 1] @ Hd.T) % 2, S[vg == 1])     # valid OSD output solves H e = s
    R.relaybp_destroy(h)


def test_osd_on_random_posteriors_and_lambda_limits():
    """OSD against the oracle on arbitrary soft inputs (random posteriors with
    ties) for the FP32 two-shot decoder's DEM; lambda outside 0..64 is
    rejected."""
    import torch
    from paper_2607_27644_b300 import relaybp as R
    dem = circuit_dem("ZSZ-LP-160", 0.004, 10, "Z")
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", num_sets=2))
    n = 6
    syn, _, _ = oracle.sample(dem, 8, 0, n)
    rng = np.random.default_rng(4)
    P = np.round(rng.normal(3.0, 4.0, (n, dem.n_loc)), 1)              # many exact ties
    L0 = np.log((1 - dem.priors) / dem.priors)
    syn_t = torch.from_numpy(syn.view(np.int32)).cuda()
    ix = torch.arange(n, dtype=torch.int64, device="cuda")
    Pt = torch.from_numpy(P).cuda()
    for lam in (0, 16):
        eg, vg = _osd(R, h, syn_t, Pt, ix, n, lam)
        oo = oracle.osd(dem.H_indptr, dem.H_indices, dem.n_det, dem.n_loc, syn, P, order=lam, weights=L0)
        assert np.array_equal(eg, oo["corrections"]), lam
        assert np.array_equal(vg.astype(bool), oo["valid"]), lam
    e = torch.zeros((n, h.wv), dtype=torch.int32, device="cuda")
    v = torch.zeros(n, dtype=torch.int32, device="cuda")
    for bad in (-1, 65):
        with pytest.raises(R.RelayBPError):
            R.relaybp_osd(h, syn_t, Pt, ix, n, bad, e, v)
    R.relaybp_destroy(h)


def test_osd_after_relay_bp_failures_p04():
    """ZSZ-LP-160 circuit DEM at p = 0.4%, FP32 two-shot decoder with 30 relay
    legs: the flagged shots go through OSD-0 and OSD-16; the failures left
    (flagged shots whose OSD answer misses the sampled observables, plus the
    decoder's undetected logical errors) are reported and never exceed the
    decoder's own."""
    import warnings
    import torch
    from paper_2607_27644_b300 import relaybp as R
    dem = circuit_dem("ZSZ-LP-160", 0.004, 10, "Z")
    kw = dict(gamma0=0.125, pre_iter=80, num_sets=30, max_iterations=60, stop_nconv=1, gamma_min=-0.15,
              gamma_max=0.61, seed=9)
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", **kw))
    shots = 4000
    syn_t = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    obs_t = torch.zeros((shots, h.wk), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 44, 0, shots, syn_t, obs_t)
    n, idx, post, stats, pobs = _flagged(R, h, syn_t, shots, shots)
    obs = obs_t.cpu().numpy().view(np.uint32)
    conv = stats[:, 0] == 1
    logical = int((conv & np.any(pobs != obs, axis=1)).sum())
    assert n == int((~conv).sum()) and n > 0
    Od = dem.dense_O().astype(np.int64)
    ix = idx[:n].cpu().numpy()
    res = {}
    for lam in (0, 16):
        eg, vg = _osd(R, h, syn_t, post, idx, n, lam)
        eh = unpack_bits(eg, dem.n_loc).astype(np.int64)
        pred = (eh @ Od.T) % 2
        truth = unpack_bits(obs[ix], dem.n_obs)
        rescued = int(((vg == 1) & np.all(pred == truth, axis=1)).sum())
        res[lam] = rescued
    warnings.warn(UserWarning(
        f"p=0.4%, {shots} shots, 30 legs: {n} flagged nonconvergences, {logical} undetected logical errors; OSD-0 "
        f"answers {res[0]} of the flagged correctly, OSD-16 {res[16]} (failures {n + logical} -> "
        f"{n - res[0] + logical} / {n - res[16] + logical})"))
    assert 0 <= res[0] <= n and 0 <= res[16] <= n
    R.relaybp_destroy(h)
