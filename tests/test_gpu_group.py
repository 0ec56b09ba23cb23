"""Batched multi-DEM decoding: several DEMs of different sizes and shot counts
in one persistent launch must give, shot for shot, what each DEM gives alone
(the per-shot arithmetic does not depend on which block or launch runs it),
and the decoder's answers must agree with the oracle."""
import numpy as np
import pytest

import oracle
from workloads.dem import circuit_dem, circuit_dems

pytestmark = pytest.mark.gpu


def _single(R, h, syn, shot0):
    import torch
    n = syn.shape[0]
    corr = torch.zeros((n, h.wv), dtype=torch.int32, device="cuda")
    pobs = torch.zeros((n, h.wk), dtype=torch.int32, device="cuda")
    stats = torch.zeros((n, 6), dtype=torch.int32, device="cuda")
    R.relaybp_decode_batch(h, syn, shot0, n, corr, pobs, stats)
    torch.cuda.synchronize()
    return corr.cpu().numpy(), pobs.cpu().numpy(), stats.cpu().numpy()


def _run_group(dems, dtype, shots, kw):
    import torch
    from paper_2607_27644_b300 import relaybp as R
    hs = [R.relaybp_build_dem(d, R.Params(msg_dtype=dtype, **kw)) for d in dems]
    syns, outs = [], []
    for i, (h, n) in enumerate(zip(hs, shots)):
        syn = torch.zeros((n, h.wc), dtype=torch.int32, device="cuda")
        R.relaybp_sample(h, 31 + i, 1000 * i, n, syn)
        syns.append(syn)
        outs.append((torch.zeros((n, h.wv), dtype=torch.int32, device="cuda"),
                     torch.zeros((n, h.wk), dtype=torch.int32, device="cuda"),
                     torch.zeros((n, 6), dtype=torch.int32, device="cuda")))
    grp = R.relaybp_group_create(hs)
    R.relaybp_group_decode(grp, syns, [1000 * i for i in range(len(hs))], shots, [o[0] for o in outs],
                           [o[1] for o in outs], [o[2] for o in outs])
    torch.cuda.synchronize()
    assert R.relaybp_group_launch_count(grp) == 1
    res = []
    for i, h in enumerate(hs):
        single = _single(R, h, syns[i], 1000 * i)
        got = tuple(t.cpu().numpy() for t in outs[i])
        for a, b in zip(single, got):
            assert np.array_equal(a, b), (i, dems[i].name)
        res.append((syns[i].cpu().numpy().view(np.uint32), got))
    R.relaybp_group_destroy(grp)
    for h in hs:
        R.relaybp_destroy(h)
    return res


def test_group_equals_single_launches_fp32():
    kw = dict(num_sets=100, gamma_min=-0.15, gamma_max=0.61, seed=5)
    dems = circuit_dems("ZSZ-LP-160", [0.001, 0.002], 10, "Z") + [circuit_dem("ZSZ-LP-60", 0.004, 3, "Z")]
    _run_group(dems, "f32", [700, 300, 1100], kw)


def test_group_mixed_codes_fp16_off_chip_state():
    """ZSZ-LP-320 and ZSZ-LP-390 in FP16: the 390 state does not fit in shared
    memory, so the whole launch keeps per-block state in global memory; each
    DEM's results still equal its single launch, and the predicted observables
    of a sample agree with the FP64 oracle."""
    kw = dict(num_sets=100, gamma_min=-0.16, gamma_max=0.7, seed=6)
    dems = [circuit_dem("ZSZ-LP-320", 0.002, 14, "Z"), circuit_dem("ZSZ-LP-390", 0.002, 16, "Z")]
    res = _run_group(dems, "f16", [160, 96], kw)
    po = oracle.DecodeParams(**kw)
    for i, (dem, (syn, (corr, pobs, stats))) in enumerate(zip(dems, res)):
        idx = np.arange(0, syn.shape[0], 8)
        # the sample's global shot indices are 1000 i + idx: decode one by one
        agree = 0
        for t, s_ in enumerate(idx):
            r1 = oracle.decode(dem, po, syn[s_:s_ + 1], shot0=1000 * i + int(s_))
            agree += int(np.array_equal(r1["pred_obs"][0, :pobs.shape[1]], pobs[s_].view(np.uint32)))
        assert agree >= len(idx) - 1


def test_autotune_keeps_results():
    """The autotuner only changes the launch shape: decodes before and after
    tuning agree bit for bit."""
    import torch
    from paper_2607_27644_b300 import relaybp as R
    dem = circuit_dem("ZSZ-LP-160", 0.001, 10, "Z")
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", num_sets=100, gamma_min=-0.15, gamma_max=0.61, seed=3))
    syn = torch.zeros((2000, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 8, 0, 2000, syn)
    before = _single(R, h, syn, 0)
    # the two-shot kernel (default for this DEM): warps per block
    shape = R.relaybp_autotune(h, syn, 0, 2000)
    assert shape["L"] == 4 and shape["L"] * shape["NB"] >= 92 and 512 <= shape["threads"] <= 640
    assert shape["ms"] > 0
    after = _single(R, h, syn, 0)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    # the general kernel: row geometry and block size
    R.relaybp_set_pair_kernel(h, False)
    shape = R.relaybp_autotune(h, syn, 0, 2000)
    assert shape["L"] * shape["NB"] >= 92 and shape["threads"] in (256, 512) and shape["ms"] > 0
    after = _single(R, h, syn, 0)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    R.relaybp_destroy(h)
