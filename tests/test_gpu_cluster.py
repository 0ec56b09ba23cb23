"""The cluster (latency-mode) kernel against the default FP32 path, through
the C ABI.

The cluster kernel spreads one shot over 1..16 CTAs and exchanges state
through distributed shared memory, but evaluates the FP32 Relay-BP iteration
(Sec. 6.1) with the same rounded operations in the same order as the
one-shot-per-block kernels, so corrections, predicted observables and every
per-shot statistic must be equal bit for bit for every cluster size, batch
size (a single shot: one cluster; many shots: every resident cluster taking
shots from the work counter) and relay option.  The default FP32 path is
itself checked against the FP64 oracle in test_gpu_parity.py."""
import numpy as np
import pytest
import torch

from workloads.dem import circuit_dem

pytestmark = pytest.mark.gpu

CIRC_KW = dict(gamma0=0.125, pre_iter=80, num_sets=1000, max_iterations=60, stop_nconv=5,
               gamma_min=-0.15, gamma_max=0.61, seed=202)


def _run(R, h, syn, shot0, timed=False):
    n = syn.shape[0]
    corr = torch.full((n, h.wv), -1, dtype=torch.int32, device="cuda")
    pobs = torch.full((n, h.wk), -1, dtype=torch.int32, device="cuda")
    stats = torch.full((n, 6), -1, dtype=torch.int32, device="cuda")
    if timed:
        times = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
        R.relaybp_decode_timed(h, syn, shot0, n, times, d_corrections=corr, d_pred_obs=pobs, d_stats=stats)
        torch.cuda.synchronize()
        t = times.cpu().numpy()
        assert np.all(t[:, 1] > t[:, 0]) and np.all(t[:, 0] > 0)
    else:
        R.relaybp_decode_batch(h, syn, shot0, n, corr, pobs, stats)
    torch.cuda.synchronize()
    return corr.cpu().numpy(), pobs.cpu().numpy(), stats.cpu().numpy()


def _equal(a, b):
    for x, y, k in zip(a, b, ("corrections", "pred_obs", "stats")):
        assert np.array_equal(x, y), (k, int(np.sum(np.any(x != y, axis=1))))


@pytest.fixture(scope="module")
def dems():
    return dict(z1=circuit_dem("ZSZ-LP-160", 0.001, 10, "Z"), z4=circuit_dem("ZSZ-LP-160", 0.004, 10, "Z"),
                x2=circuit_dem("ZSZ-LP-160", 0.002, 10, "X"))


@pytest.mark.parametrize("which,nc,shots", [("z1", 16, 1), ("z1", 16, 700), ("z4", 8, 500), ("x2", 4, 400),
                                            ("z4", 2, 150), ("z1", 3, 100), ("x2", 5, 301)])
def test_cluster_equals_default_fp32(dems, which, nc, shots):
    from paper_2607_27644_b300 import relaybp as R
    h = R.relaybp_build_dem(dems[which], R.Params(msg_dtype="f32", **CIRC_KW))
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 41 + nc, 300, shots, syn)
    ref = _run(R, h, syn, 300)
    R.relaybp_set_cluster_kernel(h, nc)
    n0 = R.relaybp_launch_count(h)
    got = _run(R, h, syn, 300)
    assert R.relaybp_launch_count(h) - n0 == 1
    _equal(got, ref)
    st = got[2]
    assert np.all(st[:, 3] >= 1) and np.all(st[:, 2] >= 1)
    if which == "z4":
        assert st[:, 1].mean() > 2.0
    R.relaybp_set_cluster_kernel(h, 0)
    _equal(_run(R, h, syn, 300), ref)
    R.relaybp_destroy(h)


@pytest.mark.parametrize("opt", ["carry", "stop_all", "timed", "noalloc"])
def test_cluster_equals_default_fp32_options(dems, opt):
    from paper_2607_27644_b300 import relaybp as R
    kw = dict(CIRC_KW)
    shots = 300
    if opt == "carry":
        kw.update(carry_messages=True)
    elif opt == "stop_all":
        kw.update(stop_all=True, num_sets=6)
    h = R.relaybp_build_dem(dems["z4"], R.Params(msg_dtype="f32", **kw))
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 5, 77, shots, syn)
    ref = _run(R, h, syn, 77)
    R.relaybp_set_cluster_kernel(h, 16)
    if opt == "noalloc":
        n = shots
        corr = torch.full((n, h.wv), -1, dtype=torch.int32, device="cuda")
        pobs = torch.full((n, h.wk), -1, dtype=torch.int32, device="cuda")
        stats = torch.full((n, 6), -1, dtype=torch.int32, device="cuda")
        R.relaybp_decode_batch_noalloc(h, syn, 77, n, corr, pobs, stats)
        torch.cuda.synchronize()
        got = (corr.cpu().numpy(), pobs.cpu().numpy(), stats.cpu().numpy())
    else:
        got = _run(R, h, syn, 77, timed=(opt == "timed"))
    _equal(got, ref)
    if opt == "stop_all":
        assert np.all(got[2][:, 2] == 7)
    R.relaybp_destroy(h)


def test_cluster_zsz550_single_shots():
    """ZSZ-LP-550 (d = 18, the largest Table 5 DEM, 4180 x 63910): 16-CTA
    clusters, one shot per call and a batch, against the default path."""
    from paper_2607_27644_b300 import relaybp as R
    dem = circuit_dem("ZSZ-LP-550", 0.001, None, "Z")
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", **dict(CIRC_KW, gamma_min=-0.12, gamma_max=0.62)))
    shots = 64
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 7, 0, shots, syn)
    ref = _run(R, h, syn, 0)
    R.relaybp_set_cluster_kernel(h, 16)
    _equal(_run(R, h, syn, 0), ref)
    one = [_run(R, h, syn[i:i + 1], i) for i in range(4)]
    for i, o in enumerate(one):
        _equal(o, tuple(x[i:i + 1] for x in ref))
    R.relaybp_destroy(h)


@pytest.mark.parametrize("dtype,nc", [("f16", 8), ("bf16", 16), ("i8", 4)])
def test_cluster_equals_one_block_kernel_low_precision(dems, dtype, nc):
    """16- and 8-bit storage (FP32 arithmetic): the cluster kernel loads and
    stores exactly as the one-shot-per-block kernel, so outputs are equal."""
    from paper_2607_27644_b300 import relaybp as R
    h = R.relaybp_build_dem(dems["z4"], R.Params(msg_dtype=dtype, **CIRC_KW))
    shots = 500
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 61, 0, shots, syn)
    ref = _run(R, h, syn, 0)
    R.relaybp_set_cluster_kernel(h, nc)
    _equal(_run(R, h, syn, 0), ref)
    assert ref[2][:, 1].mean() > 2.0
    R.relaybp_destroy(h)


def test_cluster_zsz550_fp16_eight_ctas():
    """ZSZ-LP-550 in FP16 storage fits 8-CTA clusters (FP32 needs 16)."""
    from paper_2607_27644_b300 import relaybp as R
    dem = circuit_dem("ZSZ-LP-550", 0.001, None, "Z")
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f16", **dict(CIRC_KW, gamma_min=-0.12, gamma_max=0.62)))
    shots = 48
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 8, 0, shots, syn)
    ref = _run(R, h, syn, 0)
    R.relaybp_set_cluster_kernel(h, 8)
    _equal(_run(R, h, syn, 0), ref)
    R.relaybp_destroy(h)


def test_cluster_rejects_unsupported_handles(dems):
    from paper_2607_27644_b300 import relaybp as R
    h = R.relaybp_build_dem(dems["z1"], R.Params(msg_dtype="f64", **CIRC_KW))
    with pytest.raises(R.RelayBPError, match="FP64"):
        R.relaybp_set_cluster_kernel(h, 8)
    with pytest.raises(R.RelayBPError):
        R.relaybp_set_cluster_kernel(h, 17)
    R.relaybp_destroy(h)
