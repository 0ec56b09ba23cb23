"""The two-shot FP32 decode kernel against the general one-shot-per-block
kernel, through the C ABI.

Both evaluate the same Relay-BP iteration (Sec. 6.1) with the same explicitly
rounded FP32 operations in the same order, so every output -- corrections,
predicted observables, per-shot statistics, FP64 weights and the posterior
trace -- must be equal bit for bit, whatever the batch size (odd batches and a
single shot leave one of a block's two slots idle), the relay options (message
carry-over, running every leg) or the learned row-tied weights and memory-
strength knots.  The general kernel is itself checked against the FP64 oracle
in test_gpu_parity.py; the default FP32 path of the parity tests there is this
kernel.
"""
import numpy as np
import pytest
import torch

from workloads.dem import circuit_dem

pytestmark = pytest.mark.gpu

CIRC_KW = dict(gamma0=0.125, pre_iter=80, num_sets=1000, max_iterations=60, stop_nconv=5,
               gamma_min=-0.15, gamma_max=0.61, seed=202)


def _run(R, h, syn, shot0, trace_iters=0, timed=False):
    n = syn.shape[0]
    corr = torch.full((n, h.wv), -1, dtype=torch.int32, device="cuda")
    pobs = torch.full((n, h.wk), -1, dtype=torch.int32, device="cuda")
    stats = torch.full((n, 6), -1, dtype=torch.int32, device="cuda")
    out = {}
    if timed:
        times = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
        R.relaybp_decode_timed(h, syn, shot0, n, times, d_corrections=corr, d_pred_obs=pobs, d_stats=stats)
        out["times"] = times
    else:
        R.relaybp_decode_batch(h, syn, shot0, n, corr, pobs, stats)
    if trace_iters:
        tr = torch.full((n, trace_iters, h.n_loc), float("nan"), dtype=torch.float64, device="cuda")
        R.relaybp_decode_trace(h, syn, shot0, n, trace_iters, tr, None)
        out["trace"] = tr
    torch.cuda.synchronize()
    out.update(corr=corr, pobs=pobs, stats=stats)
    return {k: v.cpu().numpy() for k, v in out.items()}


def _both(R, h, syn, shot0, **kw):
    R.relaybp_set_pair_kernel(h, True)
    n0 = R.relaybp_launch_count(h)
    a = _run(R, h, syn, shot0, **kw)
    R.relaybp_set_pair_kernel(h, False)
    b = _run(R, h, syn, shot0, **kw)
    R.relaybp_set_pair_kernel(h, True)
    return a, b, R.relaybp_launch_count(h) - n0


def _equal(a, b):
    for k in a:
        if k == "times":
            continue
        x, y = a[k], b[k]
        if x.dtype.kind == "f":
            assert np.array_equal(x, y, equal_nan=True), k
        else:
            assert np.array_equal(x, y), (k, int(np.sum(np.any(x != y, axis=tuple(range(1, x.ndim))))))


@pytest.fixture(scope="module")
def dems():
    return dict(z1=circuit_dem("ZSZ-LP-160", 0.001, 10, "Z"), z4=circuit_dem("ZSZ-LP-160", 0.004, 10, "Z"),
                x2=circuit_dem("ZSZ-LP-160", 0.002, 10, "X"))


@pytest.mark.parametrize("which,shots,trace", [("z1", 3001, 0), ("z4", 1200, 24), ("x2", 1501, 12)])
def test_pair_equals_general_kernel(dems, which, shots, trace):
    from paper_2607_27644_b300 import relaybp as R
    dem = dems[which]
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", **CIRC_KW))
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 31 + shots, 1000, shots, syn)
    a, b, launches = _both(R, h, syn, 1000, trace_iters=trace)
    _equal(a, b)
    assert launches == (4 if trace else 2)
    st = a["stats"]
    assert np.all(st[:, 1] >= 0) and np.all(st[:, 3] >= 1)            # every shot decoded
    if which == "z4":
        assert np.mean(st[:, 1]) > 2.0                                   # several legs and solutions per shot
    R.relaybp_destroy(h)


@pytest.mark.parametrize("opt", ["carry", "stop_all", "single_shot", "timed"])
def test_pair_equals_general_kernel_options(dems, opt):
    from paper_2607_27644_b300 import relaybp as R
    kw = dict(CIRC_KW)
    shots = 700
    if opt == "carry":
        kw.update(carry_messages=True)
    elif opt == "stop_all":
        kw.update(stop_all=True, num_sets=6)
        shots = 301
    elif opt == "single_shot":
        shots = 1
    h = R.relaybp_build_dem(dems["z4"], R.Params(msg_dtype="f32", **kw))
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 5, 77, shots, syn)
    a, b, _ = _both(R, h, syn, 77, timed=(opt == "timed"))
    _equal(a, b)
    if opt == "stop_all":
        assert np.all(a["stats"][:, 2] == 7)                             # every leg ran
    if opt == "timed":
        t = a["times"]
        assert np.all(t[:, 1] > t[:, 0]) and np.all(t[:, 0] > 0)
    R.relaybp_destroy(h)


def test_pair_equals_general_kernel_learned_rows(dems):
    """Row-tied weights over the first iterations of each leg and knot-drawn
    memory strengths, applied to legs 0..2 (plain legs after)."""
    from paper_2607_27644_b300 import relaybp as R
    dem = dems["z4"]
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", **CIRC_KW))
    rng = np.random.default_rng(3)
    T = 6
    wrow = torch.from_numpy(rng.uniform(0.6, 1.1, size=(T, dem.n_det)).astype(np.float32)).cuda()
    knots = torch.from_numpy(np.sort(rng.uniform(-0.2, 0.7, size=9)).astype(np.float32)).cuda()
    R.relaybp_set_learned_rows(h, wrow, knots)
    R.relaybp_set_learned_legs(h, 3)
    shots = 900
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 8, 0, shots, syn)
    a, b, _ = _both(R, h, syn, 0, trace_iters=10)
    _equal(a, b)
    R.relaybp_destroy(h)


def test_pair_kernel_autotune_and_warps(dems):
    """The warps-per-block choice and the autotuner change no output."""
    from paper_2607_27644_b300 import relaybp as R
    h = R.relaybp_build_dem(dems["z1"], R.Params(msg_dtype="f32", **CIRC_KW))
    shots = 2000
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 9, 0, shots, syn)
    ref = _run(R, h, syn, 0)
    for w in (16, 19):
        R.relaybp_set_pair_kernel(h, True, w)
        _equal(_run(R, h, syn, 0), ref)
    R.relaybp_set_pair_kernel(h, True, 0)
    tuned = R.relaybp_autotune(h, syn, 0, shots)
    assert tuned["L"] == 4 and 512 <= tuned["threads"] <= 640
    _equal(_run(R, h, syn, 0), ref)
    R.relaybp_destroy(h)
