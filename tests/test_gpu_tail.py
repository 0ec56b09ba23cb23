"""Tail offload: shots about to start relay leg `legs` leave the two-shot
kernel and finish on thread-block clusters.  Both kernels evaluate the FP32
Relay-BP iteration with the same operations in the same order, a new leg
restarts the messages at zero, and the residual restarts consistent with
e^ = 0, so every output -- corrections, predicted observables, per-shot
statistics including the FP64 weight -- must equal a decode without offload
bit for bit: with many shots handed over, with more shots than hand-over slots
(the rest stay in the two-shot kernel), with every leg run, with learned
legs before the hand-over leg, and through the host-buffer and allocation-free
entry points."""
import numpy as np
import pytest
import torch

from workloads.dem import circuit_dem

pytestmark = pytest.mark.gpu

KW = dict(gamma0=0.125, pre_iter=80, num_sets=1000, max_iterations=60, stop_nconv=5, gamma_min=-0.15,
          gamma_max=0.61, seed=202)


def _run(R, h, syn, shot0, entry="batch"):
    n = syn.shape[0]
    corr = torch.full((n, h.wv), -1, dtype=torch.int32, device="cuda")
    pobs = torch.full((n, h.wk), -1, dtype=torch.int32, device="cuda")
    stats = torch.full((n, 6), -1, dtype=torch.int32, device="cuda")
    if entry == "batch":
        R.relaybp_decode_batch(h, syn, shot0, n, corr, pobs, stats)
    elif entry == "noalloc":
        R.relaybp_decode_batch_noalloc(h, syn, shot0, n, corr, pobs, stats)
    else:
        hp = torch.full((n, h.wk), -1, dtype=torch.int32).pin_memory()
        hs = torch.full((n, 6), -1, dtype=torch.int32).pin_memory()
        R.relaybp_decode_host(h, syn.cpu().pin_memory(), shot0, n, hp, hs)
        return None, hp.numpy(), hs.numpy()
    torch.cuda.synchronize()
    return corr.cpu().numpy(), pobs.cpu().numpy(), stats.cpu().numpy()


def _equal(a, b):
    for x, y in zip(a, b):
        if x is not None and y is not None:
            assert np.array_equal(x, y), int(np.sum(np.any(x != y, axis=1)))


@pytest.fixture(scope="module")
def dem4():
    return circuit_dem("ZSZ-LP-160", 0.004, 10, "Z")


@pytest.mark.parametrize("legs,cluster,cap,shots", [(3, 16, 1024, 1500), (2, 8, 16, 1200), (6, 4, 512, 600)])
def test_offload_equals_plain(dem4, legs, cluster, cap, shots):
    from paper_2607_27644_b300 import relaybp as R
    h = R.relaybp_build_dem(dem4, R.Params(msg_dtype="f32", **KW))
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 11, 40, shots, syn)
    ref = _run(R, h, syn, 40)
    st = ref[2]
    assert (st[:, 2] > legs).sum() > 20                 # plenty of shots reach the hand-over leg
    R.relaybp_set_tail_offload(h, legs, cluster, cap)
    n0 = R.relaybp_launch_count(h)
    got = _run(R, h, syn, 40)
    assert R.relaybp_launch_count(h) - n0 == 2
    _equal(got, ref)
    if cap < 100:                                       # more long shots than slots: the rest stay put
        assert (st[:, 2] > legs).sum() > cap
    R.relaybp_set_tail_offload(h, 0)
    _equal(_run(R, h, syn, 40), ref)
    R.relaybp_destroy(h)


@pytest.mark.parametrize("case", ["stop_all", "learned", "host", "noalloc"])
def test_offload_cases(dem4, case):
    from paper_2607_27644_b300 import relaybp as R
    kw = dict(KW)
    if case == "stop_all":
        kw.update(stop_all=True, num_sets=8)
    h = R.relaybp_build_dem(dem4, R.Params(msg_dtype="f32", **kw))
    shots = 800
    if case == "learned":
        rng = np.random.default_rng(5)
        wrow = torch.from_numpy(rng.uniform(0.7, 1.1, size=(6, dem4.n_det)).astype(np.float32)).cuda()
        knots = torch.from_numpy(np.sort(rng.uniform(-0.2, 0.7, size=9)).astype(np.float32)).cuda()
        R.relaybp_set_learned_rows(h, wrow, knots)
        R.relaybp_set_learned_legs(h, 3)
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 12, 0, shots, syn)
    entry = case if case in ("host", "noalloc") else "batch"
    ref = _run(R, h, syn, 0, entry)
    R.relaybp_set_tail_offload(h, 3, 16, 2048)
    _equal(_run(R, h, syn, 0, entry), ref)
    if case == "stop_all":
        assert np.all(ref[2][:, 2] == 9)
    R.relaybp_destroy(h)


def test_offload_rejections(dem4):
    from paper_2607_27644_b300 import relaybp as R
    h = R.relaybp_build_dem(dem4, R.Params(msg_dtype="f32", carry_messages=True, **KW))
    with pytest.raises(R.RelayBPError, match="carry"):
        R.relaybp_set_tail_offload(h, 3)
    R.relaybp_destroy(h)
    h = R.relaybp_build_dem(dem4, R.Params(msg_dtype="f64", **KW))
    with pytest.raises(R.RelayBPError, match="FP64"):
        R.relaybp_set_tail_offload(h, 3)
    R.relaybp_destroy(h)


@pytest.mark.parametrize("dtype", ["f32", "i8"])
def test_offload_timed_decode(dem4, dtype):
    """relaybp_decode_timed with offload: outputs unchanged; a handed-over
    shot keeps its start time and gets its retire time from the cluster
    kernel, so every shot has start < retire."""
    from paper_2607_27644_b300 import relaybp as R
    h = R.relaybp_build_dem(dem4, R.Params(msg_dtype=dtype, **KW))
    shots = 700
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 15, 0, shots, syn)

    def timed():
        corr = torch.full((shots, h.wv), -1, dtype=torch.int32, device="cuda")
        stats = torch.full((shots, 6), -1, dtype=torch.int32, device="cuda")
        times = torch.zeros((shots, 2), dtype=torch.int64, device="cuda")
        R.relaybp_decode_timed(h, syn, 0, shots, times, d_corrections=corr, d_stats=stats)
        torch.cuda.synchronize()
        return corr.cpu().numpy(), stats.cpu().numpy(), times.cpu().numpy()

    c0, s0, _ = timed()
    R.relaybp_set_tail_offload(h, 3, 8, 1024)
    c1, s1, t1 = timed()
    assert np.array_equal(c0, c1) and np.array_equal(s0, s1)
    assert np.all(t1[:, 0] > 0) and np.all(t1[:, 1] > t1[:, 0])
    long = s1[:, 2] > 3
    assert long.sum() > 20
    R.relaybp_destroy(h)


@pytest.mark.parametrize("dtype", ["f16", "i8", "f32_one_shot"])
def test_offload_from_the_one_shot_kernel(dem4, dtype):
    """FP16 / int8 storage and FP32 with the two-shot kernel off: the one-shot
    kernel hands the shots over, the cluster kernel continues them in the same
    storage form."""
    from paper_2607_27644_b300 import relaybp as R
    msg = "f32" if dtype == "f32_one_shot" else dtype
    h = R.relaybp_build_dem(dem4, R.Params(msg_dtype=msg, **KW))
    if dtype == "f32_one_shot":
        R.relaybp_set_pair_kernel(h, False)
    shots = 900
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 13, 7, shots, syn)
    ref = _run(R, h, syn, 7)
    assert (ref[2][:, 2] > 3).sum() > 20
    R.relaybp_set_tail_offload(h, 3, 8, 1024)
    n0 = R.relaybp_launch_count(h)
    _equal(_run(R, h, syn, 7), ref)
    assert R.relaybp_launch_count(h) - n0 == 2
    R.relaybp_destroy(h)


def test_offload_in_a_group_launch():
    """Two DEMs in one persistent launch, both with offload (one cluster launch
    each after the group launch), against the group without offload."""
    from paper_2607_27644_b300 import relaybp as R
    dems = [circuit_dem("ZSZ-LP-160", 0.004, 10, "Z"), circuit_dem("ZSZ-LP-160", 0.003, 10, "X")]
    hs = [R.relaybp_build_dem(d, R.Params(msg_dtype="f16", **KW)) for d in dems]
    shots = [700, 500]
    syns = []
    for h, n in zip(hs, shots):
        x = torch.zeros((n, h.wc), dtype=torch.int32, device="cuda")
        R.relaybp_sample(h, 14, 0, n, x)
        syns.append(x)

    def run():
        grp = R.relaybp_group_create(hs)
        outs = [(torch.full((n, h.wv), -1, dtype=torch.int32, device="cuda"),
                 torch.full((n, h.wk), -1, dtype=torch.int32, device="cuda"),
                 torch.full((n, 6), -1, dtype=torch.int32, device="cuda")) for h, n in zip(hs, shots)]
        R.relaybp_group_decode(grp, syns, [0, 0], shots, [o[0] for o in outs], [o[1] for o in outs],
                               [o[2] for o in outs])
        torch.cuda.synchronize()
        n_l = R.relaybp_group_launch_count(grp)
        R.relaybp_group_destroy(grp)
        return [tuple(t.cpu().numpy() for t in o) for o in outs], n_l

    ref, n_ref = run()
    for h in hs:
        R.relaybp_set_tail_offload(h, 3, 8, 1024)
    got, n_got = run()
    assert n_ref == 1 and n_got == 3
    for a, b in zip(got, ref):
        _equal(a, b)
    for h in hs:
        R.relaybp_destroy(h)
