"""relaybp_decode_host (host buffers in and out) against relaybp_decode_batch
on device buffers: predicted observables and per-shot statistics equal shot
for shot, one launch per call, pinned and pageable host memory, the two-shot
and the cluster kernels."""
import numpy as np
import pytest
import torch

from workloads.dem import circuit_dem

pytestmark = pytest.mark.gpu

KW = dict(gamma0=0.125, pre_iter=80, num_sets=1000, max_iterations=60, stop_nconv=5, gamma_min=-0.15,
          gamma_max=0.61, seed=202)


@pytest.fixture(scope="module")
def dem160():
    return circuit_dem("ZSZ-LP-160", 0.001, 10, "Z")


@pytest.mark.parametrize("shots,cluster", [(70_001, 0), (5_000, 0), (20_000, 16)])
def test_decode_host_equals_decode_batch(dem160, shots, cluster):
    from paper_2607_27644_b300 import relaybp as R
    h = R.relaybp_build_dem(dem160, R.Params(msg_dtype="f32", **KW))
    if cluster:
        R.relaybp_set_cluster_kernel(h, cluster)
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 3, 500, shots, syn)
    pobs = torch.zeros((shots, h.wk), dtype=torch.int32, device="cuda")
    stats = torch.zeros((shots, 6), dtype=torch.int32, device="cuda")
    R.relaybp_decode_batch(h, syn, 500, shots, None, pobs, stats)
    torch.cuda.synchronize()
    h_syn = syn.cpu().pin_memory()
    h_pobs = torch.full((shots, h.wk), -1, dtype=torch.int32).pin_memory()
    h_stats = torch.full((shots, 6), -1, dtype=torch.int32).pin_memory()
    n0 = R.relaybp_launch_count(h)
    R.relaybp_decode_host(h, h_syn, 500, shots, h_pobs, h_stats)
    assert R.relaybp_launch_count(h) - n0 == 1
    assert np.array_equal(h_pobs.numpy(), pobs.cpu().numpy())
    assert np.array_equal(h_stats.numpy(), stats.cpu().numpy())
    # a second call through the same staging buffers, pageable host memory
    h_pobs2 = np.full((shots, h.wk), -1, dtype=np.int32)
    R.relaybp_decode_host(h, syn.cpu().numpy(), 500, shots, h_pobs2, None)
    assert np.array_equal(h_pobs2, pobs.cpu().numpy())
    R.relaybp_destroy(h)


def test_sync_waits_for_the_stream_and_reports_success():
    """relaybp_sync on the stream a decode was queued on returns once the
    decode has finished: every shot's statistics are written when it returns,
    with no other synchronisation."""
    from paper_2607_27644_b300 import relaybp as R
    from workloads.dem import code_capacity_dem
    dem = code_capacity_dem("ZSZ-LP-160", 0.05)
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f64", num_sets=50, seed=101))
    shots = 4000
    st = torch.cuda.Stream()
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    stats = torch.full((shots, 6), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    R.relaybp_sample(h, 5, 0, shots, syn, None, None, st)
    R.relaybp_decode_batch(h, syn, 0, shots, None, None, stats, st)
    host = torch.empty((shots, 6), dtype=torch.int32).pin_memory()
    with torch.cuda.stream(st):
        host.copy_(stats, non_blocking=True)
    R.relaybp_sync(h, st)
    assert int(host[:, 3].min()) >= 1            # every shot ran at least one iteration
    R.relaybp_destroy(h)
