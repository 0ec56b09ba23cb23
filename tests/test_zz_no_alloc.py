"""The allocation-free decode entry point against the regular one.

relaybp_decode_batch_noalloc exists for callers that must not allocate device
memory while decoding (real-time loops that cannot absorb cudaMalloc's
synchronisation, programs whose device memory belongs to another allocator).
It decodes with a fixed scratch array compiled into the library; its results
must equal relaybp_decode_batch's, on two calls in a row (the array keeps the
previous call's contents, so the second call checks that what must start at
zero is cleared).  This file is collected last so that a stop-at-first-failure
run has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _decode(R, h, syn, shot0, fn):
    import torch
    n = syn.shape[0]
    corr = torch.full((n, h.wv), -1, dtype=torch.int32, device="cuda")
    pobs = torch.full((n, h.wk), -1, dtype=torch.int32, device="cuda")
    stats = torch.full((n, 6), -1, dtype=torch.int32, device="cuda")
    fn(h, syn, shot0, n, corr, pobs, stats)
    torch.cuda.synchronize()
    return corr.cpu().numpy(), pobs.cpu().numpy(), stats.cpu().numpy()


@pytest.mark.parametrize("case", ["circuit_f32", "code_capacity_f64"])
def test_noalloc_matches_decode_batch_twice(case):
    import torch
    from paper_2607_27644_b300 import relaybp as R
    from workloads.dem import circuit_dem, code_capacity_dem
    if case == "circuit_f32":
        dem = circuit_dem("ZSZ-LP-160", 0.001, 10, "Z")
        params = R.Params(msg_dtype="f32", num_sets=1000, gamma_min=-0.15, gamma_max=0.61, seed=202)
        shots = 3000
    else:
        dem = code_capacity_dem("ZSZ-LP-160", 0.05)
        params = R.Params(msg_dtype="f64", num_sets=50, seed=101)
        shots = 2000
    h = R.relaybp_build_dem(dem, params)
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 77, 5000, shots, syn)
    ref = _decode(R, h, syn, 5000, R.relaybp_decode_batch)
    for _ in range(2):
        got = _decode(R, h, syn, 5000, R.relaybp_decode_batch_noalloc)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)
    # a different shot range through the same array right after
    syn2 = torch.zeros((shots // 2, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 78, 0, shots // 2, syn2)
    a = _decode(R, h, syn2, 0, R.relaybp_decode_batch)
    b = _decode(R, h, syn2, 0, R.relaybp_decode_batch_noalloc)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    R.relaybp_destroy(h)


def test_noalloc_rejects_state_beyond_its_limits():
    """A DEM whose per-shot state does not fit on chip would need off-chip
    state the allocation-free entry point does not have: a clear error."""
    import torch
    from paper_2607_27644_b300 import relaybp as R
    rng = np.random.default_rng(1)
    C, V = 1500, 70_000
    rows = [np.sort(rng.choice(V, 8, replace=False)) for _ in range(C)]
    indptr = np.r_[0, np.cumsum([len(r) for r in rows])].astype(np.int32)
    h = R.relaybp_build(indptr, np.concatenate(rows), C, V, np.full(V, 0.01), params=R.Params(num_sets=2))
    syn = torch.zeros((4, h.wc), dtype=torch.int32, device="cuda")
    with pytest.raises(R.RelayBPError, match="allocation-free"):
        R.relaybp_decode_batch_noalloc(h, syn, 0, 4)
    R.relaybp_destroy(h)


def test_noalloc_allocates_nothing_on_a_fresh_handle():
    """On a fresh handle, before any regular decode: after one warm-up call
    (module loading, the array's address lookup), a second call leaves the
    device's free memory unchanged, and its results equal the regular entry
    point's (run afterwards)."""
    import torch
    from paper_2607_27644_b300 import relaybp as R
    from workloads.dem import circuit_dem
    dem = circuit_dem("ZSZ-LP-160", 0.001, 10, "Z")
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", num_sets=1000, gamma_min=-0.15, gamma_max=0.61,
                                          seed=303))
    shots = 2000
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    R.relaybp_sample(h, 79, 0, shots, syn)
    outs = [(torch.full((shots, h.wv), -1, dtype=torch.int32, device="cuda"),
             torch.full((shots, h.wk), -1, dtype=torch.int32, device="cuda"),
             torch.full((shots, 6), -1, dtype=torch.int32, device="cuda")) for _ in range(2)]
    torch.cuda.synchronize()
    R.relaybp_decode_batch_noalloc(h, syn, 0, shots, *outs[0])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    R.relaybp_decode_batch_noalloc(h, syn, 0, shots, *outs[1])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes during the call"
    ref = _decode(R, h, syn, 0, R.relaybp_decode_batch)
    for a, b in zip(ref, outs[1]):
        assert np.array_equal(a, b.cpu().numpy())
    R.relaybp_destroy(h)
