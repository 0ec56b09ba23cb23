"""Classical channel coding on the GPU (Sec. 6.2): the ZSZ-2BGA-64 seed code
([64, 32, 10], the left seed code of ZSZ-LP-160) over BPSK-AWGN with flooding
sum-product BP (boxplus-phi, 100 iterations, LLRs clipped at 20), through the
C ABI, against the FP64 oracle.  The device's log, cos, log1p and expm1 are
not glibc's, so agreement is to rounding, not bit for bit: channel LLRs
within 1e-12 relative; from the same LLRs, decisions, validity and
iteration counts identical on >= 99.9% / 99.9% / 99% of frames and final
posteriors within 1e-6 relative where the iterations agree; frame error
rates within 2 sigma at 1.5 dB (FP64 and FP32)."""
import math

import numpy as np
import pytest

import oracle
from workloads.zsz import gf2_nullspace, load_code

pytestmark = pytest.mark.gpu


def _csr(H):
    H = np.asarray(H, dtype=np.uint8)
    indptr = np.r_[0, np.cumsum(H.sum(1))].astype(np.int32)
    indices = np.concatenate([np.nonzero(r)[0] for r in H]).astype(np.int32)
    return indptr, indices


@pytest.fixture(scope="module")
def code64():
    H = load_code("ZSZ-LP-160").H_left
    ip, ix = _csr(H)
    return H, ip, ix


def _codewords(H, frames, seed):
    G = gf2_nullspace(H)
    rng = np.random.default_rng(seed)
    c = (rng.integers(0, 2, (frames, G.shape[0])) @ G) % 2
    return c.astype(np.uint8)


def test_llr_sampler_matches_oracle(code64):
    import torch
    from paper_2607_27644_b300 import relaybp as R
    H, ip, ix = code64
    m, n = H.shape
    frames = 3000
    cw = _codewords(H, frames, 1)
    packed = oracle.pack_bits(cw)
    spa = R.relaybp_spa_create(ip, ix, m, n)
    d_cw = torch.from_numpy(packed.view(np.int32)).cuda()
    # 1.0 dB, and sigma = 0.3 where 2 y / sigma^2 passes the clip at 20 on most bits
    for sigma in (oracle.awgn_sigma(1.0, 0.5), 0.3):
        Lo = oracle.awgn_llr(n, sigma, 77, 500, frames, codewords=packed)
        Lg = torch.zeros((frames, n), dtype=torch.float64, device="cuda")
        spa.llr(sigma, 77, 500, frames, Lg, d_codewords=d_cw)
        torch.cuda.synchronize()
        Lg = Lg.cpu().numpy()
        assert np.allclose(Lg, Lo, rtol=1e-12, atol=1e-12)
        assert np.array_equal(Lg < 0, Lo < 0)
        if sigma == 0.3:
            assert np.abs(Lg).max() == 20.0 and (np.abs(Lg) == 20.0).mean() > 0.5
    spa.destroy()


@pytest.mark.parametrize("ebn0", [1.0, 2.5])
def test_sum_product_matches_oracle_from_the_same_llrs(code64, ebn0):
    import torch
    from paper_2607_27644_b300 import relaybp as R
    H, ip, ix = code64
    m, n = H.shape
    frames = 4000
    L = oracle.awgn_llr(n, oracle.awgn_sigma(ebn0, 0.5), 9, 0, frames)
    ro = oracle.sum_product(ip, ix, m, n, L, max_iter=100, posteriors=True)
    spa = R.relaybp_spa_create(ip, ix, m, n)
    Lt = torch.from_numpy(L).cuda()
    bits = torch.zeros((frames, (n + 31) // 32), dtype=torch.int32, device="cuda")
    iters = torch.zeros(frames, dtype=torch.int32, device="cuda")
    valid = torch.zeros(frames, dtype=torch.int32, device="cuda")
    post = torch.zeros((frames, n), dtype=torch.float64, device="cuda")
    spa.decode(Lt, frames, bits, iters, valid, post)
    torch.cuda.synchronize()
    bg, ig, vg, pg = bits.cpu().numpy().view(np.uint32), iters.cpu().numpy(), valid.cpu().numpy(), post.cpu().numpy()
    same_bits = np.all(bg == ro["bits"], axis=1)
    assert (~same_bits).sum() <= math.floor(0.001 * frames)
    assert ((vg == 1) != ro["valid"]).sum() <= math.floor(0.001 * frames)
    same_it = ig == ro["iters"]
    assert same_it.mean() >= 0.99
    rel = np.abs(pg - ro["posteriors"]) / np.maximum(1.0, np.abs(ro["posteriors"]))
    assert rel[same_it & ro["valid"]].max() <= 1e-6
    assert np.all(((oracle.unpack_bits(bg, n)[vg == 1].astype(np.int64) @ H.T) % 2) == 0)
    spa.destroy()


def test_frame_error_rate_within_two_sigma(code64):
    """1.5 dB, 20,000 all-zero frames sampled on the device (FP64 and FP32
    decoding) against the oracle's sampler and decoder on the same frames."""
    import torch
    from paper_2607_27644_b300 import relaybp as R
    from paper_2607_27644_b300.stats import agree_within
    H, ip, ix = code64
    m, n = H.shape
    frames, sigma = 20000, oracle.awgn_sigma(1.5, 0.5)
    ro = oracle.sum_product(ip, ix, m, n, oracle.awgn_llr(n, sigma, 3, 0, frames), max_iter=100)
    fer_o = int((~ro["valid"] | ro["bits"].any(1)).sum())
    spa = R.relaybp_spa_create(ip, ix, m, n)
    for dt in (torch.float64, torch.float32):
        Lg = torch.zeros((frames, n), dtype=dt, device="cuda")
        spa.llr(sigma, 3, 0, frames, Lg)
        bits = torch.zeros((frames, (n + 31) // 32), dtype=torch.int32, device="cuda")
        iters = torch.zeros(frames, dtype=torch.int32, device="cuda")
        valid = torch.zeros(frames, dtype=torch.int32, device="cuda")
        spa.decode(Lg, frames, bits, iters, valid)
        torch.cuda.synchronize()
        fer_g = int(((valid == 0) | (bits != 0).any(1)).sum())
        assert fer_o > 20 and agree_within(fer_o, frames, fer_g, frames), (dt, fer_o, fer_g)
    spa.destroy()
