"""Learned form: GPU forward loss and backward gradients against the FP64
oracle -- the loss directly, the gradients by central finite differences of
the oracle's forward (coordinates where a min/argmin kink lies within the
step, seen as FD(h) != FD(h/2), are excluded) -- for both training objectives
(cross-entropy against the sampled error, soft syndrome) and both training
precisions (FP64, and FP32, which training uses)."""
import numpy as np
import pytest

import oracle
from oracle import unpack_bits
from workloads.dem import circuit_dem

pytestmark = pytest.mark.gpu


def _setup(dem, T, seed, dtype):
    import torch
    from paper_2607_27644_b300 import relaybp as R
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.6, 1.4, (T, dem.n_edges))
    knots = np.cumsum(np.r_[-0.2, rng.uniform(0.02, 0.07, 16)])
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", num_sets=1))
    return R, h, w, knots


def _gpu_loss_grad(R, h, w, knots, syn, err, shot0, dtype, gseed, objective=0):
    import torch
    tw = torch.tensor(w, dtype=dtype, device="cuda")
    tk = torch.tensor(knots, dtype=dtype, device="cuda")
    ts = torch.from_numpy(syn.view(np.int32)).cuda()
    te = torch.from_numpy(err.view(np.int32)).cuda()
    shots = syn.shape[0]
    prec = R._prec(dtype)
    tape = torch.empty(R.relaybp_learned_tape_bytes(h, prec, w.shape[0], shots), dtype=torch.uint8, device="cuda")
    loss = torch.zeros(shots, dtype=torch.float64, device="cuda")
    R.relaybp_learned_forward(h, tw, tk, gseed, ts, te, shot0, shots, tape, loss, objective=objective)
    gw = torch.zeros_like(tw)
    gk = torch.zeros_like(tk)
    R.relaybp_learned_backward(h, tw, tk, gseed, te, shot0, shots, tape, 1.0, gw, gk, objective=objective,
                               d_syndromes=ts)
    torch.cuda.synchronize()
    return loss.cpu().numpy(), gw.cpu().numpy().astype(np.float64), gk.cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def small_dem():
    return circuit_dem("ZSZ-LP-60", 0.004, 2, "Z")


@pytest.mark.parametrize("objective", [0, 1])
def test_forward_loss_matches_oracle(small_dem, objective):
    import torch
    dem = small_dem
    for dtype, T, tol in ((torch.float64, 8, 1e-10), (torch.float32, 3, 1e-4)):
        R, h, w, knots = _setup(dem, T, 1, dtype)
        syn, _, err = oracle.sample(dem, 3, 100, 24, want_errors=True)
        lo, _ = oracle.learned_loss(dem, w, knots, 9, syn, err, shot0=100, objective=objective)
        lg, _, _ = _gpu_loss_grad(R, h, w, knots, syn, err, 100, dtype, 9, objective)
        assert np.allclose(lg, lo, rtol=tol, atol=tol), (dtype, np.abs(lg - lo).max())
        R.relaybp_destroy(h)


# FP64 gradients to 1e-5 relative; FP32 (what training runs) to 5e-3 relative
# of max(1, |FD|): its forward rounds every message to 2^-24 and the unrolled
# map amplifies that a few times per iteration over the T = 6 iterations.
@pytest.mark.parametrize("dtype,objective,tol", [("f64", 0, 1e-5), ("f64", 1, 1e-5), ("f32", 0, 5e-3),
                                                 ("f32", 1, 5e-3)])
def test_gradients_match_finite_differences(small_dem, dtype, objective, tol):
    import torch
    dem = small_dem
    T = 6
    tdt = torch.float64 if dtype == "f64" else torch.float32
    R, h, w, knots = _setup(dem, T, 2, tdt)
    if dtype == "f32":
        w = w.astype(np.float32).astype(np.float64)
        knots = knots.astype(np.float32).astype(np.float64)
    syn, _, err = oracle.sample(dem, 4, 0, 16, want_errors=True)
    _, gw, gk = _gpu_loss_grad(R, h, w, knots, syn, err, 0, tdt, 11, objective)

    def L(wv, kv):
        return oracle.learned_loss(dem, wv, kv, 11, syn, err, objective=objective)[0].sum()

    def fd(fun, x, idx, hh):
        xp, xm = x.copy(), x.copy()
        xp[idx] += hh
        xm[idx] -= hh
        return (fun(xp) - fun(xm)) / (2 * hh)

    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(40):
        t, e = int(rng.integers(T)), int(rng.integers(dem.n_edges))
        f1 = fd(lambda x: L(x, knots), w, (t, e), 1e-6)
        f2 = fd(lambda x: L(x, knots), w, (t, e), 5e-7)
        if abs(f1 - f2) > 1e-6 * max(1.0, abs(f1)):
            continue
        assert abs(gw[t, e] - f1) <= tol * max(1.0, abs(f1)), (t, e, gw[t, e], f1)
        checked += 1
    assert checked >= 30
    kchecked = 0
    for k in range(knots.size):
        f1 = fd(lambda x: L(w, x), knots, k, 1e-7)
        f2 = fd(lambda x: L(w, x), knots, k, 5e-8)
        if abs(f1 - f2) > 1e-5 * max(1.0, abs(f1)):
            continue
        assert abs(gk[k] - f1) <= 10 * tol * max(1.0, abs(f1)), (k, gk[k], f1)
        kchecked += 1
    assert kchecked >= 12
    R.relaybp_destroy(h)


def test_training_reduces_loss():
    """Gradient steps at scale (ZSZ-LP-160 circuit DEM, FP32, T = 10): Adam on a
    fixed batch of self-sampled shots lowers that batch's loss.  The unrolled
    min-sum map is piecewise linear and chaotic, so the loss along the steps is
    rough and the gradient sums (float atomics) vary between runs: the test
    asks for the best iterate, which is the one training keeps, to be >= 2%
    below the start."""
    import torch
    from paper_2607_27644_b300 import relaybp as R
    from paper_2607_27644_b300.learned import LearnedParams
    dem = circuit_dem("ZSZ-LP-160", 0.002, 10, "Z")
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", num_sets=1))
    T, B = 10, 256
    model = LearnedParams(T, dem.n_edges, -0.15, 0.61)
    opt = torch.optim.Adam(model.parameters(), lr=3e-3)

    def batch(shot0):
        syn = torch.zeros((B, h.wc), dtype=torch.int32, device="cuda")
        err = torch.zeros((B, h.wv), dtype=torch.int32, device="cuda")
        R.relaybp_sample(h, 4, shot0, B, syn, None, err)
        return syn, err

    s, e = batch(10**9)
    losses = []
    for step in range(30):
        opt.zero_grad()
        loss = model.loss(h, s, e, 10**9, 77)
        loss.backward()
        opt.step()
        losses.append(float(loss))
    with torch.no_grad():
        losses.append(float(model.loss(h, s, e, 10**9, 77)))
    assert min(losses[1:]) < 0.98 * losses[0], losses
    k = model.knots().detach().cpu().numpy()
    assert np.all(np.diff(k) >= 0)
    R.relaybp_destroy(h)


def test_learned_decode_unit_weights_equal_plain():
    import torch
    from paper_2607_27644_b300 import relaybp as R
    from gpu_util import gpu_decode
    dem = circuit_dem("ZSZ-LP-160", 0.001, 10, "Z")
    p = R.Params(msg_dtype="f32", num_sets=100, gamma_min=-0.15, gamma_max=0.61, seed=3)
    h = R.relaybp_build_dem(dem, p)
    syn, _, _ = oracle.sample(dem, 5, 0, 600)
    plain = gpu_decode(h, syn)
    w = torch.ones((7, dem.n_edges), dtype=torch.float32, device="cuda")
    R.relaybp_set_learned(h, w, None)
    ones = gpu_decode(h, syn)
    for k in ("corrections", "pred_obs", "stats", "weights"):
        assert np.array_equal(plain[k], ones[k]), k
    R.relaybp_destroy(h)


def test_learned_decode_matches_oracle():
    import torch
    from paper_2607_27644_b300 import relaybp as R
    from gpu_util import gpu_decode
    dem = circuit_dem("ZSZ-LP-160", 0.001, 10, "Z")
    kw = dict(num_sets=100, gamma_min=-0.15, gamma_max=0.61, seed=4)
    rng = np.random.default_rng(6)
    T = 8
    w = rng.uniform(0.75, 1.0, (T, dem.n_edges))
    knots = np.cumsum(np.r_[-0.15, rng.uniform(0.02, 0.07, 16)])
    h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", **kw))
    tw = torch.tensor(w, dtype=torch.float32, device="cuda")
    tk = torch.tensor(knots, dtype=torch.float32, device="cuda")
    R.relaybp_set_learned(h, tw, tk)
    syn, obs, _ = oracle.sample(dem, 6, 0, 300)
    rg = gpu_decode(h, syn)
    ro = oracle.decode(dem, oracle.DecodeParams(**kw), syn, w=w.astype(np.float32).astype(np.float64),
                       knots=knots.astype(np.float32).astype(np.float64))
    Hd = dem.dense_H().astype(np.int64)
    S = unpack_bits(syn, dem.n_det)
    for r in (ro, rg):
        eh = unpack_bits(r["corrections"], dem.n_loc).astype(np.int64)
        conv = r["stats"][:, 0] == 1
        assert np.array_equal((eh[conv] @ Hd.T) % 2, S[conv])
    same = np.all(ro["pred_obs"][:, :rg["pred_obs"].shape[1]] == rg["pred_obs"], axis=1)
    assert (~same).sum() <= 0
    R.relaybp_destroy(h)


def test_row_tied_weights_equal_expanded_per_edge_weights():
    """Tied weights travel in the check state; decoding equals the per-edge
    path with the same weights expanded over each row, bit for bit."""
    import torch
    from paper_2607_27644_b300 import relaybp as R
    from gpu_util import gpu_decode
    dem = circuit_dem("ZSZ-LP-160", 0.001, 10, "Z")
    kw = dict(num_sets=50, gamma_min=-0.15, gamma_max=0.61, seed=9, stop_nconv=2)
    T = 6
    rng = np.random.default_rng(10)
    wrow = rng.uniform(0.7, 1.0, (T, dem.n_det)).astype(np.float32)
    row_of = np.repeat(np.arange(dem.n_det), np.diff(dem.H_indptr))
    wedge = wrow[:, row_of].copy()
    knots = np.cumsum(np.r_[-0.15, rng.uniform(0.02, 0.07, 16)]).astype(np.float32)
    syn, _, _ = oracle.sample(dem, 12, 0, 500)
    ha = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", **kw))
    hb = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", **kw))
    tk = torch.tensor(knots, device="cuda")
    R.relaybp_set_learned(ha, torch.tensor(wedge, device="cuda"), tk)
    R.relaybp_set_learned_rows(hb, torch.tensor(wrow, device="cuda"), tk)
    a, b = gpu_decode(ha, syn), gpu_decode(hb, syn)
    for k in ("corrections", "pred_obs", "stats", "weights"):
        assert np.array_equal(a[k], b[k]), k
    R.relaybp_destroy(ha)
    R.relaybp_destroy(hb)


def test_learned_legs_cutoff_matches_oracle():
    """Learned parameters in legs 0..n-1 and plain legs after.  On the GPU,
    bit for bit: a cutoff of 0 is the plain decoder, a cutoff past the last
    leg is the fully learned decoder, and a cutoff of 2 equals the fully
    learned decoder on every shot settled in legs 0 and 1.  Against the
    oracle under the same cutoff: every claimed success is valid and the
    predicted observables agree on >= 99% of shots.  At p = 0.2% about 14% of
    shots run past leg 0, where FP32 and FP64 trajectories part (the iteration
    map amplifies rounding), hence the looser bound than the 99.9% at p = 0.1%."""
    import torch
    from paper_2607_27644_b300 import relaybp as R
    from gpu_util import gpu_decode
    dem = circuit_dem("ZSZ-LP-160", 0.002, 10, "Z")   # about 8% of shots run past leg 1
    kw = dict(num_sets=60, gamma_min=-0.15, gamma_max=0.61, seed=21, stop_nconv=1)
    rng = np.random.default_rng(22)
    T = 8
    w = rng.uniform(0.75, 1.0, (T, dem.n_edges)).astype(np.float32)
    knots = np.cumsum(np.r_[-0.15, rng.uniform(0.02, 0.07, 16)]).astype(np.float32)
    syn, _, _ = oracle.sample(dem, 23, 0, 400)
    hp = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", **kw))
    hl = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", **kw))
    R.relaybp_set_learned(hl, torch.tensor(w, device="cuda"), torch.tensor(knots, device="cuda"))
    keys = ("corrections", "pred_obs", "stats", "weights")
    full = gpu_decode(hl, syn)
    R.relaybp_set_learned_legs(hl, 0)
    a, b = gpu_decode(hp, syn), gpu_decode(hl, syn)
    for k in keys:
        assert np.array_equal(a[k], b[k]), k
    R.relaybp_set_learned_legs(hl, kw["num_sets"] + 1)
    c = gpu_decode(hl, syn)
    for k in keys:
        assert np.array_equal(full[k], c[k]), k
    R.relaybp_set_learned_legs(hl, 2)
    rg = gpu_decode(hl, syn)
    early = (full["stats"][:, 0] == 1) & (full["stats"][:, 2] <= 2)
    for k in keys:
        assert np.array_equal(full[k][early], rg[k][early]), k
    assert (rg["stats"][:, 2] > 2).any()     # shots reached the plain legs
    ro = oracle.decode(dem, oracle.DecodeParams(**kw), syn, w=w.astype(np.float64), knots=knots.astype(np.float64),
                       learned_legs=2)
    Hd = dem.dense_H().astype(np.int64)
    S = unpack_bits(syn, dem.n_det)
    for r in (ro, rg):
        eh = unpack_bits(r["corrections"], dem.n_loc).astype(np.int64)
        conv = r["stats"][:, 0] == 1
        assert np.array_equal((eh[conv] @ Hd.T) % 2, S[conv])
    same = np.all(ro["pred_obs"][:, :rg["pred_obs"].shape[1]] == rg["pred_obs"], axis=1)
    assert (~same).sum() <= len(syn) // 100
    with pytest.raises(RuntimeError):
        R.relaybp_set_learned_legs(hl, -2)
    R.relaybp_destroy(hp)
    R.relaybp_destroy(hl)


def test_trained_parameters_lower_mean_iterations():
    """What training gains, at the same stopping rule: row-tied weights of leg
    0 trained on self-sampled shots of the ZSZ-LP-160 circuit DEM at p = 0.2%
    (soft-syndrome objective over T = 20 iterations at gamma0, from the
    uniform weight that decodes held-out shots in the fewest iterations, 200
    Adam steps of 512 shots, checkpoint selection on 16,384 held-out shots)
    decode 2^17 fresh shots at p = 0.1% -- learned leg 0, plain legs after,
    stop after the first solution -- in at least 5% fewer mean iterations than
    the same decoder with unit weights (the ablation); failures agree within 2
    sigma.  Iterations are clipped at the learned legs' horizon (80 + 60) so a
    shot left to the plain legs counts once; both means are reported."""
    import warnings
    import torch
    from paper_2607_27644_b300 import relaybp as R
    from paper_2607_27644_b300.learned import train_rows
    from paper_2607_27644_b300.stats import agree_within
    from workloads.dem import circuit_dems
    d_inf, d_train = circuit_dems("ZSZ-LP-160", [0.001, 0.002], 10, "Z")
    decoder = dict(gamma0=0.125, pre_iter=80, num_sets=1000, max_iterations=60, stop_nconv=5, gamma_min=-0.15,
                   gamma_max=0.61, seed=24301)
    wrow, knots, info = train_rows(d_inf, d_train, decoder, 200, T=20, leg0=True, select_shots=16384,
                                   warm_start=(1.0, 0.9, 0.85, 0.8, 0.75, 0.7))
    legs = info["learned_legs"]
    horizon = decoder["pre_iter"] + legs * decoder["max_iterations"]
    p1 = R.Params(msg_dtype="f32", **dict(decoder, stop_nconv=1))
    hl, hu = R.relaybp_build_dem(d_inf, p1), R.relaybp_build_dem(d_inf, p1)
    R.relaybp_set_learned_rows(hl, wrow, knots)
    R.relaybp_set_learned_legs(hl, legs)
    N, shot0 = 1 << 17, 3 * 10**9
    syn = torch.empty((N, hl.wc), dtype=torch.int32, device="cuda")
    obs = torch.empty((N, hl.wk), dtype=torch.int32, device="cuda")
    R.relaybp_sample(hl, 7, shot0, N, syn, obs)
    res = {}
    for name, h in (("learned", hl), ("unit", hu)):
        pobs = torch.empty((N, h.wk), dtype=torch.int32, device="cuda")
        st = torch.empty((N, 6), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
        R.relaybp_decode_batch(h, syn, shot0, N, None, pobs, st)
        R.relaybp_count_failures(h, pobs, obs, st, N, cnt)
        it = st[:, 3].double()
        res[name] = (float(it.clamp(max=horizon).mean()), float(it.mean()), int(cnt[3]))
    warnings.warn(UserWarning(
        f"trained vs unit parameters, 2^17 shots, stop after the first solution: mean iterations (clipped) "
        f"{res['learned'][0]:.3f} vs {res['unit'][0]:.3f}, unclipped {res['learned'][1]:.2f} vs {res['unit'][1]:.2f}, "
        f"failures {res['learned'][2]} vs {res['unit'][2]}; warm start {info['warm_start']}; "
        f"kept training step {info['selection'].split()[-1]}"))
    assert res["learned"][0] <= 0.95 * res["unit"][0]
    assert agree_within(res["learned"][2], N, res["unit"][2], N)
    R.relaybp_destroy(hl)
    R.relaybp_destroy(hu)
