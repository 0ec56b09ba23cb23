"""Learned Relay-BP: trainable message weights and memory-strength distribution.

Not in arXiv 2607.27644 (which decodes with plain Relay-BP).  The model:
per-iteration, per-edge weights w[t][e] on the min-sum check-to-variable
messages and a monotone piecewise-linear inverse CDF of the memory strength
(K segments) in place of the uniform interval.  The loss, summed over T
unrolled iterations of one memory-BP leg, is the binary cross-entropy of the
posteriors against the sampled errors (objective 0) or the soft syndrome
(objective 1: -log of the probability that each check holds its syndrome bit
under the posteriors, which rewards settling early); forward and backward run
in the library's CUDA kernels (relaybp_learned_forward / _backward), wrapped
here in a torch.autograd.Function so torch optimisers can train the
parameters.  Decoding applies the weights to the first T iterations of each
learned leg and unit weights after them.
"""
from __future__ import annotations

import torch

from . import relaybp as R


class LearnedLoss(torch.autograd.Function):
    """loss = mean over shots of the summed per-iteration objective."""

    @staticmethod
    def forward(ctx, w, knots, handle, syndromes, errors, shot0: int, gamma_seed: int, objective: int = 0):
        shots = syndromes.shape[0]
        T = w.shape[0]
        prec = R._prec(w.dtype)
        tape = torch.empty(R.relaybp_learned_tape_bytes(handle, prec, T, shots), dtype=torch.uint8,
                           device=w.device)
        loss = torch.empty(shots, dtype=torch.float64, device=w.device)
        R.relaybp_learned_forward(handle, w, knots, gamma_seed, syndromes, errors, shot0, shots, tape, loss,
                                  objective=objective)
        ctx.save_for_backward(w, knots, syndromes, errors, tape)
        ctx.meta = (handle, shot0, gamma_seed, shots, objective)
        return loss.mean().to(w.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        w, knots, syndromes, errors, tape = ctx.saved_tensors
        handle, shot0, gamma_seed, shots, objective = ctx.meta
        gw = torch.zeros_like(w)
        gk = torch.zeros_like(knots)
        scale = float(grad_out.item()) / shots
        R.relaybp_learned_backward(handle, w, knots, gamma_seed, errors, shot0, shots, tape, scale, gw, gk,
                                   objective=objective, d_syndromes=syndromes)
        return gw, gk, None, None, None, None, None, None


class LearnedParams(torch.nn.Module):
    """Message weights initialised to 1 and knots from raw parameters kept
    monotone: knots[0] = theta[0], knots[k+1] = knots[k] + softplus(theta[k+1]);
    initialised to the uniform interval [gamma_min, gamma_max].

    Weights are per edge ([T, E]) or, with row_of_edge given, tied per check
    row ([T, C], expanded to edges for the loss) -- the form the decode kernel
    applies at no extra memory traffic (relaybp_set_learned_rows)."""

    def __init__(self, T: int, n_edges: int, gamma_min: float, gamma_max: float, K: int = 16,
                 dtype=torch.float32, device="cuda", row_of_edge=None, n_rows: int = 0,
                 fixed_gamma: float | None = None):
        super().__init__()
        self.row_of_edge = None
        if row_of_edge is not None:
            self.row_of_edge = torch.as_tensor(row_of_edge, dtype=torch.long, device=device)
            self.w = torch.nn.Parameter(torch.ones((T, n_rows), dtype=dtype, device=device))
        else:
            self.w = torch.nn.Parameter(torch.ones((T, n_edges), dtype=dtype, device=device))
        # fixed_gamma: every variable takes this strength (two equal knots, not
        # trained) -- the unrolled leg is then leg 0, which runs at gamma0
        self.theta = None
        if fixed_gamma is not None:
            self.register_buffer("fixed_knots", torch.full((2,), fixed_gamma, dtype=dtype, device=device))
            return
        step = (gamma_max - gamma_min) / K
        inv_sp = float(torch.log(torch.expm1(torch.tensor(step, dtype=torch.float64))))
        theta = torch.full((K + 1,), inv_sp, dtype=dtype, device=device)
        theta[0] = gamma_min
        self.theta = torch.nn.Parameter(theta)

    def knots(self):
        if self.theta is None:
            return self.fixed_knots
        return torch.cat([self.theta[:1], self.theta[:1] + torch.cumsum(torch.nn.functional.softplus(self.theta[1:]),
                                                                        0)])

    def edge_weights(self):
        return self.w if self.row_of_edge is None else self.w.index_select(1, self.row_of_edge)

    def loss(self, handle, syndromes, errors, shot0: int, gamma_seed: int, objective: int = 0):
        return LearnedLoss.apply(self.edge_weights().contiguous(), self.knots(), handle, syndromes, errors, shot0,
                                 gamma_seed, objective)


def train_rows(d_inf, d_train, decoder: dict, steps: int, T: int = 10, lr: float = 3e-3, objective: int = 1,
               device="cuda", batch: int = 512, select_shots: int = 8192, learned_legs: int = 50,
               sample_seed: int = 4, select_seed: int = 5, leg0: bool = False,
               warm_start: tuple | None = None):
    """Train row-tied message weights [T, C] and memory-strength knots on
    self-sampled shots of d_train (the training DEM: the same detectors and
    faults as d_inf at another noise strength) with the library's forward and
    backward kernels and Adam.  leg0=True trains the weights of leg 0 alone:
    the unrolled leg runs at the decoder's gamma0 for every variable, as leg 0
    does, the knots stay at gamma0 (two equal knots, not trained) and
    learned_legs is 1, so every later leg is the plain method.  warm_start, a
    tuple of candidate values, starts the gradient steps from the uniform
    weight among them (every row and iteration alike) that decodes the
    held-out shots below in the fewest mean iterations -- a one-parameter fit
    on the decoding objective, which the per-row gradient steps then refine.
    Every 25 steps the current parameters decode
    select_shots held-out shots of d_inf (stop after the first solution,
    learned legs 0..learned_legs-1, plain legs after), and the checkpoint with
    the fewest mean iterations -- clipped at the learned legs' horizon, so a
    shot left to the plain legs counts once -- is kept; step 0 (unit weights
    and the uniform interval, or the warm start, whose candidates include 1)
    is a candidate, so the result never decodes slower than no training on
    that sample.  decoder: Relay-BP parameters (Params
    fields).  Returns (wrow, knots, info) with wrow and knots FP32 device
    tensors for relaybp_set_learned_rows."""
    import numpy as np
    import time
    from . import relaybp as R
    dev = torch.device(device) if isinstance(device, str) else device
    E = d_inf.n_edges
    DECODER = dict(decoder)
    # T unrolled iterations (default 10: summed over 30 the losses are
    # dominated by iterations past the map's chaotic horizon, where marginals
    # grow without bound; over 10 they train steadily)
    BT = batch
    # ---- training (untimed) ---------------------------------------------------
    ht = R.relaybp_build_dem(d_train, R.Params(msg_dtype="f32", **DECODER))
    row_of = np.repeat(np.arange(d_inf.n_det), np.diff(d_inf.H_indptr))
    if leg0:
        learned_legs = 1
    model = LearnedParams(T, E, DECODER["gamma_min"], DECODER["gamma_max"], device=dev, row_of_edge=row_of,
                          n_rows=d_inf.n_det, fixed_gamma=float(DECODER.get("gamma0", 0.125)) if leg0 else None)
    opt = torch.optim.Adam(model.parameters(), lr=lr)
    syn_t = torch.empty((BT, ht.wc), dtype=torch.int32, device=dev)
    err_t = torch.empty((BT, ht.wv), dtype=torch.int32, device=dev)
    syn_v = torch.empty((2 * BT, ht.wc), dtype=torch.int32, device=dev)
    err_v = torch.empty((2 * BT, ht.wv), dtype=torch.int32, device=dev)
    R.relaybp_sample(ht, sample_seed, 9 * 10**8, 2 * BT, syn_v, None, err_v)     # held-out shots
    # model selection on the decoding objective: every 25 steps the current
    # parameters decode held-out shots of the inference DEM (stop after the
    # first solution, learned legs only); the checkpoint with the fewest mean
    # iterations is kept.  Step 0 (unit weights, uniform gamma) is a
    # candidate, so selection never keeps parameters slower than no training.
    NSEL, SEL0 = select_shots, 8 * 10**8
    hsel = R.relaybp_build_dem(d_inf, R.Params(msg_dtype="f32", **dict(DECODER, stop_nconv=1)))
    syn_s = torch.empty((NSEL, hsel.wc), dtype=torch.int32, device=dev)
    st_s = torch.empty((NSEL, 6), dtype=torch.int32, device=dev)
    R.relaybp_sample(hsel, select_seed, SEL0, NSEL, syn_s, None, None)
    t0 = time.perf_counter()
    hist, sel_hist, best, best_state, best_step = [], [], float("inf"), None, 0

    def held_out():
        with torch.no_grad():
            return float(model.loss(ht, syn_v, err_v, 9 * 10**8, 0x5EED, objective))

    def held_out_iterations():
        with torch.no_grad():
            w_ = model.w.detach().float().contiguous()          # the handle keeps these pointers:
            k_ = model.knots().detach().float().contiguous()    # hold them until the decode is read
            R.relaybp_set_learned_rows(hsel, w_, k_)
            R.relaybp_set_learned_legs(hsel, learned_legs)
            R.relaybp_decode_batch(hsel, syn_s, SEL0, NSEL, None, None, st_s)
            # iterations clipped at the learned legs' horizon: a shot left to
            # the plain legs counts once, not by its full run
            horizon = DECODER["pre_iter"] + learned_legs * DECODER["max_iterations"]
            it = float(st_s[:, 3].clamp(max=horizon).double().mean())
            del w_, k_
            return it

    def checkpoint(k):
        nonlocal best, best_state, best_step
        hist.append(round(held_out(), 3))
        it = held_out_iterations()
        sel_hist.append(round(it, 3))
        if it < best:
            best, best_step = it, k
            best_state = {n: t.detach().clone() for n, t in model.state_dict().items()}

    warm = None
    if warm_start:
        scores = {}
        with torch.no_grad():
            for v in warm_start:
                model.w.fill_(float(v))
                scores[float(v)] = round(held_out_iterations(), 3)
            v_best = min(scores, key=scores.get)     # first of equal scores
            model.w.fill_(v_best)
        warm = {"candidates": scores, "chosen": v_best}
    checkpoint(0)
    for k in range(steps):
        R.relaybp_sample(ht, sample_seed, k * BT, BT, syn_t, None, err_t)
        opt.zero_grad()
        loss = model.loss(ht, syn_t, err_t, k * BT, 0x5EED, objective)
        loss.backward()
        torch.nn.utils.clip_grad_norm_(model.parameters(), 1.0)
        opt.step()
        with torch.no_grad():
            model.w.clamp_(0.0, 2.0)
        if (k + 1) % 25 == 0 or k == steps - 1:
            checkpoint(k + 1)
    model.load_state_dict(best_state)
    R.relaybp_destroy(hsel)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    wrow = model.w.detach().float().contiguous()
    knots = model.knots().detach().float().contiguous()
    info = {"steps": steps, "batch": BT, "shots": steps * BT, "unrolled_iterations": T,
            "learned_legs": learned_legs,
            "memory_strength": (f"leg 0 only: gamma0 = {float(DECODER.get('gamma0', 0.125)):g} in training, plain "
                                f"legs after" if leg0 else "learned knots in legs 1..learned_legs-1"),
            "objective": ["cross-entropy against the sampled error", "soft syndrome"][objective],
            "optimizer": f"Adam {lr:g}, grad-norm clip 1, weights in [0, 2]",
            "weights": "tied per check row and iteration; unit past the trained horizon", "seconds": train_s,
            "warm_start": warm,
            "held_out_loss_every_25_steps": hist, "held_out_mean_iterations_every_25_steps": sel_hist,
            "selection": f"fewest held-out mean iterations, clipped at the learned legs' horizon ({NSEL} shots of "
                         f"the inference DEM, stop after the first solution); kept step {best_step}"}
    R.relaybp_destroy(ht)
    return wrow, knots, info
