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
                 dtype=torch.float32, device="cuda", row_of_edge=None, n_rows: int = 0):
        super().__init__()
        self.row_of_edge = None
        if row_of_edge is not None:
            self.row_of_edge = torch.as_tensor(row_of_edge, dtype=torch.long, device=device)
            self.w = torch.nn.Parameter(torch.ones((T, n_rows), dtype=dtype, device=device))
        else:
            self.w = torch.nn.Parameter(torch.ones((T, n_edges), dtype=dtype, device=device))
        step = (gamma_max - gamma_min) / K
        inv_sp = float(torch.log(torch.expm1(torch.tensor(step, dtype=torch.float64))))
        theta = torch.full((K + 1,), inv_sp, dtype=dtype, device=device)
        theta[0] = gamma_min
        self.theta = torch.nn.Parameter(theta)

    def knots(self):
        return torch.cat([self.theta[:1], self.theta[:1] + torch.cumsum(torch.nn.functional.softplus(self.theta[1:]),
                                                                        0)])

    def edge_weights(self):
        return self.w if self.row_of_edge is None else self.w.index_select(1, self.row_of_edge)

    def loss(self, handle, syndromes, errors, shot0: int, gamma_seed: int, objective: int = 0):
        return LearnedLoss.apply(self.edge_weights().contiguous(), self.knots(), handle, syndromes, errors, shot0,
                                 gamma_seed, objective)
