"""Helpers shared by the GPU tests: run the CUDA path through the C-ABI binding
and bring results back as numpy arrays."""
import numpy as np
import torch

from paper_2607_27644_b300 import relaybp as R


def to_dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def gpu_sample(h, seed, shot0, shots, errors=False):
    syn = torch.zeros((shots, h.wc), dtype=torch.int32, device="cuda")
    obs = torch.zeros((shots, h.wk), dtype=torch.int32, device="cuda")
    err = torch.zeros((shots, h.wv), dtype=torch.int32, device="cuda") if errors else None
    R.relaybp_sample(h, seed, shot0, shots, syn, obs, err)
    torch.cuda.synchronize()
    u = lambda t: None if t is None else t.cpu().numpy().view(np.uint32)
    return u(syn), u(obs), u(err)


def gpu_decode(h, syn_np, shot0=0, trace_iters=0):
    shots = syn_np.shape[0]
    syn = to_dev(syn_np)
    corr = torch.zeros((shots, h.wv), dtype=torch.int32, device="cuda")
    pobs = torch.zeros((shots, h.wk), dtype=torch.int32, device="cuda")
    stats = torch.zeros((shots, 6), dtype=torch.int32, device="cuda")
    trace = None
    if trace_iters:
        trace = torch.full((shots, trace_iters, h.n_loc), float("nan"), dtype=torch.float64, device="cuda")
        R.relaybp_decode_trace(h, syn, shot0, shots, trace_iters, trace, None)
    R.relaybp_decode_batch(h, syn, shot0, shots, corr, pobs, stats)
    torch.cuda.synchronize()
    st = stats.cpu()
    return dict(corrections=corr.cpu().numpy().view(np.uint32), pred_obs=pobs.cpu().numpy().view(np.uint32),
                stats=st[:, :4].numpy().copy(), weights=st.view(torch.float64)[:, 2].numpy().copy(),
                trace=None if trace is None else trace.cpu().numpy())


def params_pair(**kw):
    """The same decoder parameters for the oracle and the CUDA path."""
    import oracle
    dt = kw.pop("msg_dtype", "f32")
    return oracle.DecodeParams(**kw), R.Params(msg_dtype=dt, **kw)
