"""World-size-2 replica runs on CPU (gloo): the sharded counters equal a
one-process run over the same global shot range, shot for shot."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2607_27644_b300.replicas import shot_range, reduce_counters

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _counters(dem, params, seed, shot0, n):
    import oracle
    syn, obs, _ = oracle.sample(dem, seed, shot0, n)
    r = oracle.decode(dem, params, syn, shot0=shot0, n_threads=1)
    conv = r["stats"][:, 0] == 1
    logical = conv & np.any(r["pred_obs"] != obs, axis=1)
    return np.array([n, (~conv).sum(), logical.sum(), (~conv).sum() + logical.sum()], dtype=np.int64)


def _worker(rank, world, port, steps, batch, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from workloads.dem import code_capacity_dem
    dem = code_capacity_dem("ZSZ-LP-60", 0.08)
    p = oracle.DecodeParams(num_sets=5, seed=3)
    acc = np.zeros(4, dtype=np.int64)
    for k in range(steps):
        s0, n = shot_range(rank, world, steps, batch, k)
        acc += _counters(dem, p, 17, s0, n)
    c, t = reduce_counters(torch.from_numpy(acc), 1.0 + rank)
    if rank == 0:
        out.put((c.numpy().tolist(), t))
    dist.destroy_process_group()


def test_shot_ranges_partition():
    seen = []
    for r in range(3):
        for k in range(4):
            s0, n = shot_range(r, 3, 4, 10, k)
            seen.extend(range(s0, s0 + n))
    assert sorted(seen) == list(range(120))
    with pytest.raises(ValueError):
        shot_range(3, 3, 4, 10, 0)


def test_two_rank_counters_match_single_process():
    import oracle
    from workloads.dem import code_capacity_dem
    oracle.build()
    world, steps, batch = 2, 3, 40
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, steps, batch, q)) for r in range(world)]
    for p in procs:
        p.start()
    c, t = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    dem = code_capacity_dem("ZSZ-LP-60", 0.08)
    ref = _counters(dem, oracle.DecodeParams(num_sets=5, seed=3), 17, 0, world * steps * batch)
    assert c == ref.tolist()
    assert t == 2.0
