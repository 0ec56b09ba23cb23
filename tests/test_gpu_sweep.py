"""The gamma-interval grid search and LER sweep (Sec. 6.1, Table 9) through
the CUDA path: GpuDecoder samples and decodes on the device through the C ABI,
and its tallies are compared with the same sweep run with the FP64 oracle as
the decoder on the [[60,12,6]] code's circuit DEMs (2 rounds, both memory
bases).  In FP64 the device decode is the literal-order kernel, so every grid
point's failure tally must be identical; in FP32 the tallies agree within
2 sigma."""
import numpy as np
import pytest

import oracle
from oracle import DecodeParams
from paper_2607_27644_b300.stats import agree_within
from paper_2607_27644_b300.sweep import GpuDecoder, Tally, gamma_grid_search
from workloads.dem import circuit_dems
from workloads.zsz import load_code

pytestmark = pytest.mark.gpu

P = 0.01
KW = dict(gamma0=0.125, pre_iter=30, num_sets=4, max_iterations=20, stop_nconv=2, seed=5)
N = 300
GMIN, GMAX = [-0.24, 0.0], [0.3, 0.66]


class OracleDecoder:
    def run(self, dem, params, shots, shot0=0):
        po = DecodeParams(gamma0=params.gamma0, pre_iter=params.pre_iter, num_sets=params.num_sets,
                          max_iterations=params.max_iterations, stop_nconv=params.stop_nconv,
                          gamma_min=params.gamma_min, gamma_max=params.gamma_max, seed=params.seed)
        syn, obs, _ = oracle.sample(dem, 2, shot0, shots)
        r = oracle.decode(dem, po, syn, shot0=shot0)
        conv = r["stats"][:, 0] == 1
        wrong = np.any(r["pred_obs"][:, :obs.shape[1]] != obs, axis=1)
        return Tally(shots, int((~conv).sum() + (conv & wrong).sum()), int((~conv).sum()), int((conv & wrong).sum()))


@pytest.fixture(scope="module")
def dems60():
    return {"Z": circuit_dems("ZSZ-LP-60", [P], 2, "Z")[0], "X": circuit_dems("ZSZ-LP-60", [P], 2, "X")[0]}


@pytest.fixture(scope="module")
def oracle_sweep(dems60):
    from paper_2607_27644_b300 import relaybp as R
    k = load_code("ZSZ-LP-60").k
    return gamma_grid_search(OracleDecoder(), dems60, R.Params(msg_dtype="f64", **KW), GMIN, GMAX, N, P, 2, k)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_grid_search_through_the_cuda_path(dems60, oracle_sweep, dtype):
    from paper_2607_27644_b300 import relaybp as R
    k = load_code("ZSZ-LP-60").k
    best_o, pts_o = oracle_sweep
    best_g, pts_g = gamma_grid_search(GpuDecoder(batch=128, sample_seed=2), dems60, R.Params(msg_dtype=dtype, **KW),
                                      GMIN, GMAX, N, P, 2, k)
    assert [p.gamma for p in pts_g] == [p.gamma for p in pts_o]
    assert sum(p.pooled.failures for p in pts_o) > 0
    for po_, pg_ in zip(pts_o, pts_g):
        for b in ("X", "Z"):
            to, tg = po_.per_basis[b], pg_.per_basis[b]
            assert tg.shots == to.shots == N and tg.failures == tg.nonconverged + tg.logical
            if dtype == "f64":
                assert vars(tg) == vars(to), (po_.gamma, b)
            else:
                assert agree_within(to.failures, N, tg.failures, N), (po_.gamma, b)
    if dtype == "f64":
        assert best_g.gamma == best_o.gamma
