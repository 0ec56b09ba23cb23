"""Benchmark: decoded shots/s of batched Relay-BP at p = 0.1% circuit noise.

Workload (the configuration the metric is quoted on): ZSZ-LP-160, Table 10
syndrome-extraction schedule, d = 10 rounds, Z-memory, idling-free
depolarising circuit noise p = 0.001 (DEM 704 detectors x 10,400 faults), the
paper's decoder settings (gamma0 0.125, pre_iter 80, num_sets 1000,
max_iterations 60, stop_nconv 5, FP32 messages) with the ZSZ-LP-160 gamma
interval [-0.15, 0.61] of Table 9; 10^6 shots per run (steps x batch).

A step is one pass of the hot path over one batch: Philox fault sampling
(s = H e, obs = O e), the persistent Relay-BP decode, and failure accounting.

Arms:
  default           the CUDA path (inputs resident on the device when timing
                    starts; `e2e` repeats the decode through the host-buffer
                    entry point with the copies inside the timed region)
  --impl reference  the FP64 CPU oracle on the host cores, on a bounded sample
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(code="ZSZ-LP-160", rounds=10, basis="Z", p=0.001)
DECODER = dict(gamma0=0.125, pre_iter=80, num_sets=1000, max_iterations=60, stop_nconv=5,
               gamma_min=-0.15, gamma_max=0.61, seed=0x5EED)
METRIC = "decoded shots/s at p=0.1% circuit noise, learned vs plain Relay-BP at equal LER"
SAMPLE_SEED = 2


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=125_000, help="shots per step and per GPU")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=96, help="shots of the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--streams", type=int, default=3, help="zsz160: streams (handle sets) the steps rotate over")
    ap.add_argument("--workload", default="zsz160",
                    choices=["zsz160", "mixed", "learned", "stream550", "gamma_sweep", "latency"],
                    help="zsz160: the headline workload; mixed: nine DEMs in one persistent launch; "
                         "learned: train, then learned vs plain Relay-BP at equal LER; stream550: ZSZ-LP-550 "
                         "d=18 in CUDA-graph batches with int8 storage and per-shot latency; gamma_sweep: "
                         "Table 9's gamma-interval grid search and the XZ-averaged LER-vs-p curve; latency: "
                         "Table 5's single-shot latency of ZSZ-LP-320/390/550, one thread-block cluster per shot")
    ap.add_argument("--latency-shots", type=int, default=2000, help="latency: timed shots per code and basis")
    ap.add_argument("--latency-max-shots", type=int, default=5,
                    help="latency: shots per code and basis timed with every relay leg run (max latency)")
    ap.add_argument("--cluster", type=int, default=16, help="latency: CTAs per thread-block cluster")
    ap.add_argument("--tail-legs", type=int, default=50,
                    help="zsz160: hand shots about to start this relay leg to cluster-kernel launches (0: off)")
    ap.add_argument("--tail-cluster", type=int, default=8, help="zsz160: CTAs per cluster of the tail offload")
    ap.add_argument("--sweep-shots", type=int, default=200_000, help="gamma_sweep: shots per point and basis")
    ap.add_argument("--stream-batch", type=int, default=1 << 16, help="stream550: shots per graph batch")
    ap.add_argument("--train-steps", type=int, default=300, help="learned: Adam steps of 512 shots at p=0.2%%")
    ap.add_argument("--learned-msg", default="bf16", choices=["bf16", "f16", "f32"], help="learned: message storage")
    ap.add_argument("--objective", type=int, default=1, choices=[0, 1],
                    help="learned: training loss, 0 cross-entropy against the sampled error, 1 soft syndrome")
    ap.add_argument("--train-T", type=int, default=20, help="learned: unrolled iterations of training")
    ap.add_argument("--learned-legs", default="leg0", choices=["leg0", "legs50"],
                    help="learned: weights in leg 0 trained at gamma0 with plain legs after (leg0), or weights and "
                         "memory-strength knots in legs 0-49 (legs50)")
    ap.add_argument("--warm-start", default="1,0.9,0.85,0.8,0.75,0.7",
                    help="learned: candidate uniform weights for the warm start ('' for none)")
    ap.add_argument("--learned-steps", type=int, default=16,
                    help="default workload: timed steps of the learned arm and of its ablation")
    ap.add_argument("--train-lr", type=float, default=3e-3, help="learned: Adam learning rate")
    ap.add_argument("--no-learned", action="store_true", help="default workload: skip the learned and ablation arms")
    ap.add_argument("--learned-train-steps", type=int, default=300,
                    help="default workload: Adam steps of 512 shots training the learned arm")
    ap.add_argument("--mixed-base", type=int, default=2000, help="mixed: shots per unit of the 2:5:10 mix")
    ap.add_argument("--msg", default=None, choices=["f16", "bf16", "f32", "i8"],
                    help="message storage (default: f32 for zsz160, f16 for mixed)")
    return ap.parse_args()


def _measured_peaks():
    """HBM copy bandwidth and bf16 GEMM peaks measured on this GPU type
    (MEASURED_PEAKS.json beside this file), or {} when absent."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _dem():
    from workloads.dem import circuit_dem
    return circuit_dem(WORKLOAD["code"], WORKLOAD["p"], WORKLOAD["rounds"], WORKLOAD["basis"])


def _config(dem, batch, steps, world, extra=None, streams=3):
    c = {"workload": f"{WORKLOAD['code']} circuit-level Z-memory, d={WORKLOAD['rounds']}, p={WORKLOAD['p']}, "
                     f"DEM {dem.n_det}x{dem.n_loc} (E={dem.n_edges}), plain Relay-BP",
         "decoder": dict(DECODER), "shots_per_step_per_gpu": batch, "steps": steps,
         "shots_total": batch * steps * world,
         "l2": "flushed before every step on that step's stream (256 MiB write)",
         "parallelism": f"replicas x{world} (shot ranges); steps rotate over {streams} streams, one handle each"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _cpu_baseline(dem, n_shots):
    import numpy as np
    import oracle
    syn, _, _ = oracle.sample(dem, SAMPLE_SEED, 10**9, n_shots)
    p = oracle.DecodeParams(**DECODER)
    t0 = time.perf_counter()
    oracle.decode(dem, p, syn, shot0=10**9)
    dt = time.perf_counter() - t0
    return n_shots / dt, dt, oracle.max_threads()


def run_reference(a):
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle
    dem = _dem()
    syn, _, _ = oracle.sample(dem, SAMPLE_SEED, 0, a.cpu_sample * (a.steps + a.warmup))
    p = oracle.DecodeParams(**DECODER)
    n = a.cpu_sample
    for w in range(a.warmup):
        oracle.decode(dem, p, syn[w * n:(w + 1) * n], shot0=w * n)
    t0 = time.perf_counter()
    for k in range(a.steps):
        b = (a.warmup + k) * n
        oracle.decode(dem, p, syn[b:b + n], shot0=b)
    dt = time.perf_counter() - t0
    v = n * a.steps / dt
    cores = oracle.max_threads()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "shots/s", "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (Philox-sampled syndromes of the circuit DEM)",
            "config": _config(dem, n, a.steps, 1, {"arm": "FP64 CPU oracle, OpenMP over shots",
                                                    "l2": "n/a (host CPU)",
                                                    "parallelism": f"{cores} host threads over the shots of a step",
                                                    "sample": f"{n} shots per step, a bounded sample of the "
                                                              "workload"}),
            "cpu_baseline": {"value": v, "unit": "shots/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} shots per step x {a.steps} steps"},
            "e2e": {"value": v, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2607_27644_b300 import relaybp as R

    rank, world, local = _dist()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dem = _dem()
    # Handles on several streams, steps rotating over them: the rare shot that
    # runs all relay legs overlaps the next batches instead of idling the GPU at
    # the end of its launch.  (Each handle owns its work counter, so launches
    # may overlap.)
    NS = max(1, a.streams)
    msg = a.msg or "f32"
    hs = [R.relaybp_build_dem(dem, R.Params(msg_dtype=msg, **DECODER)) for _ in range(NS)]
    h = hs[0]
    tail = a.tail_legs if msg == "f32" else 0
    for x in hs:
        if tail:
            R.relaybp_set_tail_offload(x, tail, a.tail_cluster, 256)
    B, K, W = a.batch, a.steps, a.warmup
    streams = [torch.cuda.Stream(device=dev) for _ in range(NS)]
    st = streams[0]
    bufs = [dict(syn=torch.empty((B, h.wc), dtype=torch.int32, device=dev),
                 obs=torch.empty((B, h.wk), dtype=torch.int32, device=dev),
                 pobs=torch.empty((B, h.wk), dtype=torch.int32, device=dev),
                 stats=torch.empty((B, 6), dtype=torch.int32, device=dev)) for _ in range(NS)]
    syn, obs, pobs, stats = bufs[0]["syn"], bufs[0]["obs"], bufs[0]["pobs"], bufs[0]["stats"]
    counters = torch.zeros(4, dtype=torch.int64, device=dev)
    # per-stream iteration sums: an in-place add on one element from several
    # streams at once would lose updates
    iters_total = torch.zeros(NS, dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.int32, device=dev)
    from paper_2607_27644_b300.replicas import shot_range, reduce_counters

    def step(k, dec_events=None):
        q = k % NS
        s_, b_, h_ = streams[q], bufs[q], hs[q]
        shot0, _ = shot_range(rank, world, K + W, B, k)
        with torch.cuda.stream(s_):
            flush.fill_(k)                      # evict L2 before each step (256 MiB write)
            R.relaybp_sample(h_, SAMPLE_SEED, shot0, B, b_["syn"], b_["obs"], None, s_)
            if dec_events:
                dec_events[0].record(s_)
            R.relaybp_decode_batch(h_, b_["syn"], shot0, B, None, b_["pobs"], b_["stats"], s_)
            if dec_events:
                dec_events[1].record(s_)
            R.relaybp_count_failures(h_, b_["pobs"], b_["obs"], b_["stats"], B, counters, s_)
            iters_total[q:q + 1].add_(b_["stats"][:, 3].sum())

    def join():
        for s_ in streams[1:]:
            streams[0].wait_stream(s_)

    for w in range(W):
        step(K + w)
    torch.cuda.synchronize()
    counters.zero_()
    iters_total.zero_()
    dec_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = sum(R.relaybp_launch_count(x) for x in hs)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start.record(streams[0])
        for s_ in streams[1:]:
            s_.wait_stream(streams[0])
        for k in range(K):
            step(k, dec_ev[k])
        join()
        t_end.record(streams[0])
        torch.cuda.synchronize()
    launches = sum(R.relaybp_launch_count(x) for x in hs) - l0
    if world > 1:
        dist.barrier()
    ms = t_start.elapsed_time(t_end)
    dec_ms = [e0.elapsed_time(e1) for e0, e1 in dec_ev]
    cnt, ms_max = reduce_counters(torch.cat([counters, iters_total.sum().reshape(1)]), ms)
    cnt = cnt[:4]
    shots_total = B * K * world
    value = shots_total / (ms_max / 1e3)

    # ---- end to end from pinned host memory --------------------------------
    # Every step: host -> device copy of that step's syndromes (pinned), decode,
    # device -> host copy of the predicted observables and per-shot stats, on the
    # same rotating streams as the device-resident run; the host clock spans
    # the whole loop up to the last copy landing in host memory.  The single
    # synchronous call (relaybp_decode_host, one step at a time) is reported
    # beside it.
    e2e = None
    if not a.no_e2e:
        hsyn = []
        with torch.cuda.stream(st):
            for k in range(K):
                R.relaybp_sample(h, SAMPLE_SEED, shot_range(rank, world, K + W, B, k)[0], B, syn, obs, None, st)
                t = torch.empty((B, h.wc), dtype=torch.int32, pin_memory=True)
                t.copy_(syn, non_blocking=False)
                hsyn.append(t)
        hpobs = [torch.empty((B, h.wk), dtype=torch.int32, pin_memory=True) for _ in range(K)]
        hstats = [torch.empty((B, 6), dtype=torch.int32, pin_memory=True) for _ in range(K)]
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for k in range(K):
            q = k % NS
            s_, b_, h_ = streams[q], bufs[q], hs[q]
            with torch.cuda.stream(s_):
                b_["syn"].copy_(hsyn[k], non_blocking=True)
                R.relaybp_decode_batch(h_, b_["syn"], shot_range(rank, world, K + W, B, k)[0], B, None, b_["pobs"],
                                       b_["stats"], s_)
                hpobs[k].copy_(b_["pobs"], non_blocking=True)
                hstats[k].copy_(b_["stats"], non_blocking=True)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        # the synchronous host-buffer call, one step
        hp = torch.empty((B, h.wk), dtype=torch.int32, pin_memory=True)
        hstat = torch.empty((B, 6), dtype=torch.int32, pin_memory=True)
        t1 = time.perf_counter()
        R.relaybp_decode_host(h, hsyn[0], shot_range(rank, world, K + W, B, 0)[0], B, hp, hstat, st)
        sync_s = time.perf_counter() - t1
        _, e2e_max = reduce_counters(torch.zeros(1, dtype=torch.int64, device=dev), e2e_s)
        e2e = {"value": shots_total / e2e_max, "unit": "shots/s", "h2d_bytes_per_step": B * h.wc * 4,
               "d2h_bytes_per_step": B * (h.wk * 4 + 24),
               "path": f"pinned host syndromes -> device -> relaybp_decode_batch -> host predicted observables + "
                       f"per-shot stats, steps rotating over {NS} streams, host clock to the last copy",
               "sync_call_shots_per_s": B / sync_s,
               "sync_call": "relaybp_decode_host, one step, synchronous (copies and decode in one call)"}

    # ---- the metric's learned side: learned vs plain at equal LER ----------
    # Row-tied weights trained here (soft-syndrome objective, p = 0.2%,
    # untimed; by default leg 0's weights at gamma0 from a one-parameter warm
    # start), then --learned-steps batches of fresh shots -- the plain arm's
    # shots first -- decoded by (i) the learned decoder -- learned legs, then
    # plain legs in the same launch, stop after the first solution -- and (ii)
    # the ablation, plain Relay-BP with the same stop-after-first rule:
    # learned vs ablation is what the trained parameters gain, learned vs
    # plain also counts the stopping rule.  FP32, two-shot kernel, same
    # streams.
    learned = None
    if not a.no_learned and world == 1:
        from paper_2607_27644_b300.stats import agree_within
        from workloads.dem import circuit_dems
        d_train = circuit_dems(WORKLOAD["code"], [0.002], WORKLOAD["rounds"], WORKLOAD["basis"])[0]
        wrow, knots, info = train_learned(a, dev, dem, d_train, a.learned_train_steps)
        arm = {}
        KL = max(1, a.learned_steps)
        for kind in ("learned", "ablation"):
            hk = []
            for q in range(NS):
                x = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", **dict(DECODER, stop_nconv=1)))
                if kind == "learned":
                    R.relaybp_set_learned_rows(x, wrow, knots)
                    R.relaybp_set_learned_legs(x, info["learned_legs"])
                if tail:                        # past the learned legs, both arms alike
                    R.relaybp_set_tail_offload(x, max(tail, 50), a.tail_cluster, 256)
                hk.append(x)
            cnt_k = torch.zeros(4, dtype=torch.int64, device=dev)
            it_k = torch.zeros(NS, dtype=torch.int64, device=dev)       # per stream

            def astep(k):
                q = k % NS
                s_, b_, h_ = streams[q], bufs[q], hk[q]
                shot0, _ = shot_range(rank, world, KL + W, B, k)
                with torch.cuda.stream(s_):
                    flush.fill_(k)
                    R.relaybp_sample(h_, SAMPLE_SEED, shot0, B, b_["syn"], b_["obs"], None, s_)
                    R.relaybp_decode_batch(h_, b_["syn"], shot0, B, None, b_["pobs"], b_["stats"], s_)
                    R.relaybp_count_failures(h_, b_["pobs"], b_["obs"], b_["stats"], B, cnt_k, s_)
                    it_k[q:q + 1].add_(b_["stats"][:, 3].sum())

            for w_ in range(W):
                astep(KL + w_)
            torch.cuda.synchronize()
            cnt_k.zero_()
            it_k.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with ClockSampler(local) as clk_k:
                e0.record(streams[0])
                for s_ in streams[1:]:
                    s_.wait_stream(streams[0])
                for k in range(KL):
                    astep(k)
                join()
                e1.record(streams[0])
                torch.cuda.synchronize()
            ms_k = e0.elapsed_time(e1)
            ck = cnt_k.cpu().tolist()
            arm[kind] = {"value": B * KL / (ms_k / 1e3), "unit": "shots/s", "shots": ck[0], "failures": ck[3],
                         "nonconverged": ck[1], "logical": ck[2], "block_ler": ck[3] / max(1, ck[0]),
                         "mean_iterations": float(it_k.sum().item()) / (B * KL), "clocks": clk_k.summary()}
            for x in hk:
                R.relaybp_destroy(x)
        cp = cnt.cpu().tolist()
        lv, ab = arm["learned"], arm["ablation"]
        learned = dict(lv)
        learned.update({
            "decoder": ("FP32; learned row-tied weights in the first T iterations of leg 0 (unit after), plain legs "
                        "after in the same launch" if info["learned_legs"] == 1 else
                        "FP32; learned row-tied weights (first T iterations of a leg, unit after) and memory-strength "
                        "knots in legs 0-49, plain legs after in the same launch") + "; stop after the first solution",
            "ablation": ab, "train": info,
            "speedup_vs_plain": lv["value"] / value, "speedup_vs_ablation": lv["value"] / ab["value"],
            "mean_iterations_vs_ablation": lv["mean_iterations"] / ab["mean_iterations"],
            "equal_ler_2sigma_vs_plain": bool(agree_within(lv["failures"], lv["shots"], cp[3], cp[0])),
            "equal_ler_2sigma_vs_ablation": bool(agree_within(lv["failures"], lv["shots"], ab["failures"],
                                                              ab["shots"])),
            "note": f"{KL} batches of {B} shots, the plain arm's first; speedup_vs_plain mostly measures the stopping rule (first solution "
                    "vs five), speedup_vs_ablation and mean_iterations_vs_ablation what the trained parameters "
                    "gain at the same rule"})

    # ---- roofline of the dominant kernel (relay_decode_kernel) --------------
    sink = torch.zeros(4096, dtype=torch.float32, device=dev)
    with torch.cuda.stream(st):
        reps = 1 << 14
        for _ in range(2):
            R.relaybp_probe_smem_read(reps, sink, st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        nb = 0.0
        for _ in range(5):
            nb += R.relaybp_probe_smem_read(reps, sink, st)
        e1.record(st)
        torch.cuda.synchronize()
    smem_gbs = nb / (e0.elapsed_time(e1) / 1e3) / 1e9
    iters_rank = int(iters_total.sum().item())
    wall_s = ms / 1e3
    E, V, C = dem.n_edges, dem.n_loc, dem.n_det
    b_m = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2, "i8": 1}[msg]
    bytes_per_iter = 4 * b_m * E + 16 * V + (V + C) / 8.0
    dec_avg_s = sum(dec_ms) / len(dec_ms) / 1e3
    per_launch = (iters_rank / K) * bytes_per_iter / dec_avg_s / 1e9
    achieved = iters_rank * bytes_per_iter / wall_s / 1e9
    edge_updates = iters_rank * E / wall_s
    hbm_gbs = _measured_peaks().get("hbm_gbs")
    # DRAM bytes (read + write) of one 3,000-shot decode launch of the two-shot
    # kernel (ncu, same kernel build), scaled by shots to one launch of this
    # run: the state stays on chip; DRAM carries syndromes in, results out and
    # the L2 write-backs of the per-block memory-strength rows
    # DRAM bytes of one two-shot-kernel launch of 3,000 shots (ncu capture of
    # this build), scaled to the step's shots
    traffic = (4205056 + 4014080) * B / 3000 if (msg == "f32" and B >= 3000) else None
    roof = {"bound": "smem", "achieved": achieved, "peak": smem_gbs, "unit": "GB/s", "frac": achieved / smem_gbs,
            "traffic": traffic,
            "kernel": (("relay_pair_kernel<23> (two shots per block, FP32)"
                        + (f"; shots reaching relay leg {tail} finish in relay_cluster_kernel ({a.tail_cluster} "
                           "CTAs per shot)" if tail else "")) if msg == "f32"
                       else f"relay_decode_kernel<{msg}>"),
            "algorithmic_bytes": f"per shot-iteration 4*b_m*E + 16*V + (V+C)/8 (b_m={b_m})",
            "peak_source": "measured live: conflict-free 16-B shared-memory loads on all SMs (relaybp_probe_smem_read)",
            "achieved_basis": f"algorithmic bytes of all decode launches / the timed region ({NS} launches in flight "
                              "at once; the decode kernels fill >99.7% of device time in the serialised ncu launch "
                              "list of this command with 2 steps: two-shot kernel 73.4%, cluster kernel of the "
                              "handed-over shots 26.3%)",
            "achieved_per_launch": per_launch, "decode_ms_per_launch": dec_avg_s * 1e3,
            "edge_updates_per_s": edge_updates,
            "hbm_equivalent": ({"peak_gbs": hbm_gbs, "frac": achieved / hbm_gbs,
                                "note": "the same algorithmic bytes against the measured HBM copy bandwidth: the "
                                        "bound a layout with messages in HBM would face"} if hbm_gbs else None),
            "mean_iterations_per_shot": iters_rank / (B * K)}
    c = cnt.cpu().tolist()
    line = {"metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": msg, "data": "synthetic: Philox-sampled faults of the ZSZ-LP-160 circuit DEM (no dataset)",
            "config": _config(dem, B, K, world, streams=NS, extra={
                "tail_offload": ({"legs": tail, "cluster_ctas": a.tail_cluster,
                                  "note": "shots about to start this relay leg finish on thread-block clusters "
                                          "(bit-identical outputs)"} if tail else None)}), "clocks": clk.summary(), "gpu_launches": launches * world,
            "roofline": roof, "e2e": e2e,
            "ler": {"shots": c[0], "failures": c[3], "nonconverged": c[1], "logical": c[2],
                    "block_ler": c[3] / max(1, c[0])},
            "learned": learned}
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        v, dt, cores = _cpu_baseline(dem, a.cpu_sample)
        line["cpu_baseline"] = {"value": v, "unit": "shots/s", "cores": cores, "kind": "oracle",
                                "sample": f"{a.cpu_sample} shots of the same workload ({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    for x in hs:
        R.relaybp_destroy(x)
    if world > 1:
        dist.destroy_process_group()


# Mixed workload: ZSZ-LP-320/390/550 (d = 14/16/18, Table 5 DEMs) at
# p in {0.1, 0.2, 0.3}% with each code's Table 9 gamma interval and the
# paper's other decoder settings; per step the DEMs get 2:5:10 x base shots in
# round-robin order (the 2x10^5 .. 10^6 spread of the workload, scaled).
MIXED_CODES = [("ZSZ-LP-320", 14, (-0.16, 0.66)), ("ZSZ-LP-390", 16, (-0.16, 0.7)),
               ("ZSZ-LP-550", 18, (-0.12, 0.62))]
MIXED_P = [0.001, 0.002, 0.003]
MIXED_RATIO = [2, 5, 10]


def _tail_offload(R, handles, a):
    """Tail offload on every handle (--tail-legs, --tail-cluster; the next
    larger cluster where a DEM's slice does not fit shared memory); the
    setting reported in the JSON line, or None."""
    if a.tail_legs <= 0:
        return None
    used = set()
    for x in handles:
        for nc in (a.tail_cluster, 16):
            try:
                R.relaybp_set_tail_offload(x, a.tail_legs, nc, 256)
                used.add(nc)
                break
            except R.RelayBPError:
                if nc == 16:
                    raise
    return {"legs": a.tail_legs, "cluster_ctas": sorted(used),
            "note": "shots about to start this relay leg finish on thread-block clusters (bit-identical outputs)"}


def run_mixed(a):
    import torch
    from paper_2607_27644_b300 import relaybp as R
    from workloads.dem import circuit_dems

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dems, params = [], []
    for code, rounds, (gmin, gmax) in MIXED_CODES:
        for d in circuit_dems(code, MIXED_P, rounds, "Z"):
            dems.append(d)
            params.append(dict(DECODER, gamma_min=gmin, gamma_max=gmax))
    mmsg = a.msg or "f16"
    # one handle set and group per stream: steps rotate over the streams so the
    # rare shot that runs all relay legs overlaps the next steps
    NS = max(1, a.streams)
    HS = [[R.relaybp_build_dem(d, R.Params(msg_dtype=mmsg, **pp)) for d, pp in zip(dems, params)] for _ in range(NS)]
    hs = HS[0]
    tail = _tail_offload(R, [x for hh in HS for x in hh], a)
    grps = [R.relaybp_group_create(x) for x in HS]
    n = len(hs)
    shots = [MIXED_RATIO[i % 3] * a.mixed_base for i in range(n)]
    K, W = a.steps, max(1, a.warmup)
    streams = [torch.cuda.Stream(device=dev) for _ in range(NS)]

    def bufset():
        return dict(syn=[torch.empty((shots[i], hs[i].wc), dtype=torch.int32, device=dev) for i in range(n)],
                    obs=[torch.empty((shots[i], hs[i].wk), dtype=torch.int32, device=dev) for i in range(n)],
                    pobs=[torch.empty((shots[i], hs[i].wk), dtype=torch.int32, device=dev) for i in range(n)],
                    stats=[torch.empty((shots[i], 6), dtype=torch.int32, device=dev) for i in range(n)])
    bufs = [bufset() for _ in range(NS)]
    counters = torch.zeros((n, 4), dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.int32, device=dev)

    def step(k):
        q = k % NS
        b_, h_, st_ = bufs[q], HS[q], streams[q]
        flush.fill_(k)
        s0 = [(rank * (K + W) + k) * shots[i] for i in range(n)]
        for i in range(n):
            R.relaybp_sample(h_[i], SAMPLE_SEED + i, s0[i], shots[i], b_["syn"][i], b_["obs"][i], None, st_)
        R.relaybp_group_decode(grps[q], b_["syn"], s0, shots, None, b_["pobs"], b_["stats"], st_)
        for i in range(n):
            R.relaybp_count_failures(h_[i], b_["pobs"][i], b_["obs"][i], b_["stats"][i], shots[i], counters[i], st_)

    # eager runs size every scratch buffer before capture (one per stream)
    for q in range(NS):
        with torch.cuda.stream(streams[q]):
            step(q + NS * (K + W))                # k % NS == q: stream q's buffers and group
    torch.cuda.synchronize()
    graphs = {}
    for k in list(range(K)) + [K + w for w in range(W)]:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=streams[k % NS]):
            step(k)
        graphs[k] = g
    for w in range(W):
        with torch.cuda.stream(streams[(K + w) % NS]):
            graphs[K + w].replay()
    torch.cuda.synchronize()
    counters.zero_()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t0.record(streams[0])
        for s_ in streams[1:]:
            s_.wait_stream(streams[0])
        for k in range(K):
            with torch.cuda.stream(streams[k % NS]):
                graphs[k].replay()
        for s_ in streams[1:]:
            streams[0].wait_stream(s_)
        t1.record(streams[0])
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    # graph replays do not pass through the host counters: count what one step launches
    per_step = 2 * n + 1 + (n if tail else 0)       # samples, group launch, counts (+ one cluster launch per DEM)
    total = sum(shots) * K
    c = counters.cpu().numpy()
    from paper_2607_27644_b300.stats import per_qubit_round
    per_dem = []
    for i, d in enumerate(dems):
        f = int(c[i, 3])
        per_dem.append({"dem": d.name, "shots": int(c[i, 0]), "failures": f, "nonconverged": int(c[i, 1]),
                        "logical": int(c[i, 2]), "block_ler": f / max(1, c[i, 0])})
    line = {"metric": "decoded shots/s, nine ZSZ-LP DEMs in one persistent launch", "value": total / (ms / 1e3),
            "unit": "shots/s", "n_gpus": 1, "steps": K, "warmup": W, "ms_per_step": ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": mmsg,
            "data": "synthetic: Philox-sampled faults of the Table 5 circuit DEMs",
            "config": {"workload": "ZSZ-LP-320/390/550 (d=14/16/18) x p in {0.001,0.002,0.003}, Z-memory, "
                                   f"one group launch per step, CUDA-graph replay, steps rotating over {NS} streams",
                       "shots_per_step": sum(shots), "mix": shots, "decoder": "paper settings, Table 9 gamma",
                       "tail_offload": tail,
                       "l2": "flushed before every step (256 MiB write, inside the graph)"},
            "clocks": clk.summary(), "gpu_launches": per_step * K, "per_dem": per_dem}
    print(json.dumps(line), flush=True)
    for g_ in grps:
        R.relaybp_group_destroy(g_)
    for x in HS:
        for h in x:
            R.relaybp_destroy(h)


def train_learned(a, dev, d_inf, d_train, steps):
    """The library's trainer (row-tied weights, checkpoint selection by
    held-out decoding iterations) with this benchmark's settings."""
    from paper_2607_27644_b300.learned import train_rows
    warm = tuple(float(x) for x in a.warm_start.split(",") if x.strip()) or None
    return train_rows(d_inf, d_train, DECODER, steps, T=a.train_T, lr=a.train_lr, objective=a.objective,
                      device=dev, leg0=a.learned_legs == "leg0", warm_start=warm, select_shots=16384)


def run_learned(a):
    """Learned Relay-BP (trained on self-sampled shots at p = 0.2%) against
    plain Relay-BP (paper settings, FP32) on the same fresh shots at p = 0.1%.

    Learned decoder: learned row-tied message weights for the first T
    iterations of each learned leg (unit weights after them) -- leg 0 by
    default, or legs 0..49 with a learned memory-strength distribution
    (--learned-legs legs50); plain legs after that in the same launch (the fallback for shots the learned legs leave unconverged);
    stop after the first solution; FP32 messages (the two-shot kernel) and
    the --learned-msg storage.  Ablations run plain Relay-BP with the same
    stop-after-one rule at both precisions: what the learned parameters gain
    is learned vs ablation; learned vs plain also counts the stopping rule."""
    import numpy as np
    import torch
    from paper_2607_27644_b300 import relaybp as R
    from paper_2607_27644_b300.learned import LearnedParams
    from paper_2607_27644_b300.stats import agree_within
    from workloads.dem import circuit_dems

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    d_inf, d_train = circuit_dems(WORKLOAD["code"], [0.001, 0.002], WORKLOAD["rounds"], WORKLOAD["basis"])
    E = d_inf.n_edges
    wrow, knots, train_info = train_learned(a, dev, d_inf, d_train, a.train_steps)
    # ---- decoders: one handle set per stream ------------------------------------
    # learned parameters for the learned legs (leg 0 by default, legs 0..49
    # with --learned-legs legs50), then plain legs (unit weights, uniform
    # gamma) up to the paper's 1000 in the same launch: the plain fallback for
    # the shots the learned legs do not settle; stop after the first solution
    NS, LEGS = 3, train_info["learned_legs"]
    learned_params = dict(DECODER, stop_nconv=1)
    B, K, W = a.batch, a.steps, a.warmup
    streams = [torch.cuda.Stream(device=dev) for _ in range(NS)]
    H = []
    for q in range(NS):
        hh = {"plain": R.relaybp_build_dem(d_inf, R.Params(msg_dtype="f32", **DECODER))}
        for msg in ("f32", a.learned_msg):
            hl = R.relaybp_build_dem(d_inf, R.Params(msg_dtype=msg, **learned_params))
            R.relaybp_set_learned_rows(hl, wrow, knots)
            R.relaybp_set_learned_legs(hl, LEGS)
            hh["learned_" + msg] = hl
            hh["ablation_" + msg] = R.relaybp_build_dem(d_inf, R.Params(msg_dtype=msg, **learned_params))
        if a.tail_legs > 0:                     # every arm alike: shots reaching that leg finish on clusters
            for x in hh.values():
                R.relaybp_set_tail_offload(x, max(a.tail_legs, LEGS), a.tail_cluster, 256)
        H.append(hh)
    hp = H[0]["plain"]
    bufs = [dict(syn=torch.empty((B, hp.wc), dtype=torch.int32, device=dev),
                 obs=torch.empty((B, hp.wk), dtype=torch.int32, device=dev),
                 pobs=torch.empty((B, hp.wk), dtype=torch.int32, device=dev),
                 stats=torch.empty((B, 6), dtype=torch.int32, device=dev)) for _ in range(NS)]
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.int32, device=dev)

    def step(kind, k, cnt, it):
        q = k % NS
        st_, b_, h_ = streams[q], bufs[q], H[q]
        s0 = 5 * 10**8 + k * B
        with torch.cuda.stream(st_):
            flush.fill_(k)
            R.relaybp_sample(h_["plain"], SAMPLE_SEED, s0, B, b_["syn"], b_["obs"], None, st_)
            R.relaybp_decode_batch(h_[kind], b_["syn"], s0, B, None, b_["pobs"], b_["stats"], st_)
            R.relaybp_count_failures(h_["plain"], b_["pobs"], b_["obs"], b_["stats"], B, cnt, st_)
            it[q:q + 1].add_(b_["stats"][:, 3].sum())     # per stream: no cross-stream update

    out = {}
    kinds = ["plain"] + [f"{x}_{m}" for m in dict.fromkeys(("f32", a.learned_msg)) for x in ("learned", "ablation")]
    for kind in kinds:
        cnt = torch.zeros(4, dtype=torch.int64, device=dev)
        it = torch.zeros(NS, dtype=torch.int64, device=dev)
        for w_ in range(W):
            step(kind, K + w_, cnt, it)
        torch.cuda.synchronize()
        cnt.zero_()
        it.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            e0.record(streams[0])
            for s_ in streams[1:]:
                s_.wait_stream(streams[0])
            for k in range(K):
                step(kind, k, cnt, it)
            for s_ in streams[1:]:
                streams[0].wait_stream(s_)
            e1.record(streams[0])
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        c = cnt.cpu().tolist()
        out[kind] = {"shots_per_s": B * K / (ms / 1e3), "ms_per_step": ms / K, "shots": c[0], "failures": c[3],
                     "nonconverged": c[1], "logical": c[2], "block_ler": c[3] / max(1, c[0]),
                     "mean_iterations": float(it.sum().item()) / (B * K), "clocks": clk.summary()}
    lp, lm = out["plain"], a.learned_msg
    arms = {}
    for m in dict.fromkeys(("f32", lm)):
        ll, lab = out["learned_" + m], out["ablation_" + m]
        arms[m] = {"learned": ll, "ablation_plain_stop1": lab,
                   "speedup_vs_ablation": ll["shots_per_s"] / lab["shots_per_s"],
                   "mean_iterations_vs_ablation": ll["mean_iterations"] / lab["mean_iterations"],
                   "speedup_vs_plain": ll["shots_per_s"] / lp["shots_per_s"],
                   "equal_ler_2sigma_vs_plain": bool(agree_within(ll["failures"], ll["shots"], lp["failures"],
                                                                  lp["shots"])),
                   "equal_ler_2sigma_vs_ablation": bool(agree_within(ll["failures"], ll["shots"], lab["failures"],
                                                                     lab["shots"]))}
    best = max(arms.values(), key=lambda x: x["learned"]["shots_per_s"])
    line = {"metric": METRIC, "value": best["learned"]["shots_per_s"], "unit": "shots/s", "n_gpus": 1, "steps": K,
            "warmup": W, "ms_per_step": best["learned"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: Philox-sampled faults of the ZSZ-LP-160 circuit DEMs",
            "config": {"workload": "learned vs plain Relay-BP, ZSZ-LP-160 d=10, inference p=0.001, training p=0.002",
                       "train": train_info,
                       "learned_decoder": ("learned row-tied weights in leg 0" if LEGS == 1 else
                                           f"learned weights + knots in legs 0-{LEGS - 1}")
                                          + ", plain legs after (in-kernel fallback), stop_nconv=1; FP32 and " + lm
                                          + " message storage",
                       "ablation": "plain Relay-BP with the same stop_nconv=1 rule at the same storage precision",
                       "pipeline": "3 streams, steps rotate, L2 flushed before every step",
                       "tail_offload": ({"legs": max(a.tail_legs, LEGS), "cluster_ctas": a.tail_cluster,
                                         "arms": "all"} if a.tail_legs > 0 else None),
                       "plain_decoder": "FP32, paper settings (stop_nconv=5)", "shots_per_step": B},
            "plain": lp, "arms": arms,
            "note": "speedup_vs_plain mostly measures the stopping rule (stop after the first solution vs five); "
                    "speedup_vs_ablation is what the learned parameters gain at the same rule",
            "clocks": best["learned"]["clocks"]}
    print(json.dumps(line), flush=True)
    for hh in H:
        for x in hh.values():
            R.relaybp_destroy(x)


def run_stream550(a):
    """ZSZ-LP-550 (DEM 4180 x 63,910, d = 18, p = 0.1%, Z-memory) decoded in
    graph-captured batches over rotating streams with int8 storage: shots/s,
    LER per qubit-round with 95% Clopper-Pearson bounds, and per-shot latency
    percentiles from device timestamps at shot start and retire."""
    import numpy as np
    import torch
    from paper_2607_27644_b300 import relaybp as R
    from paper_2607_27644_b300.stats import clopper_pearson, per_qubit_round
    from workloads.dem import circuit_dems

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    code, rounds, (gmin, gmax) = MIXED_CODES[2]
    t_build = time.perf_counter()
    dem = circuit_dems(code, [0.001], rounds, "Z")[0]
    t_build = time.perf_counter() - t_build
    msg = a.msg or "i8"
    NS, B, K, W = max(1, a.streams), a.stream_batch, a.steps, max(1, a.warmup)
    hs = [R.relaybp_build_dem(dem, R.Params(msg_dtype=msg, **dict(DECODER, gamma_min=gmin, gamma_max=gmax)))
          for _ in range(NS)]
    h = hs[0]
    tail = _tail_offload(R, hs, a)
    streams = [torch.cuda.Stream(device=dev) for _ in range(NS)]
    bufs = [dict(syn=torch.empty((B, h.wc), dtype=torch.int32, device=dev),
                 obs=torch.empty((B, h.wk), dtype=torch.int32, device=dev),
                 pobs=torch.empty((B, h.wk), dtype=torch.int32, device=dev),
                 stats=torch.empty((B, 6), dtype=torch.int32, device=dev)) for _ in range(NS)]
    times = [torch.zeros((B, 2), dtype=torch.int64, device=dev) for _ in range(K + W)]
    counters = torch.zeros(4, dtype=torch.int64, device=dev)
    iters = torch.zeros(NS, dtype=torch.int64, device=dev)     # per stream: no cross-stream update
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.int32, device=dev)

    def step(k):
        q = k % NS
        b_, h_ = bufs[q], hs[q]
        s0 = (rank * (K + W) + k) * B
        flush.fill_(k)
        R.relaybp_sample(h_, SAMPLE_SEED, s0, B, b_["syn"], b_["obs"], None, streams[q])
        R.relaybp_decode_timed(h_, b_["syn"], s0, B, times[k], None, b_["pobs"], b_["stats"], streams[q])
        R.relaybp_count_failures(h_, b_["pobs"], b_["obs"], b_["stats"], B, counters, streams[q])
        iters[q:q + 1].add_(b_["stats"][:, 3].sum())

    # one eager step per stream sizes every scratch buffer, then each step is
    # captured once on its stream and replayed
    for q in range(NS):
        with torch.cuda.stream(streams[q]):
            R.relaybp_sample(hs[q], SAMPLE_SEED, 0, B, bufs[q]["syn"], bufs[q]["obs"], None, streams[q])
            R.relaybp_decode_timed(hs[q], bufs[q]["syn"], 0, B, times[K], None, bufs[q]["pobs"], bufs[q]["stats"],
                                   streams[q])
    torch.cuda.synchronize()
    graphs = {}
    for k in list(range(K)) + [K + w for w in range(W)]:
        q = k % NS
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=streams[q]):
            step(k)
        graphs[k] = g
    for w in range(W):
        with torch.cuda.stream(streams[(K + w) % NS]):
            graphs[K + w].replay()
    torch.cuda.synchronize()
    counters.zero_()
    iters.zero_()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t0.record(streams[0])
        for s_ in streams[1:]:
            s_.wait_stream(streams[0])
        for k in range(K):
            with torch.cuda.stream(streams[k % NS]):
                graphs[k].replay()
        for s_ in streams[1:]:
            streams[0].wait_stream(s_)
        t1.record(streams[0])
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    c = counters.cpu().tolist()
    tt = torch.cat([times[k] for k in range(K)]).cpu().numpy().astype(np.int64)
    service = (tt[:, 1] - tt[:, 0]) / 1e6
    sojourn = np.concatenate([(times[k][:, 1] - times[k][:, 0].min()).cpu().numpy() / 1e6 for k in range(K)])
    pct = lambda x, q: float(np.percentile(x, q))
    shots, fails = int(c[0]), int(c[3])
    blk = fails / max(1, shots)
    lo, hi = clopper_pearson(fails, shots)
    kq = dem.n_obs
    line = {"metric": "decoded shots/s, ZSZ-LP-550 circuit level, graph-captured batches", "value": B * K / (ms / 1e3),
            "unit": "shots/s", "n_gpus": 1, "steps": K, "warmup": W, "ms_per_step": ms / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": msg,
            "data": "synthetic: Philox-sampled faults of the ZSZ-LP-550 circuit DEM (no dataset)",
            "config": {"workload": f"ZSZ-LP-550 circuit-level Z-memory, d={rounds}, p=0.001, DEM {dem.n_det}x"
                                   f"{dem.n_loc} (E={dem.n_edges}), plain Relay-BP, Table 9 gamma [{gmin}, {gmax}]",
                       "shots_per_batch": B, "batches": K, "streams": NS,
                       "state": "per-block region of global memory (L2-resident): one shot's state exceeds shared "
                                "memory even in int8",
                       "l2": "flushed before every batch (256 MiB write, inside the graph)",
                       "dem_build_s": t_build, "tail_offload": tail},
            "clocks": clk.summary(), "gpu_launches": (4 if tail else 3) * K,
            "ler": {"shots": shots, "failures": fails, "nonconverged": int(c[1]), "logical": int(c[2]),
                    "block_ler": blk, "block_ler_95": [lo, hi],
                    "per_qubit_round": per_qubit_round(blk, rounds, kq),
                    "per_qubit_round_95": [per_qubit_round(lo, rounds, kq), per_qubit_round(hi, rounds, kq)]},
            "latency_ms": {"service_p50": pct(service, 50), "service_p99": pct(service, 99),
                           "service_p99.9": pct(service, 99.9),
                           "service_max": float(service.max()), "service_mean": float(service.mean()),
                           "in_batch_p50": pct(sojourn, 50), "in_batch_p99": pct(sojourn, 99),
                           "definition": "service = retire - start of the shot's thread block (device %globaltimer); "
                                         "in_batch = retire - first start in its batch"},
            "mean_iterations_per_shot": float(iters.sum().item()) / (B * K)}
    print(json.dumps(line), flush=True)
    for x in hs:
        R.relaybp_destroy(x)


# Table 5 (L40S): mean / p99 / p99.9 / max single-shot latency in ms, and
# Table 12 (ZSZ-LP-390 on a B200): mean / p99 / p99.9.
PAPER_LATENCY = {"ZSZ-LP-320": (1.2, 2.0, 3.2, 201.0), "ZSZ-LP-390": (1.5, 2.6, 3.9, 260.0),
                 "ZSZ-LP-550": (2.2, 3.3, 4.6, 393.0)}
PAPER_LATENCY_B200_390 = (2.068, 3.554, 5.248)


def run_latency(a):
    """Single-shot decoding latency (Sec. 6.1, Table 5; App. F, Table 12):
    the ZSZ-LP-320/390/550 circuit-level X- and Z-memory DEMs at p = 0.1%
    (d = 14/16/18) with the paper's decoder settings and Table 9 gamma in
    FP32, one shot per call, each decoded by one thread-block cluster of
    --cluster CTAs.  Per-shot time between CUDA events around the call (the
    launch included): mean, p50, p99, p99.9, averaged over X and Z like the
    paper; max latency with every relay leg run (the paper's stopping rule
    'All'); e2e: the same shots through relaybp_decode_host (host syndrome
    in, host prediction out, synchronised per shot)."""
    import numpy as np
    import torch
    from paper_2607_27644_b300 import relaybp as R
    from workloads.dem import circuit_dem

    rank, world, local = _dist()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N, W, NM = a.latency_shots, max(3, a.warmup), a.latency_max_shots
    per, launches, e2e_ms, h2d, d2h = {}, 0, [], 0, 0
    pct = lambda x, q: float(np.percentile(x, q))
    with ClockSampler(local) as clk:
        for code, rounds, (gmin, gmax) in MIXED_CODES:
            res = {}
            for basis in ("Z", "X"):
                t_build = time.perf_counter()
                dem = circuit_dem(code, 0.001, rounds, basis)
                t_build = time.perf_counter() - t_build
                prm = dict(DECODER, gamma_min=gmin, gamma_max=gmax)
                h = R.relaybp_build_dem(dem, R.Params(msg_dtype="f32", **prm))
                R.relaybp_set_cluster_kernel(h, a.cluster)
                syn = torch.zeros((N + W, h.wc), dtype=torch.int32, device=dev)
                R.relaybp_sample(h, SAMPLE_SEED, 0, N + W, syn)
                corr = torch.zeros((1, h.wv), dtype=torch.int32, device=dev)
                pobs = torch.zeros((1, h.wk), dtype=torch.int32, device=dev)
                stats = torch.zeros((N + W, 6), dtype=torch.int32, device=dev)
                for i in range(W):
                    R.relaybp_decode_batch(h, syn[i:i + 1], i, 1, corr, pobs, stats[i:i + 1])
                torch.cuda.synchronize()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(N)]
                for i in range(N):
                    s_ = W + i
                    ev[i][0].record()
                    R.relaybp_decode_batch(h, syn[s_:s_ + 1], s_, 1, corr, pobs, stats[s_:s_ + 1])
                    ev[i][1].record()
                torch.cuda.synchronize()
                launches += N
                ms = np.array([x.elapsed_time(y) for x, y in ev])
                st = stats[W:].cpu().numpy()
                # end to end through the host-buffer entry point (a sample of the same shots)
                ne = min(N, 200)
                h_syn = syn[W:W + ne].cpu().pin_memory()
                h_pobs = torch.zeros((1, h.wk), dtype=torch.int32).pin_memory()
                h_st = torch.zeros((1, 6), dtype=torch.int32).pin_memory()
                te = []
                for i in range(ne):
                    t0 = time.perf_counter()
                    R.relaybp_decode_host(h, h_syn[i:i + 1], W + i, 1, h_pobs, h_st)
                    te.append((time.perf_counter() - t0) * 1e3)
                launches += ne
                e2e_ms += te
                h2d, d2h = h.wc * 4, h.wk * 4 + 24
                # worst case: every relay leg run
                mx = []
                if NM > 0:
                    R.relaybp_set_params(h, R.Params(msg_dtype="f32", stop_all=True, **prm))
                    for i in range(NM):
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record()
                        R.relaybp_decode_batch(h, syn[W + i:W + i + 1], W + i, 1, corr, pobs, stats[W + i:W + i + 1])
                        e1.record()
                        torch.cuda.synchronize()
                        mx.append(e0.elapsed_time(e1))
                    launches += NM
                res[basis] = {"dem": [dem.n_det, dem.n_loc], "edges": int(h.n_edges), "dem_build_s": t_build,
                              "mean": float(ms.mean()), "p50": pct(ms, 50), "p99": pct(ms, 99),
                              "p99.9": pct(ms, 99.9), "max_seen": float(ms.max()),
                              "max_all_legs": float(np.mean(mx)) if mx else None,
                              "e2e_mean": float(np.mean(te)), "mean_iterations": float(st[:, 3].mean()),
                              "mean_legs": float(st[:, 2].mean()), "converged": float(st[:, 0].mean())}
                R.relaybp_destroy(h)
            xz = {k: (res["X"][k] + res["Z"][k]) / 2 for k in ("mean", "p99", "p99.9", "e2e_mean")}
            xz["max_all_legs"] = ((res["X"]["max_all_legs"] + res["Z"]["max_all_legs"]) / 2
                                  if res["X"]["max_all_legs"] is not None else None)
            pm = PAPER_LATENCY[code]
            per[code] = {"d": rounds, "X": res["X"], "Z": res["Z"], "xz": xz,
                         "paper_l40s": {"mean": pm[0], "p99": pm[1], "p99.9": pm[2], "max": pm[3]},
                         "mean_vs_paper": xz["mean"] / pm[0]}
    v = per["ZSZ-LP-390"]["xz"]["mean"]
    line = {"metric": "single-shot decoding latency, ZSZ-LP-390 circuit level p=0.1%, XZ-averaged mean",
            "value": v, "unit": "ms", "n_gpus": 1, "steps": N, "warmup": W, "ms_per_step": v,
            "higher_is_better": False, "scaling": "none (one shot at a time)",
            "vs_baseline": v / PAPER_LATENCY["ZSZ-LP-390"][0], "dtype": "f32",
            "data": "synthetic: Philox-sampled faults of the circuit DEMs (no dataset)",
            "config": {"workload": "Table 5: ZSZ-LP-320/390/550 circuit-level X- and Z-memory, d = 14/16/18, "
                                   "p = 0.001, paper decoder settings, Table 9 gamma, one shot per call",
                       "kernel": f"relay_cluster_kernel, {a.cluster} CTAs (one per SM) per shot, state in "
                                 "distributed shared memory",
                       "timing": "CUDA events around each single-shot call (launch included); L2 not flushed "
                                 "(a real-time decoder keeps its DEM resident)"},
            "per_code": per,
            "paper_b200_390": dict(zip(("mean", "p99", "p99.9"), PAPER_LATENCY_B200_390)),
            "e2e": {"value": float(np.mean(e2e_ms)), "unit": "ms", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "definition": "relaybp_decode_host per shot: pinned host syndrome in, prediction and "
                                  "statistics out, synchronised (mean over all codes and bases)"},
            "clocks": clk.summary(), "gpu_launches": launches}
    print(json.dumps(line), flush=True)


def run_gamma_sweep(a):
    """ZSZ-LP-160: the gamma-interval grid search of Table 9 at p_sweep = 0.2%
    (X- and Z-memory, fewest pooled failures), then the XZ-averaged LER per
    qubit-round at p = 0.1/0.2/0.3% with the chosen interval and with Table
    9's, 95% Clopper-Pearson bounds."""
    import torch
    from paper_2607_27644_b300 import relaybp as R
    from paper_2607_27644_b300.sweep import GpuDecoder, gamma_grid_search, ler_curve
    from workloads.dem import circuit_dems
    from workloads.zsz import load_code

    _, _, local = _dist()
    torch.cuda.set_device(local)
    code, rounds = WORKLOAD["code"], WORKLOAD["rounds"]
    k = load_code(code).k
    ps = [0.001, 0.002, 0.003]
    zs, xs = circuit_dems(code, ps, rounds, "Z"), circuit_dems(code, ps, rounds, "X")
    dems = {p: {"Z": z, "X": x} for p, z, x in zip(ps, zs, xs)}
    dec = GpuDecoder(batch=1 << 16, sample_seed=SAMPLE_SEED)
    base = R.Params(msg_dtype=a.msg or "f32", **DECODER)
    t0 = time.perf_counter()
    best, grid = gamma_grid_search(dec, dems[0.002], base, [-0.24, -0.15, -0.05], [0.5, 0.61, 0.7],
                                   a.sweep_shots, 0.002, rounds, k)
    t_grid = time.perf_counter() - t0
    chosen = R.Params(**dict(vars(base), gamma_min=best.gamma[0], gamma_max=best.gamma[1]))
    curve = ler_curve(dec, dems, chosen, a.sweep_shots, rounds, k, shot0=10**9)
    table9 = ler_curve(dec, dems, base, a.sweep_shots, rounds, k, shot0=10**9)
    dt = time.perf_counter() - t0
    shots = 2 * a.sweep_shots * (len(grid) + 2 * len(ps))
    line = {"metric": "gamma-interval grid search and XZ-averaged LER per qubit-round, ZSZ-LP-160",
            "value": shots / dt, "unit": "shots/s", "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": base.msg_dtype,
            "data": "synthetic: Philox-sampled faults of the ZSZ-LP-160 circuit DEMs (X and Z memory)",
            "config": {"workload": f"{code}, d={rounds}, grid at p_sweep=0.002, curve at p in {ps}",
                       "shots_per_point_and_basis": a.sweep_shots, "grid_seconds": t_grid},
            "chosen_gamma": list(best.gamma), "table9_gamma": [DECODER["gamma_min"], DECODER["gamma_max"]],
            "grid": [q.as_dict() for q in grid], "curve_chosen": [q.as_dict() for q in curve],
            "curve_table9": [q.as_dict() for q in table9]}
    print(json.dumps(line), flush=True)


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "mixed":
        run_mixed(a)
    elif a.workload == "learned":
        run_learned(a)
    elif a.workload == "stream550":
        run_stream550(a)
    elif a.workload == "gamma_sweep":
        run_gamma_sweep(a)
    elif a.workload == "latency":
        run_latency(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
