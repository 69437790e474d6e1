#!/usr/bin/env python3
"""Benchmark of the hot path: one full-tree CFR+ iteration per step on the holdem169_depth12 workload.

Workload: seeded synthetic two-player zero-sum tree, ~1.0e8 nodes (1326-way root deal of 2-card
combos bucketed to 169 classes, depth 12, 4-5 actions, u1 ~ U[-100, 100]); CFR+ with linear
averaging, FP32 reach/values/regrets with FP64 cumulative regrets and strategy sums.  The resident
state (~1.7 GB) is larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the plain recursive FP64 CPU oracle on
the host cores over a bounded sample of the same workload (its first deals).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tree-node updates/sec and CFR iterations/sec (HBM roofline %); time to exploitability 1e-3"
UNIT = "node-updates/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--only", choices=["network-gemm"], default=None,
                    help="run one measurement alone (profiling): the value network's matrix products")
    ap.add_argument("--workload", default="holdem169_depth12")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--nodes", type=int, default=None,
                    help="same workload family rescaled to about this many nodes (profiling captures)")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--variant", choices=["plus", "vanilla"], default="plus")
    ap.add_argument("--fuse-levels", type=int, default=-1,
                    help="FP32 mode: deepest depths run by the fused kernel (-1 automatic, 0 none)")
    ap.add_argument("--tail-slots", type=int, default=0,
                    help="FP32 mode, last two depths: 0 per-slot loads and atomics (default), 1 slot-dense tiles "
                         "with staged strategy entries, 2 the same with bulk-reduced regrets")
    ap.add_argument("--head-levels", type=int, default=-1,
                    help="FP32 mode: depths below the root run by the two head launches (-1 as many as qualify, 0 none)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-error", action="store_true", help="skip the error-against-the-oracle block")
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-exploitability-1e-3 measurement")
    ap.add_argument("--no-leaf", action="store_true", help="skip the learned-leaf depth-limited measurement")
    ap.add_argument("--leaf-samples-per-node", type=int, default=256)
    ap.add_argument("--leaf-train-steps", type=int, default=10000)
    ap.add_argument("--batched-games", type=int, default=4096,
                    help="subgames of the batched measurement (0: skip it)")
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), util=float(parts[4]),
                                 reasons=[n for n, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                                             "sw_power_cap"), parts[6:10]) if v == "Active"]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        loaded = [r for r in rows if r["util"] > 0] or rows
        sm = sorted(r["sm"] for r in loaded)
        reasons = sorted({x for r in loaded for x in r["reasons"]})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r["smax"] for r in rows), "reasons": reasons,
                "samples": len(loaded)}


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        v = json.load(open(p)).get("hbm_gbs")
        if v:
            return float(v), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback (6.8 TB/s, earlier GB300 copy measurement)"


def kernel_source_hash() -> str:
    """Hash of the sources that define the single-game iteration's kernels, their launch and the layout
    they read (the batch and value-network sources do not change its traffic)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2408_14778_gb300", "csrc")
    for f in ("kernels.cuh", "stream.cuh", "cfr_api.cu", "layout.cpp", "layout.hpp"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, precision: str, phase: str):
    """ncu DRAM bytes per launch of the given phase's kernel, from the committed summary, if it was taken on the
    current kernel sources."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p):
        return None
    want = kernel_source_hash()
    for line in open(p):
        if line.startswith("#"):
            continue
        kv = dict(x.split("=", 1) for x in line.split() if "=" in x)
        if (kv.get("kernels_sha") == want and kv.get("workload") == workload and kv.get("precision") == precision
                and kv.get("phase") == phase.replace(" ", "_")):
            return float(kv["dram_bytes_per_launch"])
    return None


def oracle_sample(g, budget_s: float, threads: int = 1):
    """First-deals sub-game sized so one oracle iteration on `threads` host threads takes about
    budget_s seconds."""
    import gamegen

    per_deal = int(g.meta["public_nodes"])
    rate = 1.0e7 * max(threads, 1)             # oracle node-updates/s, order of magnitude, sizing only
    k = max(1, min(int(g.meta["deals"]), int(budget_s * rate / per_deal)))
    return gamegen.first_deals(g, k)


def oracle_threads() -> int:
    """Host threads of the oracle's multi-threaded passes (all of this host's cores by default)."""
    import oracle

    return oracle.max_threads()


TTT_TARGET = 1e-3          # exploitability (NashConv / 2), absolute, payoff units
TTT_CHECK = 25             # iterations between exploitability evaluations
TTT_MAX_ITERS = 100000
TTT_ORACLE_SECONDS = 60.0
LEAF_BLUEPRINT_ITERS = 4000
LEAF_REFRESH = 10            # depth-limited solving: iterations between leaf refreshes
LEAF_MAX_ITERS = 20000


def _ttt_run(step, expl, max_iters: int, max_seconds: float) -> dict:
    """Iterates in chunks of TTT_CHECK until the exploitability of the average strategy is at most
    TTT_TARGET; the time includes the evaluations."""
    t0, it, ex = time.perf_counter(), 0, float("inf")
    while it < max_iters and time.perf_counter() - t0 < max_seconds:
        step(TTT_CHECK)
        it += TTT_CHECK
        ex = expl()
        if ex <= TTT_TARGET:
            break
    return {"reached": ex <= TTT_TARGET, "seconds": time.perf_counter() - t0, "iterations": it, "exploitability": ex}


def time_to_exploitability(args, local: int) -> dict:
    """CFR+ (linear averaging, simultaneous updates) on the 13-rank fold/showdown game (payoffs up to 8):
    time until the average strategy's exploitability reaches 1e-3, on the GPU (FP32 mode) for the full
    2e6-node game and a 2e5-node cut, and for the oracle (one core) on the same cut."""
    import gamegen
    import oracle
    import paper_2408_14778_gb300 as cfr

    out = {"target": TTT_TARGET, "check_every": TTT_CHECK, "variant": "cfr+ linear averaging, simultaneous",
           "time_includes": "iterations and the exploitability evaluations"}
    # the variants of the same solver on the full game (GPU, FP32 mode)
    g = gamegen.config("rank13_depth10", seed=args.seed)
    for name, variant, mode in (("cfr+_alternating", cfr.CFR_PLUS, cfr.CFR_ALTERNATING),
                                ("linear_cfr", cfr.CFR_LINEAR, cfr.CFR_SIMULTANEOUS),
                                ("discounted_cfr_1.5_0_2", cfr.CFR_DISCOUNTED, cfr.CFR_SIMULTANEOUS),
                                ("discounted_cfr_1.5_0_2_alternating", cfr.CFR_DISCOUNTED, cfr.CFR_ALTERNATING)):
        s = cfr.cfr_load_tree(g, variant=variant, precision=cfr.CFR_FP32, update_mode=mode, device=local,
                              dcfr=(1.5, 0.0, 2.0))
        cfr.cfr_synchronize(s)
        r = _ttt_run(lambda n: cfr.cfr_iterate(s, n), lambda: cfr.cfr_exploitability(s)[1], TTT_MAX_ITERS, 30.0)
        r["nodes"] = g.num_nodes
        out[f"gpu_rank13_depth10_{name}"] = r
        s.close()
    for name, nodes in (("rank13_depth10", None), ("rank13_depth10_2e5", 200_000)):
        g = gamegen.config("rank13_depth10", seed=args.seed, target_nodes=nodes)
        s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32, device=local)
        cfr.cfr_synchronize(s)
        r = _ttt_run(lambda n: cfr.cfr_iterate(s, n), lambda: cfr.cfr_exploitability(s)[1], TTT_MAX_ITERS, 30.0)
        r["nodes"] = g.num_nodes
        # the final exploitability against the oracle's best responses to the same average strategy
        r["oracle_error_abs"] = abs(2 * r["exploitability"] - oracle.Oracle(g).exploitability(
            profile=cfr.cfr_average_strategy(s))[0]) / 2
        out[f"gpu_{name}"] = r
        s.close()
        if nodes is not None:
            o = oracle.Oracle(g)
            r = _ttt_run(lambda n: o.iterate(n, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR),
                         lambda: o.exploitability()[1], TTT_MAX_ITERS, TTT_ORACLE_SECONDS)
            r.update(nodes=g.num_nodes, cores=1, capped_at_seconds=TTT_ORACLE_SECONDS)
            out[f"oracle_{name}"] = r
    return out


def measured_bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        v = json.load(open(p)).get("bf16_tflops")
        if v:
            return float(v), "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    except (OSError, ValueError):
        pass
    return 1900.0, "fallback (1.9 PFLOP/s bf16 burst, earlier GB300 measurement)"


def network_gemm_measurement(net, local: int, batch: int = 4096, reps: int = 5) -> dict:
    """The value network's matrix products (402 -> 3 x 1024 ReLU -> 338) at a batch of 4096: forward and
    backward time of the last of reps passes (CUDA events around the products) against the bf16 peak."""
    import torch

    import paper_2408_14778_gb300 as cfr

    xb = torch.randn(batch, 402, device=f"cuda:{local}")
    tb = torch.randn(batch, 338, device=f"cuda:{local}")
    for _ in range(reps):
        cfr.cfr_mlp_forward(net, xb)
        cfr.cfr_mlp_backward(net, xb, tb)
    st = cfr.cfr_mlp_gemm_stats(net)
    peak, src = measured_bf16_peak()
    fwd, bwd = st["fwd_flops"] / st["fwd_us"] / 1e6, st["bwd_flops"] / st["bwd_us"] / 1e6
    return {"batch": batch, "forward_tflops": fwd, "backward_tflops": bwd, "forward_us": st["fwd_us"],
            "backward_us": st["bwd_us"], "peak_tflops": peak, "peak_source": src, "forward_frac": fwd / peak,
            "backward_frac": bwd / peak,
            "instruction": "every product: tcgen05.mma kind::f16 (bf16, fp32 accumulator in tensor memory, TMA "
                           "operands); weight gradients from transposed copies of the layer inputs and output "
                           "gradients, split over the batch with fp32 vector atomics"}


def run_network_gemm_only(args, local: int):
    """--only network-gemm: the value network's products alone (for profiling), one JSON line."""
    import paper_2408_14778_gb300 as cfr
    from paper_2408_14778_gb300 import depth_limited as dl

    cfr.build()
    net = dl.make_network(seed=args.seed, device=local)
    print(json.dumps({"network_gemm": network_gemm_measurement(net, local, reps=max(1, args.steps))}), flush=True)


def learned_leaf_measurement(args, local: int, ttt: dict | None) -> dict:
    """Depth-limited CFR+ with the learned leaf network on the 13-rank fold/showdown game (2e6 nodes) cut
    at game depth 6: training samples from full-depth GPU CFR+ solves of the cut subgames under random
    ranges, the network (402 -> 3 x 1024 ReLU -> 338, BF16 tensor-core kernels) trained by the library,
    then the depth-limited solve with the leaves refreshed on the device every iteration.  Its
    exploitability is measured in the depth-limited game and, in the full game, with the strategy of a
    full-depth CFR+ solve below the cut; an untrained network of the same shape is the baseline."""
    import numpy as np
    import torch

    import gamegen
    import paper_2408_14778_gb300 as cfr
    from paper_2408_14778_gb300 import depth_limited as dl

    out = {"game": "rank13_depth10 (13-rank fold/showdown, 156 deals, depth 10)", "cut_game_depth": 6,
           "variant": "cfr+ linear averaging, simultaneous", "target": TTT_TARGET, "check_every": TTT_CHECK}
    g = gamegen.config("rank13_depth10", seed=args.seed)
    t0 = time.perf_counter()
    cut = dl.cut_game(g, depth=5, seed=args.seed)
    out["cut"] = {"full_nodes": g.num_nodes, "depth_limited_nodes": int(cut.game.parent.shape[0]),
                  "cut_public_nodes": int(cut.cut_nodes.size), "leaves": int(cut.leaf_nodes.size),
                  "host_seconds": time.perf_counter() - t0}
    # full-depth CFR+: the strategy below the cut (and the full-depth reference for the comparison)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32, device=local)
    cfr.cfr_synchronize(s)
    t0 = time.perf_counter()
    cfr.cfr_iterate(s, LEAF_BLUEPRINT_ITERS)
    ex_full = cfr.cfr_exploitability(s)[1]
    out["full_depth"] = {"iterations": LEAF_BLUEPRINT_ITERS, "seconds": time.perf_counter() - t0,
                         "exploitability": ex_full,
                         "time_to_1e-3": (ttt or {}).get("gpu_rank13_depth10")}
    below = cfr.cfr_average_strategy(s)
    blueprint_S = cfr.cfr_get_state(s)["strat_sum"]
    s.close()
    # the pipeline with perfect leaves: the full solve's own values at the cut, fixed
    t0 = time.perf_counter()
    y_exact = dl.blueprint_leaf_values(cut, blueprint_S, device=local)
    top = dl.solve_with_fixed_leaves(cut, y_exact, LEAF_BLUEPRINT_ITERS, device=local)
    out["depth_limited_exact_leaves"] = {
        "iterations": LEAF_BLUEPRINT_ITERS, "seconds": time.perf_counter() - t0,
        "full_game_exploitability": dl.full_game_exploitability(g, dl.combined_strategy(cut, top, below), device=local),
        "note": "leaves fixed to the full-depth solve's deal values at the cut: what a perfect network gives"}
    t0 = time.perf_counter()
    X, Y = dl.generate_samples(cut, per_node=args.leaf_samples_per_node, iterations=300, seed=args.seed,
                               device=local)
    out["samples"] = {"count": int(X.shape[0]), "per_cut_node": args.leaf_samples_per_node,
                      "solver_iterations": 300, "seconds": time.perf_counter() - t0,
                      "source": "full-depth GPU CFR+ on the cut subgames under random (Dirichlet) ranges"}
    net = dl.make_network(seed=args.seed, device=local)
    # a random tenth of the samples is held out of training
    perm = np.random.default_rng(args.seed).permutation(X.shape[0])
    nh = max(1, X.shape[0] // 10)
    Xh, Yh = X[perm[:nh]], Y[perm[:nh]]
    Xt, Yt = X[perm[nh:]], Y[perm[nh:]]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = dl.train(net, Xt, Yt, steps=args.leaf_train_steps, batch=1024, lr=1e-3, seed=args.seed, device=local)
    torch.cuda.synchronize()
    held = float(cfr.cfr_mlp_backward(net, torch.tensor(Xh, device=f"cuda:{local}"),
                                      torch.tensor(Yh, device=f"cuda:{local}")).item())
    out["training"] = {"steps": args.leaf_train_steps, "batch": 1024, "optimizer": "adam, lr 1e-3 decaying to 1e-4",
                       "samples_trained": int(Xt.shape[0]), "samples_held_out": int(nh),
                       "seconds": time.perf_counter() - t0, "mse_first": hist[0], "mse_last": hist[-1],
                       "mse_held_out": held, "note": "mean squared error of values divided by the payoff bound"}
    out["network_gemm"] = network_gemm_measurement(net, local)
    untrained = dl.make_network(seed=args.seed + 1, device=local)
    for name, model, ranges in (("trained", net, cfr.CFR_AVERAGE_STRATEGY),
                                ("trained_current_ranges", net, cfr.CFR_CURRENT_STRATEGY),
                                ("untrained", untrained, cfr.CFR_AVERAGE_STRATEGY)):
        d = dl.DepthLimitedSolver(cut, model, refresh=LEAF_REFRESH, device=local, ranges=ranges)
        cfr.cfr_synchronize(d.s)
        r = _ttt_run(d.iterate, d.exploitability, LEAF_MAX_ITERS, 20.0)
        r["leaf_refresh_every"] = LEAF_REFRESH
        r["full_game_exploitability"] = dl.full_game_exploitability(
            g, dl.combined_strategy(cut, d.average_strategy(), below), device=local)
        r["leaf_ranges"] = "average strategy" if ranges == cfr.CFR_AVERAGE_STRATEGY else "current strategy"
        r["note"] = ("exploitability: in the depth-limited game with the leaves' current values; "
                     "full_game_exploitability: in the full game, full-depth strategy below the cut")
        out[f"depth_limited_{name}"] = r
        d.close()
    return out


def batched_measurement(args, local: int) -> dict:
    import paper_2408_14778_gb300 as cfr

    wide_range = _subgames(args, dict(min_nodes=1e2, max_nodes=1e5))
    label = "log-uniform 1e2-1e5 nodes, depth 4-10, 2-5 actions"
    out = _batched_run(args, local, wide_range, label)
    out["alternating"] = _batched_run(args, local, wide_range, label, update_mode=cfr.CFR_ALTERNATING)
    small = _subgames(args, dict(min_nodes=1e2, max_nodes=1e3))
    out["small_games"] = _batched_run(args, local, small, "log-uniform 1e2-1e3 nodes, depth 4-10, 2-5 actions",
                                      ttt=False)
    return out


def _subgames(args, kw: dict):
    import gamegen

    t0 = time.perf_counter()
    games = gamegen.batch_subgames(args.batched_games, seed=args.seed, **kw)
    return games, time.perf_counter() - t0


def _batched_run(args, local: int, games_gen, label: str, ttt: bool = True, update_mode: int = 0) -> dict:
    """Batched CFR+: independent subgames (log-uniform 1e2-1e5 nodes, depth 4-10, 2-5 actions) advanced
    together by one persistent launch per call, launch shape from the autotuner.  Reports subgames/s and
    node updates/s for 500 iterations, the p50/p99 per-subgame iteration time, the exploitability reached,
    the time until every subgame's exploitability is at most 1e-3 (capped), and the same games run as ONE
    tree (a uniform chance root over them) by the plain full-tree solver on the same GPU; update_mode:
    simultaneous (0) or alternating (1) updates, for both."""
    import numpy as np
    import torch

    import gamegen
    import paper_2408_14778_gb300 as cfr

    games, gen_s = games_gen
    nodes = np.array([g.num_nodes for g in games], dtype=np.int64)
    cache = os.path.join(os.path.expanduser("~"), ".cache", "paper_2408_14778_gb300", "batch_tuning.json")
    t0 = time.perf_counter()
    tune = cfr.cfr_batch_tune(games, variant=cfr.CFR_PLUS, device=local, cache_path=cache, update_mode=update_mode)
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    fuse = tune.get("fuse_levels", -1)
    b = cfr.cfr_batch_load(games, variant=cfr.CFR_PLUS, device=local, split_nodes=tune["split_nodes"],
                           update_mode=update_mode, fuse_levels=fuse)
    cfr.cfr_batch_set_tuning(b, tune["threads_per_block"], tune["blocks_per_sm"])
    load_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(local)
    K = 500
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    cfr.cfr_batch_iterate(b, K)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    per_game = cfr.cfr_batch_game_times(b)
    nc = cfr.cfr_batch_exploitability(b)
    info = cfr.cfr_batch_get_info(b)
    # every 256th game's NashConv against the oracle's best responses to that game's average strategy
    import oracle

    checked = list(range(0, len(games), 256))
    dev = [abs(nc[i] - oracle.Oracle(games[i]).exploitability(profile=cfr.cfr_batch_average_strategy(b, i))[0])
           for i in checked]
    out = {"subgames": label, "games": len(games), "nodes_total": int(nodes.sum()), "nodes_min": int(nodes.min()),
           "nodes_max": int(nodes.max()), "nodes_mean": float(nodes.mean()), "variant": "cfr+ (linear averaging)",
           "updates": "alternating" if update_mode else "simultaneous",
           "iterations": K, "seconds": sec, "subgames_per_s": len(games) / sec,
           "node_updates_per_s": float(nodes.sum()) * K / sec,
           "per_subgame_us_per_iteration": {"p50": float(np.percentile(per_game, 50)),
                                            "p99": float(np.percentile(per_game, 99)),
                                            "max": float(per_game.max()),
                                            "note": "a resident subgame's own block time; a subgame of the forest "
                                                    "part advances with the forest, so its iteration time is the "
                                                    "forest's"},
           "exploitability_after": {"median": float(np.median(nc) / 2), "max": float(nc.max() / 2)},
           "oracle_error": {"games_checked": len(checked), "nash_conv_abs_max": float(max(dev)),
                            "note": "GPU NashConv against the oracle's best responses to the GPU's average strategy"},
           "tuning": {k: tune.get(k, -1) for k in ("split_nodes", "threads_per_block", "blocks_per_sm", "fuse_levels",
                                                   "cached")},
           "tuning_trials_us_per_iteration": tune["trials"],
           "forest_part": {"games": info["forest_games"], "nodes": info["forest_nodes"],
                           "algorithmic_bytes_per_iteration": info["forest_bytes_per_iteration"],
                           "achieved_gbs_if_alone": (info["forest_bytes_per_iteration"] * K / sec / 1e9
                                                     if info["forest_games"] == len(games) else None)},
           "host_seconds": {"generate": gen_s, "tune": tune_s, "load": load_s}}
    # the games no shared-memory image can hold (the forest part with every other game resident)
    bres = cfr.cfr_batch_load(games, variant=cfr.CFR_PLUS, device=local, split_nodes=-1, update_mode=update_mode)
    ires = cfr.cfr_batch_get_info(bres)
    out["beyond_shared_memory"] = {"games": ires["forest_games"], "nodes": ires["forest_nodes"],
                                   "node_share": ires["forest_nodes"] / float(nodes.sum())}
    bres.close()
    # time until every subgame's exploitability is at most 1e-3 (evaluations included)
    if ttt:
        b2 = cfr.cfr_batch_load(games, variant=cfr.CFR_PLUS, device=local, split_nodes=tune["split_nodes"],
                                update_mode=update_mode, fuse_levels=fuse)
        cfr.cfr_batch_set_tuning(b2, tune["threads_per_block"], tune["blocks_per_sm"])
        t0, it, worst = time.perf_counter(), 0, float("inf")
        first_s = np.full(len(games), np.nan)                 # per game: the first check at or below 1e-3
        first_it = np.full(len(games), -1, dtype=np.int64)
        while it < 20000 and time.perf_counter() - t0 < 60.0:
            cfr.cfr_batch_iterate(b2, 100)
            it += 100
            ex = cfr.cfr_batch_exploitability(b2) / 2
            now = (ex <= TTT_TARGET) & (first_it < 0)
            first_it[now] = it
            first_s[now] = time.perf_counter() - t0
            worst = float(ex.max())
            if worst <= TTT_TARGET:
                break
        done = first_it >= 0
        out["time_to_exploitability_1e-3_all"] = {"reached": worst <= TTT_TARGET,
                                                  "seconds": time.perf_counter() - t0, "iterations": it,
                                                  "worst_exploitability": worst, "check_every": 100}
        # every subgame advances with the batch, so its own time to the target is when the batch's evaluation
        # first finds it at or below 1e-3: a per-subgame distribution (evaluations included)
        out["per_subgame_time_to_exploitability_1e-3"] = {
            "games_reached": int(done.sum()),
            "seconds": {"p50": float(np.percentile(first_s[done], 50)) if done.any() else None,
                        "p99": float(np.percentile(first_s[done], 99)) if done.any() else None,
                        "max": float(first_s[done].max()) if done.any() else None},
            "iterations": {"p50": float(np.percentile(first_it[done], 50)) if done.any() else None,
                           "p99": float(np.percentile(first_it[done], 99)) if done.any() else None,
                           "max": int(first_it[done].max()) if done.any() else None},
            "note": "first evaluation (every 100 iterations) at which the subgame's exploitability is at most 1e-3"}
        b2.close()
    b.close()
    # the plain full-tree solver on the same games as one tree
    t0 = time.perf_counter()
    root = gamegen.with_chance_root(games)
    s = cfr.cfr_load_tree(root, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32, device=local, update_mode=update_mode,
                          fuse_levels=fuse)
    tree_load_s = time.perf_counter() - t0
    cfr.cfr_iterate(s, 3)
    torch.cuda.synchronize()
    e0.record(stream)
    cfr.cfr_iterate(s, K)
    e1.record(stream)
    torch.cuda.synchronize()
    sec_tree = e0.elapsed_time(e1) / 1e3
    tinfo = cfr.cfr_get_info(s)
    out["plain_full_tree_same_games"] = {"seconds": sec_tree, "iterations": K, "nodes": int(root.num_nodes),
                                         "speedup_of_batched": sec_tree / sec, "host_load_seconds": tree_load_s,
                                         "algorithmic_bytes_per_iteration": tinfo["bytes_per_iteration"],
                                         "achieved_gbs": tinfo["bytes_per_iteration"] * K / sec_tree / 1e9,
                                         "bytes_per_node_iteration": tinfo["bytes_per_iteration"] / root.num_nodes,
                                         "fuse_levels": fuse,
                                         "note": "the games under one uniform chance root, cfr_load_tree + cfr_iterate, "
                                                 "with the batch's tuned fusion setting"}
    s.close()
    return out


def _time_oracle(sub, variant: int, threads: int, seconds: float):
    import oracle

    o = oracle.Oracle(sub)
    o.iterate(1, variant=variant, avg=variant, threads=threads)
    iters, t0 = 0, time.perf_counter()
    while True:
        o.iterate(1, variant=variant, avg=variant, threads=threads)
        iters += 1
        el = time.perf_counter() - t0
        if el >= seconds and iters >= 2:
            break
    return sub.num_nodes * iters / el, iters, el, o.last_threads


def cpu_baseline(g, variant: int, seconds: float = 10.0) -> dict:
    """The oracle on this host's cores, on the first deals of the same workload: all cores (its
    multi-threaded passes, bit-identical to the one-thread walk; the reported value) and one core."""
    threads = oracle_threads()
    sub = oracle_sample(g, 0.5, threads)
    v_all, it_all, el_all, used = _time_oracle(sub, variant, 0, seconds)
    sub1 = oracle_sample(g, 0.5)
    v_one, it_one, el_one, _ = _time_oracle(sub1, variant, 1, seconds)
    return {"value": v_all, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"first {sub.meta['deals']} of {g.meta['deals']} deals ({sub.num_nodes} of {g.num_nodes} nodes), "
                      f"{it_all} full iterations in {el_all:.1f} s on {used} host threads (recursive FP64 oracle, "
                      f"subtrees of the root deal in parallel, sums in the one-thread order)",
            "host_cores": os.cpu_count(),
            "single_core": {"value": v_one, "unit": UNIT, "cores": 1,
                            "sample": f"first {sub1.meta['deals']} deals ({sub1.num_nodes} nodes), {it_one} full "
                                      f"iterations in {el_one:.1f} s, one thread"}}


def oracle_error(g, variant: int, local: int) -> dict:
    """Error of the GPU's results against the FP64 oracle on the bench workload's first deals: from the
    oracle's state after T0 iterations, one GPU iteration in FP32 mode (and one in FP64 mode) against
    the oracle's own next iteration - cumulative regret R, strategy sum S, instantaneous regret r~ and
    the next strategy sigma, each normwise (max |x - y| / max |y| over the players' slots) - and the
    NashConv of the average strategy, absolute: the GPU's against the oracle's after the same step, and
    the GPU's best responses against the oracle's on the GPU's own average strategy."""
    import numpy as np

    import oracle
    import paper_2408_14778_gb300 as cfr

    T0 = 3
    sub = oracle_sample(g, 0.5, oracle_threads())
    o = oracle.Oracle(sub)
    o.iterate(T0, variant=variant, avg=variant, threads=0)
    st0 = o.state()
    o.iterate(1, variant=variant, avg=variant, threads=0)
    ref = o.state()
    nc_ref = o.exploitability()[0]
    keep = np.repeat(sub.infoset_player != 0, sub.infoset_num_actions)

    def nw(x, y):
        x, y = np.where(keep, x, 0.0), np.where(keep, y, 0.0)
        return float(np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-30)) if y.size else 0.0

    out = {"sample": f"first {sub.meta['deals']} deals ({sub.num_nodes} nodes)", "from_iteration": T0,
           "variant": "cfr+ linear averaging" if variant else "vanilla", "nash_conv_oracle": nc_ref,
           "tolerance": {"fp32_normwise": 1e-5, "fp64_normwise": 1e-12, "nash_conv_abs": 1e-6}}
    for name, prec in (("fp32", cfr.CFR_FP32), ("fp64", cfr.CFR_FP64)):
        s = cfr.cfr_load_tree(sub, variant=cfr.CFR_PLUS if variant else cfr.CFR_VANILLA, precision=prec,
                              device=local)
        cfr.cfr_set_state(s, st0["cum_regret"], st0["strat_sum"], T0)
        cfr.cfr_iterate(s, 1)
        gs = cfr.cfr_get_state(s)
        nc = cfr.cfr_exploitability(s)[0]
        avg = cfr.cfr_average_strategy(s)
        nc_br = o.exploitability(profile=avg)[0]
        out[name] = {"cum_regret": nw(gs["cum_regret"], ref["cum_regret"]),
                     "strat_sum": nw(gs["strat_sum"], ref["strat_sum"]),
                     "inst_regret": nw(gs["inst_regret"], ref["inst_regret"]),
                     "sigma": nw(cfr.cfr_current_strategy(s), ref["sigma"]),
                     "nash_conv_abs": abs(nc - nc_ref),
                     "best_response_abs": abs(nc - nc_br)}
        s.close()
    return out


WORKLOAD_TEXT = {
    "bucket3_depth6": "6 ordered deals of 2 of 3 buckets, depth 6, |A| 2-3, u1~U[-2,2]",
    "rank13_depth10": "156 ordered deals of 2 of 13 ranks, depth 10, |A| 3-4, fold/showdown payoffs, pot in {1,2,4,8}",
    "holdem169_depth12": "1326-way deal bucketed to 169, depth 12, |A| 4-5, u1~U[-100,100]",
}
L2_BYTES = 129e6   # GB300's L2


def workload_config(args, g, info=None):
    if info is None:
        l2 = "not applicable (host cores)"
    elif info["device_bytes"] > L2_BYTES:
        l2 = "resident state larger than L2 (no flush needed)"
    else:
        l2 = "resident state fits in L2 (iterations run from L2; not a full-size measurement)"
    c = {"workload": f"{args.workload} (seed {args.seed}): {WORKLOAD_TEXT.get(args.workload, 'seeded synthetic game')}",
         "nodes": g.num_nodes, "variant": "cfr+" if args.variant == "plus" else "vanilla",
         "averaging": "linear" if args.variant == "plus" else "uniform",
         "precision": "fp32 reach/values/regrets, fp64 cumulative sums" if args.precision == "fp32" else "fp64",
         "update": "simultaneous", "l2": l2}
    if info:
        c.update(decision_nodes=info["num_decision"], terminals=info["num_terminal"], infosets=info["num_infosets"],
                 infoset_actions=info["num_q"], levels=info["num_levels"], device_bytes=info["device_bytes"],
                 fused_from_depth=info["fused_from_depth"], fused_tiles=info["fused_tiles"],
                 tail_kernel=info["tail_kernel"],
                 head_depths=info["head_depths"], pair_depth=info["pair_depth"],
                 kernels_per_iteration=info["kernels_per_iteration"])
    return c


def run_reference(args, world, rank):
    if rank != 0:
        return
    import gamegen
    import oracle

    variant = 1 if args.variant == "plus" else 0
    g = gamegen.config(args.workload, seed=args.seed, target_nodes=args.nodes)
    budget = max(0.05, 90.0 / max(args.steps + args.warmup, 1))
    threads = oracle_threads()
    sub = oracle_sample(g, budget, threads)
    o = oracle.Oracle(sub)
    o.iterate(args.warmup, variant=variant, avg=variant, threads=0)
    t0 = time.perf_counter()
    o.iterate(args.steps, variant=variant, avg=variant, threads=0)
    el = time.perf_counter() - t0
    cores = o.last_threads
    value = sub.num_nodes * args.steps / el
    sample = (f"first {sub.meta['deals']} of {g.meta['deals']} deals ({sub.num_nodes} of {g.num_nodes} nodes) per "
              f"step; recursive FP64 oracle on {cores} host threads (subtrees of the root deal in parallel)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(args, g), precision="fp64 throughout (the oracle)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import gamegen
    import paper_2408_14778_gb300 as cfr

    cfr.build()
    torch.cuda.set_device(local)
    variant = cfr.CFR_PLUS if args.variant == "plus" else cfr.CFR_VANILLA
    precision = cfr.CFR_FP32 if args.precision == "fp32" else cfr.CFR_FP64
    g = gamegen.config(args.workload, seed=args.seed, target_nodes=args.nodes)
    s = cfr.cfr_load_tree(g, variant=variant, precision=precision, device=local, fuse_levels=args.fuse_levels,
                          tail_slots=args.tail_slots, head_levels=args.head_levels)
    info = cfr.cfr_get_info(s)
    stream = torch.cuda.current_stream(local)
    cfr.cfr_iterate(s, args.warmup)
    cfr.cfr_synchronize(s)
    launches0 = cfr.cfr_get_info(s)["kernel_launches"]

    sampler = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cfr.cfr_iterate(s, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier(world)
    t = e0.elapsed_time(e1) / 1e3
    t_max = max_over_ranks(t, world, device=f"cuda:{local}")
    N = info["num_nodes"]
    value = world * N * args.steps / t_max
    iter_s = t / args.steps
    # Per-phase times: iterations launched kernel by kernel with CUDA events between the phases on the
    # solver's stream (each is a real iteration), averaged; the dominant phase gives the roofline.
    launches = cfr.cfr_get_info(s)["kernel_launches"]
    ph = [cfr.cfr_phase_times(s) for _ in range(5)]
    names = [p["name"] for p in ph[0]]
    us = np.mean([[p["us"] for p in run] for run in ph], axis=0)
    by = np.array([p["bytes"] for p in ph[0]])
    nfused = info["num_levels"] - info["fused_from_depth"]
    tail_name = {1: "k_tail", 2: "k_tail_stream", 3: "k_tail_slots", 4: "k_tail_slots (bulk regrets)"}.get(
        info["tail_kernel"], "k_fused")
    kernel_of = {cfr.CFR_PHASE_TOPDOWN: "k_topdown", cfr.CFR_PHASE_BOTTOMUP: "k_bottomup",
                 cfr.CFR_PHASE_FUSED: tail_name if nfused == 2 else "k_fused",
                 cfr.CFR_PHASE_OWN: "k_own", cfr.CFR_PHASE_TOPDOWN_PAIR: "k_pair_topdown",
                 cfr.CFR_PHASE_BOTTOMUP_PAIR: "k_pair_bottomup",
                 cfr.CFR_PHASE_UPDATE: "k_update_rows" if args.precision == "fp32" else "k_update"}
    k = int(np.argmax(us))
    peak, peak_src = measured_hbm_peak()
    dom = by[k] / (us[k] * 1e-6) / 1e9
    achieved = info["bytes_per_iteration"] / iter_s / 1e9
    roofline = {"bound": "hbm", "achieved": dom, "peak": peak, "unit": "GB/s", "frac": dom / peak,
                "traffic": recorded_traffic(args.workload, args.precision, names[k]),
                "kernel": f"{names[k]} ({kernel_of[ph[0][k]['kind']]})",
                "algorithmic_bytes_per_launch": float(by[k]), "launch_us": float(us[k]), "peak_source": peak_src,
                "iteration": {"achieved": achieved, "frac": achieved / peak,
                              "algorithmic_bytes": info["bytes_per_iteration"]}}
    phase_us = {n: round(float(u), 2) for n, u in zip(names, us)}

    e2e = None
    if not args.no_e2e:
        # End to end through the C ABI from host arrays: load (validate, lay out, upload the tree), then per
        # step one iteration and a device->host read of its root value, then the average strategy.
        s.close()
        root_buf = torch.zeros(2, dtype=torch.float64, pin_memory=True)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        s2 = cfr.cfr_load_tree(g, variant=variant, precision=precision, device=local, fuse_levels=args.fuse_levels,
                               tail_slots=args.tail_slots, head_levels=args.head_levels)
        cfr.cfr_synchronize(s2)
        load_s = time.perf_counter() - t0
        # each step's root value lands in page-locked memory; step t's is read while step t + 1 runs
        stream = torch.cuda.current_stream(local)
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        values = np.empty(args.steps)
        for t in range(args.steps):
            cfr.cfr_iterate(s2, 1)
            cfr.cfr_root_value_async(s2, root_buf.data_ptr() + 8 * (t % 2))
            ready[t % 2].record(stream)
            if t > 0:
                ready[(t - 1) % 2].synchronize()
                values[t - 1] = root_buf[(t - 1) % 2].item()
        if args.steps > 0:
            ready[(args.steps - 1) % 2].synchronize()
            values[args.steps - 1] = root_buf[(args.steps - 1) % 2].item()
        avg = cfr.cfr_average_strategy(s2)
        el = time.perf_counter() - t0
        el = max_over_ranks(el, world, device=f"cuda:{local}")
        inputs = sum(a.nbytes for a in (g.parent, g.action, g.infoset, g.infoset_player, g.infoset_num_actions,
                                        g.chance_prob, g.utility))
        e2e = {"value": world * N * args.steps / el, "unit": UNIT,
               "h2d_bytes_per_step": inputs / args.steps,
               "d2h_bytes_per_step": 8 + avg.nbytes / args.steps,
               "includes": "cfr_load_tree from host arrays (validation, layout, upload) + per step cfr_iterate(1) + "
                           "cfr_root_value_async into page-locked memory, each step's value read on the host while "
                           "the next step runs, then cfr_average_strategy",
               "root_value_last": float(values[-1]) if args.steps > 0 else None,
               "seconds": el, "load_seconds": load_s, "steps_seconds": el - load_s,
               "steps_only_value": world * N * args.steps / max(el - load_s, 1e-12),
               "note": "value counts cfr_load_tree (host validation and layout of the tree, upload) once; "
                       "steps_only_value the iterations with their per-step reads"}
        s2.close()
        del avg
    else:
        s.close()

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(g, 1 if args.variant == "plus" else 0)
    oerr = None
    if rank == 0 and world == 1 and not args.no_oracle_error:
        oerr = oracle_error(g, 1 if args.variant == "plus" else 0, local)
    ttt = None
    if rank == 0 and world == 1 and not args.no_ttt:
        ttt = time_to_exploitability(args, local)
    batched = None
    if rank == 0 and world == 1 and args.batched_games > 0:
        batched = batched_measurement(args, local)
    leaf = None
    if rank == 0 and world == 1 and not args.no_leaf:
        leaf = learned_leaf_measurement(args, local, ttt)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
                "data": "synthetic", "config": workload_config(args, g, info),
                "iterations_per_s": args.steps / t_max, "roofline": roofline, "cpu_baseline": base, "e2e": e2e,
                "gpu_launches": launches - launches0, "clocks": clocks,
                "parallelism": "replicas" if world > 1 else "single GPU"}
        line["oracle_error"] = oerr
        line["time_to_exploitability"] = ttt
        line["batched"] = batched
        line["learned_leaf"] = leaf
        line["phase_us"] = phase_us
        print(json.dumps(line), flush=True)
    del np


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.only == "network-gemm":
        if rank == 0:
            run_network_gemm_only(args, local)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
