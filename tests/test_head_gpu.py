"""The shallowest depths in one launch per direction (k_head_topdown / k_head_bottomup, FP32 mode: each
block walks the subtrees of a range of root children, the last block to finish taking the root, or, in a
batch's forest part, the subtrees of a range of games' roots) against
the oracle: a first iteration and a step from the oracle's state at T = 3 (FP32 step parity; two FP32
runs' trajectories part after a few iterations whatever their kernels, since the atomics' order differs
and regret matching amplifies it) (GPU tests)."""
import numpy as np
import pytest

import gamegen
import oracle
import paper_2408_14778_gb300 as cfr
from paritylib import TOL32, compare_nodes, compare_state, compare_step, fp32_regret_budget_check, normwise

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant,alt", [(cfr.CFR_PLUS, False), (cfr.CFR_VANILLA, False), (cfr.CFR_PLUS, True)],
                         ids=["cfr+", "vanilla", "cfr+_alternating"])
@pytest.mark.parametrize("fuse", [0, -1])
@pytest.mark.parametrize("name,nodes,levels", [("rank13_depth10", 200_000, -1), ("holdem169_depth12", 2_000_000, -1),
                                               ("holdem169_depth12", 2_000_000, 1), ("bucket3_depth6", None, -1)])
def test_head_matches_oracle(name, nodes, levels, fuse, variant, alt):
    g = gamegen.config(name, seed=2, target_nodes=nodes)
    mode = cfr.CFR_ALTERNATING if alt else cfr.CFR_SIMULTANEOUS
    s = cfr.cfr_load_tree(g, variant=variant, precision=cfr.CFR_FP32, fuse_levels=fuse, record_nodes=True,
                          head_levels=levels, update_mode=mode)
    info = cfr.cfr_get_info(s)
    assert info["head_depths"] == 2 if levels == 1 else info["head_depths"] >= 2
    o = oracle.Oracle(g, record=True)
    avg = oracle.AVG_LINEAR if variant == cfr.CFR_PLUS else oracle.AVG_UNIFORM
    o.iterate(1, variant=variant, avg=avg, alternating=alt)
    cfr.cfr_iterate(s, 1)
    compare_step(s, o, g, alt)
    o.iterate(2, variant=variant, avg=avg, alternating=alt)
    st = o.state()
    cfr.cfr_set_state(s, st["cum_regret"], st["strat_sum"], st["iteration"])
    o.iterate(1, variant=variant, avg=avg, alternating=alt)
    cfr.cfr_iterate(s, 1)
    compare_step(s, o, g, alt)
    assert np.isfinite(cfr.cfr_root_value(s))


def test_head_levels_and_eligibility():
    g = gamegen.config("rank13_depth10", seed=2, target_nodes=200_000)
    info = lambda **kw: cfr.cfr_get_info(cfr.cfr_load_tree(g, **kw))   # noqa: E731
    assert info(precision=cfr.CFR_FP32)["head_depths"] >= 2                            # on by default
    assert info(precision=cfr.CFR_FP32, head_levels=0)["head_depths"] == 0
    assert info(precision=cfr.CFR_FP32, head_levels=3)["head_depths"] == 4               # the root + 3 depths
    assert info(precision=cfr.CFR_FP64)["head_depths"] == 0
    # a root with a terminal child: no head
    util = np.zeros((5, 2))
    util[[1, 3, 4], 0] = [0.5, 1.0, -1.0]
    util[:, 1] = -util[:, 0]
    t = gamegen.GameDesc(np.array([-1, 0, 0, 2, 2], np.int32), np.array([-1, 0, 1, 0, 1], np.int32),
                         np.array([0, -1, 1, -1, -1], np.int32), np.array([0, 1], np.int8), np.array([2, 2], np.int32),
                         np.array([0.5, 0.5]), util)
    assert cfr.cfr_get_info(cfr.cfr_load_tree(t, precision=cfr.CFR_FP32))["head_depths"] == 0
    # a matrix game (player root, wide): the root's regrets come from the last block of the bottom-up head
    m = gamegen.matrix_game(np.random.default_rng(3).uniform(-1, 1, size=(200, 3)))
    s = cfr.cfr_load_tree(m, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32)
    assert cfr.cfr_get_info(s)["head_depths"] == 2
    o = oracle.Oracle(m)
    o.iterate(3, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
    cfr.cfr_iterate(s, 3)
    compare_state(s, o, TOL32, m)


def test_head_converges_like_the_oracle():
    # Over many iterations FP32 rounding re-decides near-tied regrets, so two FP32 runs' trajectories part
    # whatever their kernels; the solution quality must not: with the head and without it, NashConv of the
    # average strategy tracks the FP64 oracle's, and the GPU's best responses agree with the oracle's.
    # (On some seeds every FP32 run, with the head or without, wanders to 0.85-1.3x the oracle's NashConv
    # around T = 400; this seed's runs stay within 0.1%.)
    g = gamegen.config("rank13_depth10", seed=6, target_nodes=200_000)
    o = oracle.Oracle(g)
    a = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32)
    b = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32, head_levels=0)
    assert cfr.cfr_get_info(a)["head_depths"] >= 2 and cfr.cfr_get_info(b)["head_depths"] == 0
    for T in (100, 400):
        o.iterate(T - o.state()["iteration"], variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
        nc_o, _ = o.exploitability()
        for x in (a, b):
            cfr.cfr_iterate(x, T - cfr.cfr_get_info(x)["iteration"])
            nc_g, _ = cfr.cfr_exploitability(x)
            assert nc_g <= 1.1 * nc_o + 1e-4, (T, nc_g, nc_o)
            nc_chk, _ = o.exploitability(cfr.cfr_average_strategy(x))
            assert abs(nc_chk - nc_g) <= 1e-6


@pytest.mark.parametrize("variant,alt", [(cfr.CFR_PLUS, False), (cfr.CFR_VANILLA, False), (cfr.CFR_PLUS, True)],
                         ids=["cfr+", "vanilla", "cfr+_alternating"])
def test_forest_head_matches_oracle_game_by_game(variant, alt):
    # A batch's forest part (every game at split 1): blocks take ranges of the games' roots, and depth 0 is
    # walked like the others (no root step).  Games of 1e2-3e4 nodes and depths 4-10 (chance roots), so that
    # blocks hold subtrees of unequal sizes and depths, and two matrix games (player roots).
    rng = np.random.default_rng(21)
    games = gamegen.batch_subgames(30, seed=21, max_nodes=3e4)
    games[3:3] = [gamegen.matrix_game(rng.uniform(-1, 1, size=(8, 3)))]
    games.append(gamegen.matrix_game(rng.uniform(-1, 1, size=(32, 5))))
    mode = cfr.CFR_ALTERNATING if alt else cfr.CFR_SIMULTANEOUS
    runs = {}
    for levels in (-1, 0):
        b = cfr.cfr_batch_load(games, variant=variant, split_nodes=1, update_mode=mode, head_levels=levels)
        info = cfr.cfr_batch_get_info(b)
        assert info["forest_games"] == len(games)
        assert (info["forest_head_depths"] >= 2) if levels else info["forest_head_depths"] == 0
        cfr.cfr_batch_iterate(b, 1)
        runs[levels] = [cfr.cfr_batch_get_state(b, i) for i in range(len(games))]
    avg = oracle.AVG_LINEAR if variant == cfr.CFR_PLUS else oracle.AVG_UNIFORM
    for i, g in enumerate(games):
        o = oracle.Oracle(g)
        o.iterate(1, variant=variant, avg=avg, alternating=alt)
        os_ = o.state()
        p1 = np.repeat(g.infoset_player == 1, g.infoset_num_actions)
        sel = p1 if alt else np.ones_like(p1)
        for levels, states in runs.items():
            gs = states[i]
            for k in ("cum_regret", "strat_sum"):
                assert normwise(gs[k][sel], os_[k][sel]) <= TOL32, (i, levels, k)
            if not alt:
                fp32_regret_budget_check(g, gs, os_, _max_depth(g))


def _max_depth(g):
    d = np.full(g.num_nodes, -1)
    d[g.parent < 0] = 0
    while (d < 0).any():
        todo = np.nonzero(d < 0)[0]
        ok = d[g.parent[todo]] >= 0
        d[todo[ok]] = d[g.parent[todo[ok]]] + 1
    return int(d.max())


@pytest.mark.parametrize("variant", [cfr.CFR_VANILLA, cfr.CFR_LINEAR, cfr.CFR_DISCOUNTED],
                         ids=["vanilla", "linear", "discounted"])
def test_iterations_per_graph_launch_match_the_oracle(variant):
    # cfr_iterate(s, 5) replays a graph of four captured iterations (each with the split update) and then the
    # one-iteration graph; from the start, they must land where the oracle's five iterations do, each update
    # weighted by its own T.
    # The hold'em-shaped family draws its payoffs from a continuous distribution and the variants without
    # clipping keep regret matching well conditioned (no tie of action values or regret sum of exactly 0 in
    # FP64 against an FP32 residue, which fold/showdown payoffs and CFR+'s clipping make common), so five FP32
    # iterations stay within FP32 rounding of the oracle; an update at the wrong T or with regrets of the
    # wrong iteration moves R by tens of percent.
    g = gamegen.config("holdem169_depth12", seed=2, target_nodes=2_000_000)
    s = cfr.cfr_load_tree(g, variant=variant, precision=cfr.CFR_FP32)
    assert cfr.cfr_get_info(s)["head_depths"] >= 2
    o = oracle.Oracle(g)
    o.iterate(5, variant=variant, avg=oracle.AVG_UNIFORM if variant == cfr.CFR_VANILLA else oracle.AVG_LINEAR)
    cfr.cfr_iterate(s, 5)
    gs, os_ = cfr.cfr_get_state(s), o.state()
    assert gs["iteration"] == os_["iteration"] == 5
    for k in ("cum_regret", "strat_sum", "inst_regret"):
        assert normwise(gs[k], os_[k]) <= 1e-4, (k, normwise(gs[k], os_[k]))
