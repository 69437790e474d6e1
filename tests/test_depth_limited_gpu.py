"""Depth-limited solving with the learned leaf network on the GPU (cfr_gather_ranges,
cfr_set_leaf_values, paper_2408_14778_gb300.depth_limited) against the CPU oracle, and what the trained
network gains over an untrained one (GPU tests)."""
import numpy as np
import pytest
import torch

import gamegen
import oracle
import paper_2408_14778_gb300 as cfr
from paper_2408_14778_gb300 import depth_limited as dl
from paritylib import TOL32, normwise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def game():
    return gamegen.config("rank13_depth10", seed=3, target_nodes=30_000)


def _profile(g, rng):
    q0 = np.concatenate([[0], np.cumsum(g.infoset_num_actions)])
    prof = np.zeros(q0[-1])
    c = 0
    for h in range(g.infoset_player.shape[0]):
        n = g.infoset_num_actions[h]
        if g.infoset_player[h] == 0:
            prof[q0[h]:q0[h + 1]] = g.chance_prob[c:c + n]
            c += n
        else:
            w = rng.uniform(0.05, 1.0, n)
            prof[q0[h]:q0[h + 1]] = w / w.sum()
    return prof


def test_gathered_ranges_are_the_oracles_own_reaches(game):
    cut = dl.cut_game(game, depth=3)
    v = cut.view
    top = cut.game
    prof = _profile(top, np.random.default_rng(0))
    s = cfr.cfr_load_tree(top, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32)
    cfr.cfr_set_state(s, prof, np.zeros_like(prof), 0)          # sigma = regret matching of R = prof
    cfr.cfr_set_range_program(s, cut.seg_dst, cut.seg_entries, cut.entry_prod, cut.slots)
    x = torch.zeros((cut.cut_nodes.size, 402), dtype=torch.float32, device="cuda")
    cfr.cfr_gather_ranges(s, x)
    got = x.cpu().numpy().astype(np.float64)
    o = oracle.Oracle(top, record=True)
    o.set_state(prof, np.zeros_like(prof), 0)
    o.iterate(1)
    nodes = o.nodes()
    Pt = cut.top_public.size
    for r, c in enumerate(cut.cut_nodes):
        j = np.searchsorted(cut.top_public, c)
        for p in (1, 2):
            own = np.zeros(13)
            for k in range(v.K):
                own[v.x[p][k]] = nodes[f"own{p}"][1 + k * Pt + j]
            lo = 64 + (p - 1) * 169
            assert normwise(got[r, lo:lo + 13], own / own.sum()) <= TOL32
            assert not got[r, lo + 13:lo + 169].any()


def test_average_strategy_ranges_are_the_oracles(game):
    cut = dl.cut_game(game, depth=3)
    v = cut.view
    top = cut.game
    s = cfr.cfr_load_tree(top, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32)
    cfr.cfr_iterate(s, 7)
    cfr.cfr_set_range_program(s, cut.seg_dst, cut.seg_entries, cut.entry_prod, cut.slots)
    x = torch.zeros((cut.cut_nodes.size, 402), dtype=torch.float32, device="cuda")
    cfr.cfr_gather_ranges(s, x, cfr.CFR_AVERAGE_STRATEGY)
    got = x.cpu().numpy().astype(np.float64)
    avg = cfr.cfr_average_strategy(s)
    o = oracle.Oracle(top, record=True)                 # the oracle's own reaches under that profile
    o.set_state(avg, np.zeros_like(avg), 0)
    o.iterate(1)
    nodes = o.nodes()
    Pt = cut.top_public.size
    for r, c in enumerate(cut.cut_nodes):
        j = np.searchsorted(cut.top_public, c)
        for p in (1, 2):
            own = np.zeros(13)
            for k in range(v.K):
                own[v.x[p][k]] = nodes[f"own{p}"][1 + k * Pt + j]
            lo = 64 + (p - 1) * 169
            assert normwise(got[r, lo:lo + 13], own / own.sum()) <= TOL32


def test_leaf_values_and_one_iteration_match_the_oracle(game):
    cut = dl.cut_game(game, depth=3)
    top = cut.game
    s = cfr.cfr_load_tree(top, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32, fuse_levels=0)
    rows = cut.cut_nodes.size
    src = torch.tensor(np.random.default_rng(1).uniform(-1, 1, size=rows * 338), dtype=torch.float32, device="cuda")
    cfr.cfr_set_leaves(s, cut.leaf_nodes, cut.leaf_src)
    cfr.cfr_set_leaf_values(s, src, 8.0)
    cfr.cfr_iterate(s, 1)
    u1 = cfr.cfr_get_nodes(s)["u1"]
    want = 8.0 * src.cpu().numpy().astype(np.float64)[cut.leaf_src]
    np.testing.assert_array_equal(u1[cut.leaf_nodes], want)
    util = top.utility.copy()
    util[cut.leaf_nodes, 0] = want
    util[cut.leaf_nodes, 1] = -want
    g2 = gamegen.GameDesc(top.parent, top.action, top.infoset, top.infoset_player, top.infoset_num_actions,
                          top.chance_prob, util, {})
    o = oracle.Oracle(g2)
    o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
    gs, os_ = cfr.cfr_get_state(s), o.state()
    for k in ("cum_regret", "strat_sum"):
        assert normwise(gs[k], os_[k]) <= TOL32, k


def test_device_refresh_equals_a_host_refresh(game):
    # the solver's leaf refresh (ranges -> network -> leaves) against the same steps done by hand
    cut = dl.cut_game(game, depth=3)
    net = dl.make_network(hidden=(64, 64), seed=2)
    d = dl.DepthLimitedSolver(cut, net, refresh=1, fuse_levels=0)
    d.iterate(3)                           # refreshed after each iteration, from the average strategy
    x = torch.zeros((cut.cut_nodes.size, 402), dtype=torch.float32, device="cuda")
    x[:, :64] = torch.tensor(cut.embed, dtype=torch.float32, device="cuda")
    cfr.cfr_gather_ranges(d.s, x, cfr.CFR_AVERAGE_STRATEGY)
    y = cfr.cfr_mlp_forward(net, x).cpu().numpy().astype(np.float64)
    u1 = cfr.cfr_get_nodes(d.s)["u1"]
    np.testing.assert_allclose(u1[cut.leaf_nodes], d.umax * y.ravel()[cut.leaf_src], rtol=1e-6, atol=1e-6)


def test_trained_network_beats_an_untrained_one():
    game = gamegen.config("rank13_depth10", seed=3, target_nodes=60_000)
    cut = dl.cut_game(game, depth=4)
    X, Y = dl.generate_samples(cut, per_node=48, iterations=300, seed=4)
    assert np.isfinite(X).all() and np.isfinite(Y).all() and np.abs(Y).max() <= 1.0 + 1e-6
    trained = dl.make_network(hidden=(256, 256, 256), seed=5)
    hist = dl.train(trained, X, Y, steps=800, batch=512, lr=1e-3)
    assert hist[-1] < 0.5 * hist[0], hist
    untrained = dl.make_network(hidden=(256, 256, 256), seed=5)
    # the strategy below the cut: a full-depth solve
    full = cfr.cfr_load_tree(game, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32)
    cfr.cfr_iterate(full, 2000)
    below = cfr.cfr_average_strategy(full)
    expl = {}
    for name, net in (("trained", trained), ("untrained", untrained)):
        d = dl.DepthLimitedSolver(cut, net, refresh=1)
        d.iterate(1000)
        expl[name] = dl.full_game_exploitability(game, dl.combined_strategy(cut, d.average_strategy(), below))
        d.close()
    assert expl["trained"] < 0.5 * expl["untrained"], expl


def test_exact_leaves_reproduce_the_full_solve():
    # leaves fixed to the full solve's own deal values at the cut: the depth-limited solution, completed
    # below the cut by the full solve, is as unexploitable as the full solve (checks the cut game, the
    # leaf indices and the strategy combination end to end)
    game = gamegen.config("rank13_depth10", seed=3, target_nodes=60_000)
    cut = dl.cut_game(game, depth=4)
    full = cfr.cfr_load_tree(game, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32)
    cfr.cfr_iterate(full, 3000)
    below = cfr.cfr_average_strategy(full)
    ex_full = cfr.cfr_exploitability(full)[1]
    y = dl.blueprint_leaf_values(cut, cfr.cfr_get_state(full)["strat_sum"])
    top = dl.solve_with_fixed_leaves(cut, y, 3000)
    ex = dl.full_game_exploitability(game, dl.combined_strategy(cut, top, below))
    assert ex <= 2.0 * ex_full + 2e-3, (ex, ex_full)
