"""Batched solving (cfr_batch_*) against the oracle, game by game (GPU tests).

Every game of a batch is an independent CFR run: its first iteration is compared with the oracle's
under the FP32 budget of paritylib; after more iterations the batched best response is compared with
the oracle's best response on the batch's own average strategy, and the exploitability with the oracle
run's.
"""
import numpy as np
import pytest

import gamegen
import oracle
import paper_2408_14778_gb300 as cfr
from paritylib import TOL32, TOL_EXPL, fp32_regret_budget_check, normwise

pytestmark = pytest.mark.gpu


def _games(n=12, seed=5, max_nodes=5e3):
    return gamegen.batch_subgames(n, seed=seed, max_nodes=max_nodes)


def _max_depth(g):
    d = np.full(g.num_nodes, -1)
    d[g.parent < 0] = 0
    while (d < 0).any():
        todo = np.nonzero(d < 0)[0]
        ok = d[g.parent[todo]] >= 0
        d[todo[ok]] = d[g.parent[todo[ok]]] + 1
    return int(d.max())


@pytest.mark.parametrize("variant", [cfr.CFR_VANILLA, cfr.CFR_PLUS, cfr.CFR_LINEAR, cfr.CFR_DISCOUNTED])
def test_first_iteration_matches_oracle(variant):
    games = _games()
    b = cfr.cfr_batch_load(games, variant=variant)
    cfr.cfr_batch_iterate(b, 1)
    avg = oracle.AVG_UNIFORM if variant == cfr.CFR_VANILLA else oracle.AVG_LINEAR
    for i, g in enumerate(games):
        o = oracle.Oracle(g)
        o.iterate(1, variant=variant, avg=avg, dcfr=(1.5, 0.0, 2.0))
        gs, os_ = cfr.cfr_batch_get_state(b, i), o.state()
        assert gs["iteration"] == os_["iteration"] == 1
        for k in ("cum_regret", "strat_sum"):
            assert normwise(gs[k], os_[k]) <= TOL32, (i, k)
        fp32_regret_budget_check(g, gs, os_, _max_depth(g))


def test_exploitability_and_convergence_track_the_oracle():
    games = _games(10, seed=6)
    b = cfr.cfr_batch_load(games, variant=cfr.CFR_PLUS)
    cfr.cfr_batch_iterate(b, 150)
    nc = cfr.cfr_batch_exploitability(b)
    assert nc.shape == (len(games),)
    for i, g in enumerate(games):
        o = oracle.Oracle(g)
        avg = cfr.cfr_batch_average_strategy(b, i)
        nc_chk, _ = o.exploitability(avg)                 # the oracle's best response on the batch's strategy
        assert abs(nc_chk - nc[i]) <= TOL_EXPL, (i, nc_chk, nc[i])
        o.iterate(150, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
        nc_o, _ = o.exploitability()
        assert nc[i] <= 1.1 * nc_o + 1e-4, (i, nc[i], nc_o)


def test_batch_of_one_equals_the_single_game_solver():
    g = gamegen.public_private(seed=7, num_buckets=3, depth=9, amin=2, amax=4, p_cont=0.7)   # 6-way deal
    b = cfr.cfr_batch_load([g], variant=cfr.CFR_PLUS)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32, fuse_levels=0)
    o = oracle.Oracle(g)
    for T in (1, 2):
        cfr.cfr_batch_iterate(b, 1)
        cfr.cfr_iterate(s, 1)
        o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
        gb, gsn, os_ = cfr.cfr_batch_get_state(b, 0), cfr.cfr_get_state(s), o.state()
        for k in ("cum_regret", "strat_sum"):
            assert normwise(gb[k], os_[k]) <= TOL32 and normwise(gsn[k], os_[k]) <= TOL32
    assert abs(cfr.cfr_batch_exploitability(b)[0] - cfr.cfr_exploitability(s)[0]) <= 1e-5


def test_autotune_keeps_the_state_and_caches(tmp_path):
    games = _games(40, seed=8)
    b = cfr.cfr_batch_load(games, variant=cfr.CFR_PLUS)
    cfr.cfr_batch_iterate(b, 3)
    before = [cfr.cfr_batch_get_state(b, i) for i in (0, 17, 39)]
    cache = str(tmp_path / "tune.json")
    r = cfr.cfr_batch_autotune(b, trial_iterations=2, cache_path=cache)
    assert not r["cached"] and r["threads_per_block"] in (64, 128, 256) and r["us_per_iteration"] > 0
    after = [cfr.cfr_batch_get_state(b, i) for i in (0, 17, 39)]
    for x, y in zip(before, after):
        assert x["iteration"] == y["iteration"] == 3
        np.testing.assert_array_equal(x["cum_regret"], y["cum_regret"])
        np.testing.assert_array_equal(x["strat_sum"], y["strat_sum"])
    info = cfr.cfr_batch_get_info(b)
    assert info["tuned"] == 1 and info["threads_per_block"] == r["threads_per_block"]
    b2 = cfr.cfr_batch_load(games, variant=cfr.CFR_PLUS)
    r2 = cfr.cfr_batch_autotune(b2, cache_path=cache)
    assert r2["cached"] and r2["threads_per_block"] == r["threads_per_block"]
    cfr.cfr_batch_iterate(b2, 5)
    t = cfr.cfr_batch_game_times(b2)
    assert t.shape == (len(games),) and np.all(t > 0)
    assert cfr.cfr_batch_get_info(b2)["iteration"] == 5


@pytest.mark.parametrize("split", [-1, 1])
def test_alternating_updates_match_oracle(split):
    # resident games (split -1) and the forest part (split 1): two iterations of alternating CFR+
    games = _games(8, seed=13)
    b = cfr.cfr_batch_load(games, variant=cfr.CFR_PLUS, split_nodes=split, update_mode=cfr.CFR_ALTERNATING)
    cfr.cfr_batch_iterate(b, 1)
    for i, g in enumerate(games):
        o = oracle.Oracle(g)
        o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR, alternating=True)
        gs, os_ = cfr.cfr_batch_get_state(b, i), o.state()
        # player 1's pass starts from the same (uniform) strategy: compared to the FP32 tolerance; player
        # 2's pass follows player 1's new strategy, where regret matching may amplify FP32 rounding (the
        # single-game tests bound it per infoset), so it is judged by the convergence below
        p1 = np.repeat(g.infoset_player == 1, g.infoset_num_actions)
        for k in ("cum_regret", "strat_sum"):
            assert normwise(gs[k][p1], os_[k][p1]) <= TOL32, (i, k)
    cfr.cfr_batch_iterate(b, 300)
    nc = cfr.cfr_batch_exploitability(b)
    for i, g in enumerate(games):
        o = oracle.Oracle(g)
        o.iterate(301, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR, alternating=True)
        assert nc[i] <= 1.1 * o.exploitability()[0] + 1e-4, (i, nc[i])


def test_unsupported_configurations():
    games = _games(3, seed=9)
    for kw in (dict(precision=cfr.CFR_FP64),):
        cfg = cfr._Config()
        cfr.lib().cfr_config_init(cfr.ctypes.byref(cfg))
        for k, v in kw.items():
            setattr(cfg, k, v)
        descs = [cfr._Desc(g) for g in games]
        arr = (cfr._GameDesc * len(descs))(*[d.c for d in descs])
        h = cfr._P()
        assert cfr.lib().cfr_batch_load(arr, len(descs), cfr.ctypes.byref(cfg), cfr.ctypes.byref(h)) == \
            cfr.CFR_ERR_UNSUPPORTED
    with pytest.raises(cfr.CfrError) as e:
        cfr.cfr_batch_set_tuning(cfr.cfr_batch_load(games), 512)
    assert e.value.status == cfr.CFR_ERR_INVALID


def test_games_that_cannot_be_resident_run_in_the_forest():
    # a node of 40 actions, and a game too large for one block's shared memory, go to the forest part
    # whatever the split; the rest stay resident
    wide = gamegen.matrix_game(np.arange(80, dtype=float).reshape(2, 40) / 80.0)
    big = gamegen.batch_subgames(1, seed=11, min_nodes=40000, max_nodes=60000)[0]
    games = [wide, big] + _games(5, seed=12)
    b = cfr.cfr_batch_load(games, variant=cfr.CFR_PLUS, split_nodes=-1)
    info = cfr.cfr_batch_get_info(b)
    assert info["forest_games"] == 2 and 0 < info["smem_bytes"] <= 200 * 1024
    cfr.cfr_batch_iterate(b, 2)
    for i, g in enumerate(games):
        o = oracle.Oracle(g)
        o.iterate(2, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
        gs, os_ = cfr.cfr_batch_get_state(b, i), o.state()
        for k in ("cum_regret", "strat_sum"):
            assert normwise(gs[k], os_[k]) <= TOL32, (i, k)


def test_size_split_runs_both_parts_like_the_oracle():
    # games of >= 1500 nodes go to the forest part, the rest to the persistent kernel
    games = gamegen.batch_subgames(14, seed=10, max_nodes=2e4)
    sizes = np.array([g.num_nodes for g in games])
    assert (sizes >= 1500).any() and (sizes < 1500).any()
    b = cfr.cfr_batch_load(games, variant=cfr.CFR_PLUS, split_nodes=1500)
    info = cfr.cfr_batch_get_info(b)
    assert info["forest_games"] == int((sizes >= 1500).sum()) and info["num_games"] == len(games)
    cfr.cfr_batch_iterate(b, 1)
    for i, g in enumerate(games):
        o = oracle.Oracle(g)
        o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
        gs, os_ = cfr.cfr_batch_get_state(b, i), o.state()
        for k in ("cum_regret", "strat_sum"):
            assert normwise(gs[k], os_[k]) <= TOL32, (i, k)
        fp32_regret_budget_check(g, gs, os_, _max_depth(g))
    cfr.cfr_batch_iterate(b, 60)
    nc = cfr.cfr_batch_exploitability(b)
    for i, g in enumerate(games):
        nc_chk, _ = oracle.Oracle(g).exploitability(cfr.cfr_batch_average_strategy(b, i))
        assert abs(nc_chk - nc[i]) <= TOL_EXPL, (i, nc_chk, nc[i])
    t = cfr.cfr_batch_game_times(b)
    assert np.all(t > 0)
    assert len(set(np.round(t[sizes >= 1500], 6))) == 1          # the forest part advances together


@pytest.mark.parametrize("fuse", [-1, 2], ids=["tail_and_pair", "tail_only"])
def test_forest_fusion_settings_match_oracle(fuse):
    # The batch autotuner also chooses the forest part's fusion (cfr_config.fuse_levels): -1 fuses the last two
    # depths and runs the two above them as a pair, 2 fuses the last two only.  Games large enough that the pair
    # applies (checked on the same games under one chance root), all in the forest part, first iteration and a
    # step from the oracle's T = 3 state game by game.
    # (the head limited to a few depths, so that the pair's depths lie below it)
    games = gamegen.batch_subgames(48, seed=17, min_nodes=2e3, max_nodes=6e4)
    root = gamegen.with_chance_root(games)
    info = cfr.cfr_get_info(cfr.cfr_load_tree(root, precision=cfr.CFR_FP32, fuse_levels=fuse, head_levels=3))
    assert info["pair_depth"] == (-1 if fuse == 2 else info["fused_from_depth"] - 2)
    b = cfr.cfr_batch_load(games, variant=cfr.CFR_PLUS, split_nodes=1, fuse_levels=fuse, head_levels=3)
    assert cfr.cfr_batch_get_info(b)["forest_games"] == len(games)
    cfr.cfr_batch_iterate(b, 1)
    for i, g in enumerate(games):
        o = oracle.Oracle(g)
        o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
        gs, os_ = cfr.cfr_batch_get_state(b, i), o.state()
        for k in ("cum_regret", "strat_sum"):
            assert normwise(gs[k], os_[k]) <= TOL32, (i, k)
        fp32_regret_budget_check(g, gs, os_, _max_depth(g))
    b.close()
