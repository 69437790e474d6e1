"""The multi-threaded host layout builder (used by cfr_load_tree from 2^20 nodes on) against the
one-thread builder: the same arrays bit for bit (a hash of every field), and the same error class, on
games of every family, permuted node ids, forests, wide nodes, and malformed descriptions (no GPU)."""
import numpy as np
import pytest

import gamegen
import paper_2408_14778_gb300 as cfr


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    cfr.build()


def _games():
    yield gamegen.config("bucket3_depth6", seed=1)
    yield gamegen.config("rank13_depth10", seed=2, target_nodes=300_000)
    yield gamegen.config("holdem169_depth12", seed=3, target_nodes=500_000)
    yield gamegen.permute_nodes(gamegen.config("rank13_depth10", seed=4, target_nodes=100_000), 7)
    yield gamegen.public_private(seed=31, num_buckets=13, depth=6, amin=9, amax=12, p_cont=0.45)   # 9-12 actions
    yield gamegen.matrix_game(np.arange(200 * 40, dtype=float).reshape(200, 40) / 8000.0)            # wide nodes
    yield gamegen.public_private(seed=5, num_buckets=3, depth=5, amin=2, amax=3, p_cont=0.7, p_chance=0.3)


@pytest.mark.parametrize("k", range(7))
def test_parallel_builder_equals_serial(k):
    g = list(_games())[k]
    s0, h0, m0 = cfr.cfr_layout_digest(g, 0)
    s1, h1, m1 = cfr.cfr_layout_digest(g, 1)
    assert s0 == s1 == cfr.CFR_OK, (m0, m1)
    assert h0 == h1


def test_parallel_builder_equals_serial_on_a_forest():
    games = gamegen.batch_subgames(40, seed=6, max_nodes=3e4)
    g = gamegen.with_chance_root(games)
    # the combined tree without its root: a forest of the 40 games
    keep = np.arange(1, g.num_nodes)
    parent = np.where(g.parent[keep] == 0, -1, g.parent[keep] - 1).astype(np.int32)
    f = gamegen.GameDesc(parent, g.action[keep], g.infoset[keep], g.infoset_player, g.infoset_num_actions,
                         g.chance_prob, g.utility[keep], {})
    f.infoset_num_actions = f.infoset_num_actions.copy()
    # the first infoset was the root's chance deal: no nodes left; keep its table entry (no nodes is valid)
    s0, h0, m0 = cfr.cfr_layout_digest(f, 0, forest=True)
    s1, h1, m1 = cfr.cfr_layout_digest(f, 1, forest=True)
    assert s0 == s1 == cfr.CFR_OK, (m0, m1)
    assert h0 == h1


def _broken(g, **changes):
    d = dict(parent=g.parent.copy(), action=g.action.copy(), infoset=g.infoset.copy(),
             infoset_player=g.infoset_player.copy(), infoset_num_actions=g.infoset_num_actions.copy(),
             chance_prob=g.chance_prob.copy(), utility=g.utility.copy())
    d.update(changes)
    return gamegen.GameDesc(**d)


def test_parallel_builder_reports_the_same_errors():
    g = gamegen.config("rank13_depth10", seed=2, target_nodes=200_000)
    n = g.num_nodes
    par = g.parent.copy(); par[n // 2] = -1                              # a second root
    act = g.action.copy(); kids = np.nonzero(g.parent == g.parent[n - 1])[0]; act[kids[1]] = act[kids[0]]
    inf = g.infoset.copy(); inf[n - 5] = g.infoset_player.shape[0] + 3   # infoset out of range
    ut = g.utility.copy(); t = np.nonzero(g.infoset < 0)[0][10]; ut[t, 1] = -ut[t, 0] + 1.0   # not zero-sum
    ut2 = g.utility.copy(); ut2[t, 0] = np.inf
    cases = [_broken(g, parent=par), _broken(g, action=act), _broken(g, infoset=inf), _broken(g, utility=ut),
             _broken(g, utility=ut2)]
    for b in cases:
        s0, _, m0 = cfr.cfr_layout_digest(b, 0)
        s1, _, m1 = cfr.cfr_layout_digest(b, 1)
        assert s0 == s1 != cfr.CFR_OK, (m0, m1)
        assert m0.split(":")[0].split(" ")[0] == m1.split(":")[0].split(" ")[0], (m0, m1)
