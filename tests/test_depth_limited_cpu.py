"""Host logic of depth-limited solving (paper_2408_14778_gb300.depth_limited) against the CPU oracle.

The cut game, the subgames and the range program are index constructions; each is checked against
the oracle on the full game: with the leaves set to the full game's subtree values under a profile,
the depth-limited game reproduces the full game's node values and reaches above the cut; a subgame's
deal values equal the full game's at the cut node; the range program's products equal the oracle's own
reaches (Eq. 4) at the cut nodes.
"""
import numpy as np
import pytest

import gamegen
import oracle
from paper_2408_14778_gb300 import depth_limited as dl


@pytest.fixture(scope="module")
def game():
    return gamegen.config("rank13_depth10", seed=3, target_nodes=30_000)


def _random_profile(g, rng):
    """Random player strategies (positive, normalised per infoset); chance slots sigma_0."""
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


def _evaluate(g, prof):
    """Oracle node values and reaches under a fixed profile (regret matching of R = profile)."""
    o = oracle.Oracle(g, record=True)
    o.set_state(prof, np.zeros_like(prof), 0)
    o.iterate(1)
    return o.nodes()


def test_cut_game_reproduces_the_full_game_above_the_cut(game):
    cut = dl.cut_game(game, depth=3)
    v = cut.view
    assert cut.cut_nodes.size > 0 and v.K == 156 and v.nx == {1: 13, 2: 13}
    rng = np.random.default_rng(0)
    prof = _random_profile(game, rng)
    full = _evaluate(game, prof)
    top = cut.game
    util = top.utility.copy()
    # leaf (k, c) <- the full game's value of node (k, c)
    Pt = cut.top_public.size
    k_of = (cut.leaf_nodes - 1) // Pt
    j_of = (cut.leaf_nodes - 1) % Pt
    full_ids = v.node(k_of, cut.top_public[j_of])
    util[cut.leaf_nodes, 0] = full["u1"][full_ids]
    util[cut.leaf_nodes, 1] = -util[cut.leaf_nodes, 0]
    top = gamegen.GameDesc(top.parent, top.action, top.infoset, top.infoset_player, top.infoset_num_actions,
                           top.chance_prob, util, {})
    tprof = prof[cut.slot_to_full]
    part = _evaluate(top, tprof)
    kk = np.repeat(np.arange(v.K), Pt)
    ids = np.concatenate([[0], v.node(kk, np.tile(cut.top_public, v.K))])
    for key in ("u1", "own1", "own2", "cf1", "cf2"):
        np.testing.assert_allclose(part[key], full[key][ids], rtol=1e-12, atol=1e-15, err_msg=key)
    # the leaves' value indices name each deal's private-state pair
    np.testing.assert_array_equal(cut.leaf_src % 338, v.x[1][k_of] * 13 + v.x[2][k_of])
    np.testing.assert_array_equal(cut.leaf_src // 338, np.searchsorted(cut.cut_nodes, cut.top_public[j_of]))


def test_range_program_gives_the_own_reaches_at_the_cut(game):
    cut = dl.cut_game(game, depth=3)
    v = cut.view
    prof = _random_profile(game, np.random.default_rng(1))
    full = _evaluate(game, prof)
    tprof = prof[cut.slot_to_full]
    out = np.zeros(cut.cut_nodes.size * 402)
    for s in range(cut.seg_dst.size):           # the program, evaluated by its definition
        e0, e1 = cut.seg_entries[s], cut.seg_entries[s + 1]
        vals = np.array([np.prod(tprof[cut.slots[cut.entry_prod[e]:cut.entry_prod[e + 1]]]) for e in range(e0, e1)])
        out[cut.seg_dst[s]:cut.seg_dst[s] + e1 - e0] = vals / vals.sum()
    out = out.reshape(-1, 402)
    for r, c in enumerate(cut.cut_nodes):
        for p in (1, 2):
            own = np.zeros(13)
            for k in range(v.K):
                own[v.x[p][k]] = full[f"own{p}"][v.node(k, c)]
            np.testing.assert_allclose(out[r, 64 + (p - 1) * 169:64 + (p - 1) * 169 + 13], own / own.sum(), rtol=1e-12)
        assert not out[r, 64 + 13:64 + 169].any() and not out[r, 64 + 169 + 13:].any()


def test_subgame_values_equal_the_full_game_at_the_cut_node(game):
    cut = dl.cut_game(game, depth=3)
    v = cut.view
    prof = _random_profile(game, np.random.default_rng(2))
    full = _evaluate(game, prof)
    rng = np.random.default_rng(3)
    for c in cut.cut_nodes[:3]:
        r1, r2 = dl.random_ranges(rng, 13, 1)[0], dl.random_ranges(rng, 13, 1)[0]
        sub, s2f = dl.subgame(v, int(c), r1, r2, return_slots=True)
        sprof = np.where(s2f >= 0, prof[np.maximum(s2f, 0)], 0.0)
        sprof[:v.K] = sub.chance_prob[:v.K]           # the root deal's slots: its chance probabilities
        part = _evaluate(sub, sprof)
        D = v.descendants(int(c)).size
        np.testing.assert_allclose(part["u1"][1 + np.arange(v.K) * D], full["u1"][v.node(np.arange(v.K), c)],
                                   rtol=1e-12, atol=1e-14)
        w = v.deal_prob * r1[v.x[1]] * r2[v.x[2]]
        np.testing.assert_allclose(sub.chance_prob[:v.K], w / w.sum(), rtol=1e-14)
