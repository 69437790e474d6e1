"""The two depths above the fused last two as a pair (k_pair_topdown / k_pair_bottomup, FP32 mode: one
top-down and one bottom-up launch for depths m and m+1, depth m+1's reaches and values kept on chip and
recomputed by the bottom-up launch) against the oracle: a first iteration and a step from the oracle's
state at T = 3, with and without the nodes recorded, for CFR+, vanilla CFR and alternating updates; the
phase timer's pair phases and their bytes; when the pair is planned (GPU tests)."""
import numpy as np
import pytest

import gamegen
import oracle
import paper_2408_14778_gb300 as cfr
from paritylib import TOL32, compare_state, compare_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rank13():
    # 2.03e6 nodes, 10 decision depths: the tail at depths 8-9, the pair at 6-7 (15 912 and 47 112
    # decision nodes) once the head is limited to the root and 3 depths
    return gamegen.config("rank13_depth10", seed=0)


@pytest.mark.parametrize("variant,alt", [(cfr.CFR_PLUS, False), (cfr.CFR_VANILLA, False), (cfr.CFR_PLUS, True)],
                         ids=["cfr+", "vanilla", "cfr+_alternating"])
@pytest.mark.parametrize("record", [True, False], ids=["record", "no_record"])
def test_pair_matches_oracle(rank13, variant, alt, record):
    g = rank13
    mode = cfr.CFR_ALTERNATING if alt else cfr.CFR_SIMULTANEOUS
    s = cfr.cfr_load_tree(g, variant=variant, precision=cfr.CFR_FP32, record_nodes=record, head_levels=3,
                          update_mode=mode)
    info = cfr.cfr_get_info(s)
    assert info["pair_depth"] == info["fused_from_depth"] - 2 == 6 and info["head_depths"] == 4
    o = oracle.Oracle(g, record=record)
    avg = oracle.AVG_LINEAR if variant == cfr.CFR_PLUS else oracle.AVG_UNIFORM
    o.iterate(1, variant=variant, avg=avg, alternating=alt)
    cfr.cfr_iterate(s, 1)
    compare_step(s, o, g, alt, nodes=record)
    o.iterate(2, variant=variant, avg=avg, alternating=alt)
    st = o.state()
    cfr.cfr_set_state(s, st["cum_regret"], st["strat_sum"], st["iteration"])
    o.iterate(1, variant=variant, avg=avg, alternating=alt)
    cfr.cfr_iterate(s, 1)
    compare_step(s, o, g, alt, nodes=record)
    s.close()


def test_pair_with_head_on_the_hold_em_family():
    # holdem169_depth12 at 2e6 nodes with the head at the root and depth 1: the pair at depths 8-9 between
    # per-depth streamed launches and the tail, several steps from the oracle's states
    g = gamegen.config("holdem169_depth12", seed=3, target_nodes=2_000_000)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32, head_levels=1)
    info = cfr.cfr_get_info(s)
    assert info["pair_depth"] == info["fused_from_depth"] - 2 == 8
    o = oracle.Oracle(g)
    for _ in range(3):
        o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
        cfr.cfr_iterate(s, 1)
        compare_state(s, o, TOL32, g)
        st = o.state()
        cfr.cfr_set_state(s, st["cum_regret"], st["strat_sum"], st["iteration"])
    s.close()


def test_pair_phase_times_and_bytes(rank13):
    g = rank13
    o = oracle.Oracle(g)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32, head_levels=3)
    info = cfr.cfr_get_info(s)
    m, L, f = info["pair_depth"], info["num_levels"], info["fused_from_depth"]
    o.iterate(2, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
    st = o.state()
    cfr.cfr_set_state(s, st["cum_regret"], st["strat_sum"], st["iteration"])
    ph = cfr.cfr_phase_times(s)                               # the third iteration, kernel by kernel
    o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
    compare_state(s, o, TOL32, g)
    kinds = [p["kind"] for p in ph]
    assert kinds == ([cfr.CFR_PHASE_OWN] + [cfr.CFR_PHASE_TOPDOWN] * m + [cfr.CFR_PHASE_TOPDOWN_PAIR] +
                     [cfr.CFR_PHASE_FUSED] + [cfr.CFR_PHASE_BOTTOMUP_PAIR] + [cfr.CFR_PHASE_BOTTOMUP] * m +
                     [cfr.CFR_PHASE_UPDATE])
    assert [p["depth"] for p in ph if p["kind"] in (cfr.CFR_PHASE_TOPDOWN_PAIR, cfr.CFR_PHASE_BOTTOMUP_PAIR)] == [m, m]
    assert f == m + 2 < L
    assert all(p["us"] > 0 for p in ph)
    assert abs(sum(p["bytes"] for p in ph) - info["bytes_per_iteration"]) <= 1
    # the pair's byte model against the per-depth launches of the same two depths: depth m+1's reaches are
    # neither written nor read back (28 bytes per node of depth m+1 fewer, 4 more per node of depth m)
    t = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32, head_levels=3, fuse_levels=2)
    assert cfr.cfr_get_info(t)["pair_depth"] == -1
    ph2 = cfr.cfr_phase_times(t)
    per_depth = sum(p["bytes"] for p in ph2 if p["kind"] in (cfr.CFR_PHASE_TOPDOWN, cfr.CFR_PHASE_BOTTOMUP)
                    and p["depth"] in (m, m + 1))
    pair = sum(p["bytes"] for p in ph if p["kind"] in (cfr.CFR_PHASE_TOPDOWN_PAIR, cfr.CFR_PHASE_BOTTOMUP_PAIR))
    depth = _depths(g)
    nd = lambda d: int(((depth == d) & (g.infoset >= 0)).sum())   # noqa: E731
    assert per_depth - pair == 28 * nd(m + 1) - 4 * nd(m)
    assert info["kernels_per_iteration"] == cfr.cfr_get_info(t)["kernels_per_iteration"] - 2
    s.close()
    t.close()


def test_pair_eligibility(rank13):
    g = rank13
    info = lambda **kw: cfr.cfr_get_info(cfr.cfr_load_tree(g, **kw))   # noqa: E731
    assert info(precision=cfr.CFR_FP32, head_levels=3)["pair_depth"] == 6
    assert info(precision=cfr.CFR_FP32, head_levels=5)["pair_depth"] == 6          # head: depths 0-5
    assert info(precision=cfr.CFR_FP32, head_levels=6)["pair_depth"] == -1         # the head holds depth 6
    assert info(precision=cfr.CFR_FP32, head_levels=3, fuse_levels=2)["pair_depth"] == -1
    assert info(precision=cfr.CFR_FP32, head_levels=3, fuse_levels=0)["pair_depth"] == -1
    assert info(precision=cfr.CFR_FP64)["pair_depth"] == -1
    # too few decision nodes at the upper depth (3432 at depth 6 of this cut)
    small = gamegen.config("rank13_depth10", seed=2, target_nodes=200_000)
    assert cfr.cfr_get_info(cfr.cfr_load_tree(small, precision=cfr.CFR_FP32, head_levels=0))["pair_depth"] == -1


def _depths(g):
    d = np.full(g.num_nodes, -1, np.int64)
    d[g.parent < 0] = 0
    todo = d < 0
    while todo.any():
        idx = np.nonzero(todo)[0]
        known = d[g.parent[idx]] >= 0
        d[idx[known]] = d[g.parent[idx[known]]] + 1
        todo = d < 0
    return d
