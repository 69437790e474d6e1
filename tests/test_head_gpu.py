"""The shallowest depths in one cluster launch (k_head_topdown / k_head_bottomup, FP32 mode) against the
oracle: a first iteration and a step from the oracle's state at T = 3 (FP32 step parity; two FP32 runs'
trajectories part after a few iterations whatever their kernels, since the atomics' order differs and
regret matching amplifies it) (GPU tests)."""
import pytest

import gamegen
import oracle
import paper_2408_14778_gb300 as cfr
from paritylib import TOL32, compare_nodes, compare_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fuse", [0, -1])
@pytest.mark.parametrize("name,nodes", [("rank13_depth10", 200_000), ("holdem169_depth12", 2_000_000)])
def test_head_matches_oracle(name, nodes, fuse):
    g = gamegen.config(name, seed=2, target_nodes=nodes)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32, fuse_levels=fuse, record_nodes=True,
                          head_levels=-1)
    assert cfr.cfr_get_info(s)["head_depths"] >= 2
    o = oracle.Oracle(g, record=True)
    o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
    cfr.cfr_iterate(s, 1)
    compare_state(s, o, TOL32, g)
    compare_nodes(s, o, TOL32, g)
    o.iterate(2, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
    st = o.state()
    cfr.cfr_set_state(s, st["cum_regret"], st["strat_sum"], st["iteration"])
    o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
    cfr.cfr_iterate(s, 1)
    compare_state(s, o, TOL32, g)
    compare_nodes(s, o, TOL32, g)


def test_head_is_an_option():
    g = gamegen.config("rank13_depth10", seed=2, target_nodes=200_000)
    assert cfr.cfr_get_info(cfr.cfr_load_tree(g, precision=cfr.CFR_FP32))["head_depths"] == 0   # default off
    assert cfr.cfr_get_info(cfr.cfr_load_tree(g, precision=cfr.CFR_FP32, head_levels=-1))["head_depths"] >= 2
    assert cfr.cfr_get_info(cfr.cfr_load_tree(g, precision=cfr.CFR_FP32, head_levels=3))["head_depths"] == 3
    assert cfr.cfr_get_info(cfr.cfr_load_tree(g, precision=cfr.CFR_FP64, head_levels=-1))["head_depths"] == 0
