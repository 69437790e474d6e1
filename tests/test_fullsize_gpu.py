"""Full-size parity: the benchmark's workload and launch configuration (holdem169_depth12, ~1e8
nodes, CFR+, FP32 with FP64 sums) against the oracle, which finishes one iteration of it in seconds.

Every regret, strategy sum and strategy entry is compared (normwise 1e-5), after the first
iteration and after a step from the oracle's state at T = 3; then the exploitability of the
average strategy (1e-6 absolute).
"""
import numpy as np
import pytest

import gamegen
import oracle
import paper_2408_14778_gb300 as cfr
from paritylib import TOL32, TOL_EXPL, compare_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    cfr.build()
    g = gamegen.config("holdem169_depth12", seed=0)
    o = oracle.Oracle(g)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32)
    yield g, o, s
    s.close()


def _compare(s, o, g):
    compare_state(s, o, TOL32, g)


def test_full_size_first_iteration(full):
    g, o, s = full
    info = cfr.cfr_get_info(s)
    assert info["num_nodes"] == g.num_nodes > 9e7
    assert info["tail_kernel"] == 2                       # the last two depths streamed, per-slot atomics
    o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR, threads=0)
    cfr.cfr_iterate(s, 1)
    _compare(s, o, g)
    rv = cfr.cfr_root_value(s)
    assert np.isfinite(rv)


def test_full_size_step_from_oracle_state(full):
    g, o, s = full
    o.iterate(2, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR, threads=0)     # oracle at T = 3
    st = o.state()
    cfr.cfr_set_state(s, st["cum_regret"], st["strat_sum"], st["iteration"])
    o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR, threads=0)
    cfr.cfr_iterate(s, 1)
    _compare(s, o, g)


def test_full_size_exploitability(full):
    g, o, s = full
    nc_g, ex_g = cfr.cfr_exploitability(s)
    nc_o, ex_o = o.exploitability()
    # FP32 strategy sums differ from the FP64 oracle's by ~1e-7 relative, which moves NashConv by
    # ~1e-7 of its scale; the FP64 best response on the GPU's own average strategy must agree
    # with the oracle's to 1e-6.
    assert abs(nc_g - nc_o) <= 1e-5 * max(1.0, abs(nc_o)), (nc_g, nc_o)
    nc_chk, ex_chk = o.exploitability(cfr.cfr_average_strategy(s))
    assert abs(nc_g - nc_chk) <= TOL_EXPL and abs(ex_g - ex_chk) <= TOL_EXPL


def test_fp64_bit_identical_above_the_parallel_layout_threshold():
    # 2.0e6 nodes: the multi-threaded host layout builder (2^20 nodes and more) feeds FP64 mode, whose
    # deterministic regret sums walk the per-infoset node lists; three iterations equal the oracle's bit for bit
    g = gamegen.config("rank13_depth10", seed=5)
    assert g.num_nodes >= 1 << 20
    o = oracle.Oracle(g)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP64)
    o.iterate(3, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
    cfr.cfr_iterate(s, 3)
    gs, os_ = cfr.cfr_get_state(s), o.state()
    for k in ("cum_regret", "strat_sum"):
        np.testing.assert_array_equal(gs[k], os_[k])
    s.close()


def test_full_size_both_tail_kernels_from_oracle_state(full):
    # the last two depths by slot-dense tiles (staged strategy entries; regrets by atomics or by bulk
    # reductions) as well as by the default per-slot kernel: each one FP32 step from the oracle's state
    # against the oracle's next iteration (the module's solver is not used after this test)
    g, o, s = full
    st = o.state()
    others = [cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32, tail_slots=v) for v in (1, 2)]
    assert [cfr.cfr_get_info(x)["tail_kernel"] for x in others] == [3, 4]
    for x in [s] + others:
        cfr.cfr_set_state(x, st["cum_regret"], st["strat_sum"], st["iteration"])
        cfr.cfr_iterate(x, 1)
    o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR, threads=0)
    for x in [s] + others:
        _compare(x, o, g)
        x.close()
