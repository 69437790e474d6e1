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

pytestmark = pytest.mark.gpu


def normwise(x, y):
    return float(np.max(np.abs(np.asarray(x) - np.asarray(y))) / max(np.max(np.abs(y)), 1e-30))


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


def _compare(s, o):
    gs, os_ = cfr.cfr_get_state(s), o.state()
    for k in ("inst_regret", "cum_regret", "strat_sum"):
        e = normwise(gs[k], os_[k])
        assert e <= 1e-5, (k, e)
    e = normwise(cfr.cfr_current_strategy(s), os_["sigma"])
    assert e <= 1e-5, ("sigma", e)


def test_full_size_first_iteration(full):
    g, o, s = full
    info = cfr.cfr_get_info(s)
    assert info["num_nodes"] == g.num_nodes > 9e7
    o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
    cfr.cfr_iterate(s, 1)
    _compare(s, o)
    rv = cfr.cfr_root_value(s)
    assert np.isfinite(rv)


def test_full_size_step_from_oracle_state(full):
    g, o, s = full
    o.iterate(2, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)     # oracle at T = 3
    st = o.state()
    cfr.cfr_set_state(s, st["cum_regret"], st["strat_sum"], st["iteration"])
    o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
    cfr.cfr_iterate(s, 1)
    _compare(s, o)


def test_full_size_exploitability(full):
    g, o, s = full
    nc_g, ex_g = cfr.cfr_exploitability(s)
    nc_o, ex_o = o.exploitability()
    assert abs(nc_g - nc_o) <= 1e-6 * max(1.0, 0.0) + 1e-6, (nc_g, nc_o)
    assert abs(ex_g - ex_o) <= 1e-6
