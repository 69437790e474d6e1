"""Alternating updates, linear CFR and discounted CFR on the GPU against the oracle (GPU tests).

The oracle implements each as a direct restatement: alternating updates run player 1's pass and
update, then player 2's under player 1's new strategy; linear CFR weights iteration T's regret and
average contribution by T; discounted CFR(alpha, beta, gamma) scales the accumulated regret by
T^alpha/(T^alpha+1) where positive and T^beta/(T^beta+1) elsewhere and weights the average by T^gamma.
FP64 mode follows the oracle's operations (discounted CFR's powers come from the device's pow, so its
results agree to rounding, not bit for bit); FP32 mode is compared one step from the oracle's state.
"""
import numpy as np
import pytest

import gamegen
import oracle
import paper_2408_14778_gb300 as cfr
from paritylib import TOL32, TOL64, TOL_EXPL, compare_state

pytestmark = pytest.mark.gpu

DCFR = (1.5, 0.0, 2.0)
VARIANTS = [cfr.CFR_VANILLA, cfr.CFR_PLUS, cfr.CFR_LINEAR, cfr.CFR_DISCOUNTED]


def _avg(variant):
    return oracle.AVG_UNIFORM if variant == cfr.CFR_VANILLA else oracle.AVG_LINEAR


def _games():
    return [gamegen.config("bucket3_depth6", seed=3),
            gamegen.config("rank13_depth10", seed=4, target_nodes=60_000)]


@pytest.mark.parametrize("alt", [False, True])
@pytest.mark.parametrize("variant", VARIANTS)
def test_fp64_trajectory_matches_oracle(variant, alt):
    mode = cfr.CFR_ALTERNATING if alt else cfr.CFR_SIMULTANEOUS
    for g in _games():
        o = oracle.Oracle(g)
        s = cfr.cfr_load_tree(g, variant=variant, precision=cfr.CFR_FP64, update_mode=mode, dcfr=DCFR)
        for _ in range(3):
            o.iterate(10, variant=variant, avg=_avg(variant), alternating=alt, dcfr=DCFR)
            cfr.cfr_iterate(s, 10)
            compare_state(s, o, TOL64, g)
        assert abs(cfr.cfr_exploitability(s)[0] - o.exploitability()[0]) <= TOL_EXPL


@pytest.mark.parametrize("alt", [False, True])
@pytest.mark.parametrize("variant", [cfr.CFR_PLUS, cfr.CFR_LINEAR, cfr.CFR_DISCOUNTED])
def test_fp32_step_parity(variant, alt):
    # one FP32 iteration from the oracle's FP64 state at T = 1, 3, 20 (fused and streamed kernels included)
    g = gamegen.config("rank13_depth10", seed=5, target_nodes=400_000)
    mode = cfr.CFR_ALTERNATING if alt else cfr.CFR_SIMULTANEOUS
    o = oracle.Oracle(g)
    s = cfr.cfr_load_tree(g, variant=variant, precision=cfr.CFR_FP32, update_mode=mode, dcfr=DCFR)
    done, full = 0, 0
    for T in (1, 3, 20):
        o.iterate(T - 1 - done, variant=variant, avg=_avg(variant), alternating=alt, dcfr=DCFR)
        st = o.state()
        cfr.cfr_set_state(s, st["cum_regret"], st["strat_sum"], st["iteration"])
        o.iterate(1, variant=variant, avg=_avg(variant), alternating=alt, dcfr=DCFR)
        done = T
        cfr.cfr_iterate(s, 1)
        scale = T if variant == cfr.CFR_LINEAR else 1.0     # linear CFR weights this step's regret by T
        if not alt:
            compare_state(s, o, TOL32, g, budget_scale=scale)
            full += 1
            continue
        # Alternating: player 1's half of the step is checked like a simultaneous step.  Player 2's pass
        # runs under player 1's new strategy, which FP32 rounding may legitimately decide otherwise
        # where regret matching is ill-conditioned (a regret sum of exactly 0 against 1 ulp); player 2 is
        # checked whenever the two new player-1 strategies agree.
        compare_state(s, o, TOL32, g, budget_scale=scale, players=(1,))
        p1 = np.repeat(g.infoset_player == 1, g.infoset_num_actions)
        if np.abs(cfr.cfr_current_strategy(s)[p1] - o.state()["sigma"][p1]).max() <= TOL32:
            compare_state(s, o, TOL32, g, budget_scale=2 * scale, players=(2,))
            full += 1
    assert full >= 1


def test_fp32_alternating_converges_like_the_oracle():
    g = gamegen.config("rank13_depth10", seed=6, target_nodes=200_000)
    o = oracle.Oracle(g)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32, update_mode=cfr.CFR_ALTERNATING)
    o.iterate(200, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR, alternating=True)
    cfr.cfr_iterate(s, 200)
    nc_g, _ = cfr.cfr_exploitability(s)
    nc_o, _ = o.exploitability()
    assert nc_g <= 1.1 * nc_o + 1e-4
    nc_chk, _ = o.exploitability(cfr.cfr_average_strategy(s))
    assert abs(nc_chk - nc_g) <= TOL_EXPL


def test_phase_times_need_simultaneous_updates():
    g = gamegen.config("bucket3_depth6", seed=1)
    s = cfr.cfr_load_tree(g, update_mode=cfr.CFR_ALTERNATING)
    with pytest.raises(cfr.CfrError) as e:
        cfr.cfr_phase_times(s)
    assert e.value.status == cfr.CFR_ERR_UNSUPPORTED
    cfr.cfr_iterate(s, 2)
    assert cfr.cfr_get_info(s)["iteration"] == 2
