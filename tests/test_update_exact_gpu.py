"""The FP32-mode update (Eq. 8, Eq. 9, Eq. 10 with Eq. 14-15's clipping for CFR+) is exact IEEE
arithmetic on the solver's own state, bit for bit.

After one iteration, every player slot of an infoset with at most 32 actions must satisfy, from the
state before it (R0, S0, sigma0), the iteration's instantaneous regrets r~ and own reaches pi_i:
  R1 = R0 + double(r~)                       (CFR+: R1 = that if it is > 0, else 0)
  S1 = S0 + double(float(float(w pi_i) sigma0))   where that increment is not 0 (w = T, linear averaging;
                                                  1, uniform), else S1 = S0
  sigma1 = float(R1+) * (1 / sum) in FP32, the sum of the row's float(R1+) taken in action order
           (uniform 1/|A| when the sum is 0).
The kernel forms float(R1+) and the FP64 addition S0 + increment with integer operations (round to
nearest even on the dropped fraction bits; align, add, round on guard and sticky bits), so this test
pins those against numpy's IEEE conversions and additions exactly, independently of the oracle.
"""
import numpy as np
import pytest

import gamegen
import paper_2408_14778_gb300 as cfr
from paritylib import qbase

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    cfr.build()


def _expected(g, st0, sig0, st1, variant, linear):
    qb = qbase(g)
    na = np.diff(qb)
    rows = np.nonzero((g.infoset_player != 0) & (na <= 32))[0]
    h_of = np.repeat(np.arange(g.num_infosets), na)
    keep = np.isin(h_of, rows)

    r0 = st0["cum_regret"] + st1["inst_regret"].astype(np.float32).astype(np.float64)
    R1 = np.where(r0 > 0, r0, 0.0) if variant == cfr.CFR_PLUS else r0

    T = st1["iteration"]
    w = np.float32(T) if linear else np.float32(1.0)
    own = st1["own_reach"].astype(np.float32)
    wo = (w * own).astype(np.float32)
    inc = (wo[h_of] * sig0.astype(np.float32)).astype(np.float32)
    S1 = np.where(inc != 0, st0["strat_sum"] + inc.astype(np.float64), st0["strat_sum"])

    pos = np.where(R1 > 0, R1.astype(np.float32), np.float32(0))
    total = np.zeros(g.num_infosets, np.float32)
    for a in range(int(na.max())):                  # the row's sum in action order, in FP32
        has = na > a
        total[has] = (total[has] + pos[qb[:-1][has] + a]).astype(np.float32)
    tot = total[h_of]
    with np.errstate(divide="ignore", invalid="ignore"):          # rows with no positive regret: masked below
        f = (np.float32(1) / tot).astype(np.float32)
        sig1 = np.where(tot > 0, (pos * f).astype(np.float32), (np.float32(1) / na[h_of].astype(np.float32)))
    # rows whose positive regrets sum below FP32's normal range are normalised in FP64: left out here
    keep_sig = keep & ~((tot > 0) & (tot < np.float32(1e-30)))
    return keep, keep_sig, R1, S1, sig1


@pytest.mark.parametrize("variant", [cfr.CFR_PLUS, cfr.CFR_VANILLA])
def test_update_is_exact_ieee_arithmetic(variant):
    # 13-rank fold/showdown game, 2.03e6 nodes, 4.8e4 infosets, 1.69e5 player slots; a few iterations in
    g = gamegen.config("rank13_depth10", seed=0)
    linear = variant == cfr.CFR_PLUS
    s = cfr.cfr_load_tree(g, variant=variant, precision=cfr.CFR_FP32,
                          avg_weight=cfr.CFR_AVG_LINEAR if linear else cfr.CFR_AVG_UNIFORM)
    cfr.cfr_iterate(s, 4)
    for _ in range(3):
        st0, sig0 = cfr.cfr_get_state(s), cfr.cfr_current_strategy(s)
        cfr.cfr_iterate(s, 1)
        st1, sig1 = cfr.cfr_get_state(s), cfr.cfr_current_strategy(s)
        keep, keep_sig, R1, S1, sig_exp = _expected(g, st0, sig0, st1, variant, linear)
        assert keep.sum() > 160_000
        np.testing.assert_array_equal(st1["cum_regret"][keep], R1[keep])
        np.testing.assert_array_equal(st1["strat_sum"][keep], S1[keep])
        np.testing.assert_array_equal(sig1[keep_sig].astype(np.float32), sig_exp[keep_sig])
    s.close()
