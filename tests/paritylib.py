"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances: FP64 mode 1e-12, FP32 mode 1e-5 (normwise relative, per array:
max_i |x_i - y_i| / max_i |y_i|), exploitability 1e-6 absolute.
"""
import numpy as np

import paper_2408_14778_gb300 as cfr

TOL64, TOL32, TOL_EXPL = 1e-12, 1e-5, 1e-6


def normwise(x, y):
    x, y = np.asarray(x, float), np.asarray(y, float)
    if y.size == 0:
        return 0.0
    return float(np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-30))


def qbase(g):
    return np.concatenate([[0], np.cumsum(g.infoset_num_actions)]).astype(np.int64)


def player_mask(g):
    qb = qbase(g)
    m = np.zeros(qb[-1], bool)
    for h in range(g.num_infosets):
        if g.infoset_player[h] != 0:
            m[qb[h]:qb[h + 1]] = True
    return m


def regret_matching(g, R):
    """Eq. 9 applied to R (chance slots get sigma_0); checks the validity of FP32 strategies."""
    qb = qbase(g)
    out = np.zeros(qb[-1])
    c = 0
    for h in range(g.num_infosets):
        sl = slice(qb[h], qb[h + 1])
        n = qb[h + 1] - qb[h]
        if g.infoset_player[h] == 0:
            out[sl] = g.chance_prob[c:c + n]
            c += n
            continue
        pos = np.maximum(R[sl], 0)
        out[sl] = pos / pos.sum() if pos.sum() > 0 else 1.0 / n
    return out


def fp32_sigma_check(g, gs, os_, sig_g, tol=TOL32, players=(1, 2)):
    """Strategy parity in FP32 mode.

    The regrets themselves are compared elsewhere (normwise 1e-5).  Given the regrets' observed
    discrepancy delta_h = max_a |R_gpu(h,a) - R_oracle(h,a)|, regret matching (Eq. 9) pins sigma(h, .)
    to within tol wherever the oracle's positive regrets sum to more than 2 |A(h)| delta_h / tol (or all
    lie below -delta_h); there sigma is compared with the oracle's.  Elsewhere the FP32 rounding of
    near-zero regret sums decides the strategy - several results are correct - and it is checked to
    be the regret matching of the GPU's own regrets, as it is everywhere.  Returns the share of player
    infosets whose strategy rounding moved by more than tol.
    """
    qb = qbase(g)
    na = np.diff(qb)
    starts = qb[:-1]
    R = os_["cum_regret"]
    Rg = gs["cum_regret"]
    seg = lambda x, op: op.reduceat(x, starts) if x.size else x     # noqa: E731 - per-infoset reduction
    player = np.isin(g.infoset_player, players)
    delta = seg(np.abs(Rg - R), np.maximum)
    pos = seg(np.maximum(R, 0), np.add)
    rmax = seg(R, np.maximum)
    fixed = player & ((pos > 2 * na * delta / tol) | ((pos == 0) & (rmax < -delta)))
    err = seg(np.abs(sig_g - os_["sigma"]), np.maximum)
    bad = np.nonzero(fixed & (err > tol))[0]
    assert bad.size == 0, f"infoset {bad[0]}: sigma error {err[bad[0]]:.3e} (positive regret sum {pos[bad[0]]:.3e})"
    # the rest: the GPU's strategy is the regret matching (Eq. 9) of the GPU's own regrets
    posg = seg(np.maximum(Rg, 0), np.add)
    posg_q = np.repeat(posg, na)
    rm = np.where(posg_q > 0, np.maximum(Rg, 0) / np.where(posg_q > 0, posg_q, 1), 1.0 / np.repeat(na, na))
    dev = seg(np.abs(sig_g - rm), np.maximum)
    badr = np.nonzero(player & (dev > 1e-6))[0]
    assert badr.size == 0, f"infoset {badr[0]}: strategy is not the regret matching of the GPU's regrets"
    differ = player & ~fixed & (err > tol)            # strategies that rounding actually moved
    return float(differ.sum()) / max(int(player.sum()), 1)


def fp32_regret_budget_check(g, gs, os_, depth, scale=1.0, players=(1, 2)):
    """Per-infoset bound on one FP32 step's regret error.

    r~(h,a) = sum_{d in h} pi-check(d) (u(child_a(d)) - u(d)) (Eq. 7).  In FP32, pi-check carries at most
    2D rounding errors (D = depth; one per product and per stored sigma), a node value at most
    (2D + 1) eps U (U = max |utility|), the difference two of those plus one, and the sum over the n_h
    nodes of h at most n_h eps * sum |terms|.  Hence
        |r~_gpu - r~| <= (8 D + 8 + 2 n_h) eps32 U pi~(h)      (pi~(h) of Eq. 3),
    and the same bounds the regret after one step from exact state (CFR+ clipping is 1-Lipschitz), plus
    the rounding of the FP64 addition R + r~ on either side (half an FP64 ulp of R each), which exceeds
    the FP32 budget where an infoset's reach is tiny.  scale multiplies the bound where the step weights
    r~ (linear CFR: by T).
    """
    eps = 2.0 ** -24
    U = float(np.abs(g.utility).max())
    qb = qbase(g)
    nh = np.bincount(g.infoset[g.infoset >= 0], minlength=g.num_infosets)
    budget = scale * (8 * depth + 8 + 2 * nh) * eps * U * os_["cf_reach_sum"]
    Rg, Ro = gs["cum_regret"], os_["cum_regret"]
    # per slot: the error above the two FP64 roundings of R, then the largest per infoset
    excess = np.maximum(np.abs(Rg - Ro) - 2.0 ** -53 * (np.abs(Rg) + np.abs(Ro)), 0.0)
    dev = np.maximum.reduceat(excess, qb[:-1]) if qb[-1] else np.zeros(0)
    bad = np.nonzero(np.isin(g.infoset_player, players) & (dev > budget * (1 + 1e-9) + 1e-300))[0]
    assert bad.size == 0, (f"infoset {bad[0]}: regret error {dev[bad[0]]:.3e} above the FP32 budget "
                           f"{budget[bad[0]]:.3e}")


def compare_state(s, o, tol, g, what=("cum_regret", "strat_sum", "inst_regret"), max_rounding_share=1.0,
                  budget_scale=1.0, players=(1, 2)):
    """Regrets, sums and the strategy of the solver against the oracle.

    FP64: every array normwise within tol.  FP32 (one step from the oracle's state): arrays
    normwise within tol, each infoset's regrets within the FP32 budget of fp32_regret_budget_check,
    and strategies as in fp32_sigma_check.
    """
    gs, os_ = cfr.cfr_get_state(s), o.state()
    keep = np.repeat(np.isin(g.infoset_player, players), g.infoset_num_actions)   # the slots compared
    for k in what:
        e = normwise(np.where(keep, gs[k], 0.0), np.where(keep, os_[k], 0.0))
        assert e <= tol, f"{k}: normwise error {e:.3e} > {tol:.0e}"
    sig = cfr.cfr_current_strategy(s)
    if tol >= TOL32:
        fp32_regret_budget_check(g, gs, os_, cfr.cfr_get_info(s)["max_depth"], budget_scale, players)
        share = fp32_sigma_check(g, gs, os_, sig, tol, players)
        assert share <= max_rounding_share, f"rounding moved the strategy of {share:.2%} of infosets"
    else:
        e = normwise(np.where(keep, sig, 0.0), np.where(keep, os_["sigma"], 0.0))
        assert e <= tol, f"sigma: normwise error {e:.3e}"
    assert gs["iteration"] == os_["iteration"]
    return gs, os_


def compare_nodes(s, o, tol, g):
    """Node values (Eq. 1) and counterfactual reaches (Eq. 2) of the last iteration."""
    gn, on = cfr.cfr_get_nodes(s), o.nodes()
    dec = g.infoset >= 0
    assert normwise(gn["u1"], on["u1"]) <= tol
    assert normwise(gn["cf_reach1"][dec], on["cf1"][dec]) <= tol
    assert normwise(gn["cf_reach2"][dec], on["cf2"][dec]) <= tol
    assert np.all(np.isnan(gn["cf_reach1"][~dec]))
    return gn, on


def compare_step(s, o, g, alt, nodes=True):
    """One FP32 step (simultaneous or alternating updates) against the oracle's step from the same state;
    nodes: also the node values and reaches (the solver records them)."""
    if not alt:
        compare_state(s, o, TOL32, g)
        if nodes:
            compare_nodes(s, o, TOL32, g)
        return
    # Alternating: player 1's half of the step is checked like a simultaneous step.  Player 2's pass runs
    # under player 1's new FP32 strategy: where regret matching is ill-conditioned (a regret sum of exactly
    # 0 in FP64 against a rounding residue in FP32) the two sides legitimately decide player 1's strategy
    # differently, and player 2's regrets follow (whatever the kernels).  Player 2 is compared (normwise)
    # when the two new player-1 strategies agree to FP32 rounding.
    compare_state(s, o, TOL32, g, players=(1,))
    gs, os_ = cfr.cfr_get_state(s), o.state()
    p1 = np.repeat(g.infoset_player == 1, g.infoset_num_actions)
    p2 = np.repeat(g.infoset_player == 2, g.infoset_num_actions)
    if np.abs(cfr.cfr_current_strategy(s)[p1] - os_["sigma"][p1]).max() <= 4 * 2.0 ** -24:
        for k in ("cum_regret", "strat_sum", "inst_regret"):
            assert normwise(gs[k][p2], os_[k][p2]) <= TOL32, k
