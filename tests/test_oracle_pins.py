"""Pins of the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each test checks the oracle against something other than itself: hand-worked values, closed-form
equilibria, brute-force enumeration of the definitions (``defs.py``, path products rather than
recursion), a sequence-form LP, exact identities and published bounds.
"""
import json
import os

import numpy as np
import pytest

import gamegen
import oracle
from defs import Tree, random_profile, uniform_profile

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def hand_game():
    d = json.load(open(os.path.join(GOLDEN, "hand_two_steps.json")))
    g = d["game"]
    n = len(g["parent"])
    util = np.zeros((n, 2))
    util[:, 0] = g["u1"]
    util[:, 1] = -util[:, 0]
    game = gamegen.GameDesc(np.array(g["parent"], np.int32), np.array(g["action"], np.int32),
                            np.array(g["infoset"], np.int32), np.array(g["infoset_player"], np.int8),
                            np.array(g["infoset_num_actions"], np.int32), np.array(g["chance_prob"]), util)
    return game, d


def tiny_games(count=6, seed0=100, **kw):
    """Small public-private games with public chance nodes, general shapes."""
    out = []
    s = seed0
    while len(out) < count:
        prm = dict(deal_kind=gamegen.DEAL_BUCKET_PAIRS, num_buckets=2 + s % 2, depth=3 + s % 3, amin=2, amax=3,
                   p_cont=0.6, p_chance=0.3, payoff_kind=gamegen.PAY_UNIFORM, umax=3.0, first_actor=1 + s % 2)
        prm.update(kw)
        g = gamegen.public_private(seed=s, **prm)
        s += 1
        tr = Tree(g)
        n1 = np.prod([tr.nact[h] for h in range(tr.H) if tr.player[h] == 1] or [1])
        n2 = np.prod([tr.nact[h] for h in range(tr.H) if tr.player[h] == 2] or [1])
        if g.num_nodes <= 400 and n1 <= 4096 and n2 <= 4096:
            out.append((g, tr))
    return out


def multilevel_game():
    """Perfect-recall game whose player-1 infoset spans two depths (built by hand).

    Chance (p = 0.4 / 0.6): outcome 0 -> P1 node directly (depth 1); outcome 1 -> P2 node (depth 1)
    whose two actions lead to P1 nodes (depth 2).  P1 observes nothing, so all three P1 nodes
    share infoset 2; P1 has no earlier own action, so recall is perfect.
    """
    parent = [-1, 0, 0, 1, 1, 2, 2, 5, 5, 6, 6]
    action = [-1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1]
    infoset = [0, 2, 1, -1, -1, 2, 2, -1, -1, -1, -1]
    u1 = [0, 0, 0, 1.0, -2.0, 0, 0, 3.0, -1.0, -2.5, 2.0]
    util = np.zeros((11, 2))
    util[:, 0] = u1
    util[:, 1] = -util[:, 0]
    return gamegen.GameDesc(np.array(parent, np.int32), np.array(action, np.int32), np.array(infoset, np.int32),
                            np.array([0, 2, 1], np.int8), np.array([2, 2, 2], np.int32), np.array([0.4, 0.6]), util)


# ------------------------------------------------------------------------------------------------
# 1. hand-worked values
# ------------------------------------------------------------------------------------------------

def test_hand_worked_two_iterations_vanilla():
    game, d = hand_game()
    o = oracle.Oracle(game, record=True)
    for T in ("T1", "T2"):
        exp = d["vanilla"][T]
        o.iterate(1)
        st = o.state()
        nodes = o.nodes()
        np.testing.assert_allclose(st["inst_regret"], exp["inst_regret"], atol=1e-15)
        np.testing.assert_allclose(st["cum_regret"], exp["cum_regret"], atol=1e-15)
        np.testing.assert_allclose(st["sigma"], exp["sigma_next"], atol=1e-15)
        np.testing.assert_allclose(st["strat_sum"], exp["strat_sum"], atol=1e-15)
        for v, val in exp["u1_nodes"].items():
            assert nodes["u1"][int(v)] == pytest.approx(val, abs=1e-15)
            assert nodes["u2"][int(v)] == pytest.approx(-val, abs=1e-15)
        if "reach_cf1_cf2_own1_own2" in exp:
            for v, r in exp["reach_cf1_cf2_own1_own2"].items():
                got = [nodes[k][int(v)] for k in ("cf1", "cf2", "own1", "own2")]
                np.testing.assert_allclose(got, r, atol=1e-15)
        if "cf_reach_sum" in exp:
            np.testing.assert_allclose(st["cf_reach_sum"], exp["cf_reach_sum"], atol=1e-15)
        if "own_reach" in exp:
            np.testing.assert_allclose(st["own_reach"], exp["own_reach"], atol=1e-15)
        if "average_strategy" in exp:
            np.testing.assert_allclose(o.average_strategy(), exp["average_strategy"], atol=1e-15)


def test_hand_worked_two_iterations_cfr_plus():
    game, d = hand_game()
    o = oracle.Oracle(game)
    for T in ("T1", "T2"):
        exp = d["cfr_plus_linear"][T]
        o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
        st = o.state()
        np.testing.assert_allclose(st["cum_regret"], exp["cum_regret"], atol=1e-15)
        np.testing.assert_allclose(st["sigma"], exp["sigma_next"], atol=1e-15)
        np.testing.assert_allclose(st["strat_sum"], exp["strat_sum"], atol=1e-15)
        if "inst_regret" in exp:
            np.testing.assert_allclose(st["inst_regret"], exp["inst_regret"], atol=1e-15)


# ------------------------------------------------------------------------------------------------
# 2. matrix games with closed-form solutions
# ------------------------------------------------------------------------------------------------

def test_rock_paper_scissors_is_a_fixed_point():
    g = gamegen.matrix_game([[0, -1, 1], [1, 0, -1], [-1, 1, 0]])
    o = oracle.Oracle(g)
    rv = o.iterate(1)
    st = o.state()
    assert np.all(st["inst_regret"] == 0.0)              # every action earns 0 against uniform
    assert rv[0] == 0.0 and rv[1] == 0.0
    o.iterate(99)
    np.testing.assert_array_equal(o.current_strategy(), np.full(6, 1.0 / 3.0))
    np.testing.assert_array_equal(o.average_strategy(), np.full(6, 1.0 / 3.0))
    nc, ex = o.exploitability()
    assert nc == pytest.approx(0.0, abs=1e-15) and ex == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("a,b,c", [(1.0, 2.0, 3.0), (2.0, 0.5, 1.0)])
@pytest.mark.parametrize("variant,avg,alt,iters,tol", [(0, 0, False, 20000, 2e-2), (1, 1, False, 5000, 1e-2),
                                                     (1, 1, True, 5000, 1e-3), (2, 0, False, 5000, 2e-2),
                                                     (2, 0, True, 5000, 1e-2), (3, 0, False, 5000, 1e-2),
                                                     (3, 0, True, 5000, 1e-2)])
def test_weighted_rps_closed_form(a, b, c, variant, avg, alt, iters, tol):
    # Skew-symmetric payoff [[0,-a,b],[a,0,-c],[-b,c,0]]: the unique equilibrium is (c, b, a) / (a+b+c)
    # for both players, value 0 (each column of x^T A vanishes).
    A = np.array([[0, -a, b], [a, 0, -c], [-b, c, 0]])
    x = np.array([c, b, a]) / (a + b + c)
    o = oracle.Oracle(gamegen.matrix_game(A))
    o.iterate(iters, variant=variant, avg=avg, alternating=alt)
    avgs = o.average_strategy()
    np.testing.assert_allclose(avgs[:3], x, atol=tol)
    np.testing.assert_allclose(avgs[3:], x, atol=tol)
    assert o.expected_value(1, avgs) == pytest.approx(0.0, abs=tol)
    nc, _ = o.exploitability()
    assert nc < 5 * tol


@pytest.mark.parametrize("A", [[[3.0, -1.0], [-2.0, 1.0]], [[0.0, 4.0], [2.0, 1.0]], [[-1.5, 2.0], [1.0, -0.5]]])
def test_two_by_two_closed_form(A):
    (a, b), (c, d) = A
    den = a - b - c + d
    p, q, value = (d - c) / den, (d - b) / den, (a * d - b * c) / den   # textbook mixed equilibrium
    assert 0 < p < 1 and 0 < q < 1
    o = oracle.Oracle(gamegen.matrix_game(A))
    o.iterate(4000, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR, alternating=True)
    s = o.average_strategy()
    assert s[0] == pytest.approx(p, abs=5e-3) and s[2] == pytest.approx(q, abs=5e-3)
    assert o.expected_value(1, s) == pytest.approx(value, abs=5e-3)
    # exact equilibrium has zero exploitability
    eq = np.array([p, 1 - p, q, 1 - q])
    nc, _ = o.exploitability(eq)
    assert nc == pytest.approx(0.0, abs=1e-12)
    assert o.expected_value(1, eq) == pytest.approx(value, abs=1e-12)


# ------------------------------------------------------------------------------------------------
# 3. definitions by path enumeration (Eq. 1-10)
# ------------------------------------------------------------------------------------------------

def _set_random_strategy(o, tr, rng):
    """Drive the oracle to a random strategy: R > 0 random, so sigma = R / sum R (Eq. 9)."""
    R = np.zeros(tr.Q)
    for h in range(tr.H):
        if tr.player[h] != 0:
            w = rng.random(tr.nact[h]) + 0.05
            w[rng.random(tr.nact[h]) < 0.2] = -1.0           # some negative regrets -> zero prob
            if (w > 0).sum() == 0:
                w[0] = 1.0
            R[tr.qbase[h]:tr.qbase[h] + tr.nact[h]] = w
    o.set_state(R, np.zeros(tr.Q), 0)
    prof = np.array(tr.sigma0)
    for h in range(tr.H):
        if tr.player[h] != 0:
            r = np.maximum(R[tr.qbase[h]:tr.qbase[h] + tr.nact[h]], 0)
            prof[tr.qbase[h]:tr.qbase[h] + tr.nact[h]] = r / r.sum()
    return prof


def test_instantaneous_regret_matches_definition():
    rng = np.random.default_rng(7)
    for g, tr in tiny_games(6):
        o = oracle.Oracle(g, record=True)
        prof = _set_random_strategy(o, tr, rng)
        np.testing.assert_allclose(o.current_strategy(), prof, atol=1e-15)
        o.iterate(1)
        want = tr.inst_regret(prof)
        np.testing.assert_allclose(o.state()["inst_regret"], want, atol=1e-12, rtol=0)


def test_node_values_and_reaches_match_path_products():
    rng = np.random.default_rng(8)
    for g, tr in tiny_games(6, seed0=200):
        o = oracle.Oracle(g, record=True)
        prof = _set_random_strategy(o, tr, rng)
        rv = o.iterate(1)
        nd = o.nodes()
        for v in range(tr.n):
            assert nd["u1"][v] == pytest.approx(tr.node_value(prof, v, 1), abs=1e-12)
            assert nd["u2"][v] == pytest.approx(tr.node_value(prof, v, 2), abs=1e-12)
            want = [tr.cf_reach(prof, v, 1), tr.cf_reach(prof, v, 2), tr.own_reach(prof, v, 1), tr.own_reach(prof, v, 2)]
            np.testing.assert_allclose([nd["cf1"][v], nd["cf2"][v], nd["own1"][v], nd["own2"][v]], want, atol=1e-14)
            rc, r1, r2 = tr.reach_split(prof, v)
            assert nd["cf1"][v] == pytest.approx(rc * r2, abs=1e-14) and nd["own1"][v] == pytest.approx(r1, abs=1e-14)
        # the root payoff is the expected payoff sum_t pi(t) u(t)  (Section 2.2 / Eq. 1 agree)
        assert rv[0] == pytest.approx(tr.expected_payoff(prof, 1), abs=1e-12)


def test_average_strategy_matches_eq10_with_node_sum_weights():
    for variant, avg in ((0, 0),):
        for g, tr in tiny_games(4, seed0=300):
            o = oracle.Oracle(g)
            history = []
            for _ in range(7):
                history.append(o.current_strategy().copy())
                o.iterate(1, variant=variant, avg=avg)
            np.testing.assert_allclose(o.average_strategy(), tr.average_strategy(history), atol=1e-12)


def test_cfr_plus_regret_and_linear_average_by_definition():
    for g, tr in tiny_games(4, seed0=400):
        o = oracle.Oracle(g)
        R = np.zeros(tr.Q)
        S = np.zeros(tr.Q)
        player_q = np.zeros(tr.Q, bool)
        for h in range(tr.H):
            if tr.player[h] != 0:
                player_q[tr.qbase[h]:tr.qbase[h] + tr.nact[h]] = True
        for T in range(1, 11):
            prof = o.current_strategy().copy()
            inst = tr.inst_regret(prof)
            R = np.where(player_q, np.maximum(R + inst, 0.0), 0.0)             # regret-matching+
            for h in range(tr.H):
                if tr.player[h] != 0:
                    own = tr.own_reach(prof, tr.nodes_of[h][0], tr.player[h]) if tr.nodes_of[h] else 0.0
                    sl = slice(tr.qbase[h], tr.qbase[h] + tr.nact[h])
                    S[sl] += T * own * prof[sl]                                   # linear averaging
            o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
            st = o.state()
            np.testing.assert_allclose(st["cum_regret"], R, atol=1e-12)
            np.testing.assert_allclose(st["strat_sum"], S, atol=1e-12)
            assert np.all(st["cum_regret"] >= 0.0)
            # the next strategy: regret matching (Eq. 9) of these regrets, uniform where none is positive, so
            # that every iterate of the trajectory (not only its sums) follows from the definitions
            nxt = o.current_strategy()
            for h in range(tr.H):
                sl = slice(tr.qbase[h], tr.qbase[h] + tr.nact[h])
                if tr.player[h] == 0:
                    np.testing.assert_array_equal(nxt[sl], prof[sl])                    # chance keeps sigma_0
                    continue
                pos = np.maximum(R[sl], 0.0)
                want = pos / pos.sum() if pos.sum() > 0 else np.full(tr.nact[h], 1.0 / tr.nact[h])
                np.testing.assert_allclose(nxt[sl], want, atol=1e-12)


def test_cfr_plus_first_iteration_equals_vanilla():
    for g, tr in tiny_games(3, seed0=500):
        a, b = oracle.Oracle(g), oracle.Oracle(g)
        a.iterate(1)
        b.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
        np.testing.assert_array_equal(a.current_strategy(), b.current_strategy())
        np.testing.assert_array_equal(a.state()["strat_sum"], b.state()["strat_sum"])


def test_linear_and_discounted_first_iteration_against_vanilla():
    # At T = 1 every weight is 1 (linear CFR, and 1^gamma for discounted CFR) and the discount is
    # 1^a / (1^a + 1) = 1/2 whatever the sign: linear CFR equals vanilla, discounted CFR halves its regrets.
    for g, tr in tiny_games(3, seed0=650):
        v, lin, dis = oracle.Oracle(g), oracle.Oracle(g), oracle.Oracle(g)
        v.iterate(1)
        lin.iterate(1, variant=oracle.LINEAR)
        dis.iterate(1, variant=oracle.DISCOUNTED, dcfr=(1.5, 0.0, 2.0))
        sv, sl, sd = v.state(), lin.state(), dis.state()
        np.testing.assert_array_equal(sl["cum_regret"], sv["cum_regret"])
        np.testing.assert_array_equal(sl["strat_sum"], sv["strat_sum"])
        np.testing.assert_array_equal(sd["cum_regret"], sv["cum_regret"] * 0.5)
        np.testing.assert_array_equal(sd["strat_sum"], sv["strat_sum"])
        np.testing.assert_array_equal(dis.current_strategy(), v.current_strategy())   # RM is scale-free


@pytest.mark.parametrize("variant", [2, 3])
def test_linear_and_discounted_cfr_by_definition(variant):
    # Regrets from path enumeration (Eq. 3, 6, 7), accumulated with the variant's weights.
    a_, b_, c_ = 1.5, 0.5, 2.0
    for g, tr in tiny_games(3, seed0=660 + variant):
        o = oracle.Oracle(g)
        R = np.zeros(tr.Q)
        S = np.zeros(tr.Q)
        player_q = np.zeros(tr.Q, bool)
        for h in range(tr.H):
            if tr.player[h] != 0:
                player_q[tr.qbase[h]:tr.qbase[h] + tr.nact[h]] = True
        for T in range(1, 7):
            prof = o.current_strategy().copy()
            inst = np.where(player_q, tr.inst_regret(prof), 0.0)
            if variant == 2:
                R = R + T * inst
                w = float(T)
            else:
                x = R + inst
                R = x * np.where(x > 0, T ** a_ / (T ** a_ + 1), T ** b_ / (T ** b_ + 1))
                w = float(T) ** c_
            for h in range(tr.H):
                if tr.player[h] != 0:
                    own = tr.own_reach(prof, tr.nodes_of[h][0], tr.player[h]) if tr.nodes_of[h] else 0.0
                    sl = slice(tr.qbase[h], tr.qbase[h] + tr.nact[h])
                    S[sl] += w * own * prof[sl]
            o.iterate(1, variant=variant, dcfr=(a_, b_, c_))
            st = o.state()
            np.testing.assert_allclose(st["cum_regret"], R, rtol=1e-12, atol=1e-12)
            np.testing.assert_allclose(st["strat_sum"], S, rtol=1e-12, atol=1e-12)


def test_alternating_updates_by_definition():
    for g, tr in tiny_games(3, seed0=600):
        o = oracle.Oracle(g)
        prof = o.current_strategy().copy()
        o.iterate(1, alternating=True)
        st = o.state()
        # player 1 regrets under sigma^T
        r1 = tr.inst_regret(prof)
        mid = prof.copy()
        for h in range(tr.H):
            if tr.player[h] == 1:
                sl = slice(tr.qbase[h], tr.qbase[h] + tr.nact[h])
                pos = np.maximum(r1[sl], 0)
                mid[sl] = pos / pos.sum() if pos.sum() > 0 else 1.0 / tr.nact[h]
        # player 2 regrets under (sigma_1^{T+1}, sigma_2^T)
        r2 = tr.inst_regret(mid)
        for h in range(tr.H):
            sl = slice(tr.qbase[h], tr.qbase[h] + tr.nact[h])
            if tr.player[h] == 1:
                np.testing.assert_allclose(st["cum_regret"][sl], r1[sl], atol=1e-12)
            elif tr.player[h] == 2:
                np.testing.assert_allclose(st["cum_regret"][sl], r2[sl], atol=1e-12)


def test_multilevel_infoset_game_matches_definition():
    g = multilevel_game()
    tr = Tree(g)
    o = oracle.Oracle(g)
    hist = []
    for _ in range(5):
        prof = o.current_strategy().copy()
        hist.append(prof)
        want = tr.inst_regret(prof)
        o.iterate(1)
        np.testing.assert_allclose(o.state()["inst_regret"], want, atol=1e-13)
    assert o.recall_violations() == 0
    np.testing.assert_allclose(o.average_strategy(), tr.average_strategy(hist), atol=1e-13)


# ------------------------------------------------------------------------------------------------
# 4. best response, LP value, regret identities and bounds
# ------------------------------------------------------------------------------------------------

def test_best_response_matches_pure_strategy_enumeration():
    rng = np.random.default_rng(11)
    for g, tr in tiny_games(6, seed0=700):
        o = oracle.Oracle(g)
        for _ in range(2):
            prof = random_profile(tr, rng, zero_frac=0.2)
            for i in (1, 2):
                assert o.best_response(i, prof) == pytest.approx(tr.best_response_value(prof, i), abs=1e-12)
                assert o.expected_value(i, prof) == pytest.approx(tr.expected_payoff(prof, i), abs=1e-12)


def test_sequence_form_lp_value_and_equilibrium():
    for g, tr in tiny_games(4, seed0=800):
        x, v1 = tr.lp_solve(1)
        y, v2 = tr.lp_solve(2)
        assert v1 == pytest.approx(v2, abs=1e-7)                      # minimax theorem
        eq = tr.behavioural(y, 2, tr.behavioural(x, 1, uniform_profile(tr)))
        o = oracle.Oracle(g)
        nc, _ = o.exploitability(eq)
        assert abs(nc) < 1e-7
        assert o.expected_value(1, eq) == pytest.approx(v1, abs=1e-7)
        o.iterate(3000)
        avg = o.average_strategy()
        nc, _ = o.exploitability(avg)
        assert abs(o.expected_value(1, avg) - v1) <= nc + 1e-9        # |u1(avg) - V*| <= NashConv
        assert nc < 0.05


def test_nashconv_equals_sum_of_overall_regrets():
    # 2p zero-sum, uniform averaging: sum_i r^(T)(i) = NashConv(avg), since the realisation-weighted
    # average of Eq. 10 is the sequence-form mean and u1 + u2 = 0 (Section 2.3).
    for g, tr in tiny_games(4, seed0=900):
        o = oracle.Oracle(g)
        hist = []
        for _ in range(12):
            hist.append(o.current_strategy().copy())
            o.iterate(1)
        nc, _ = o.exploitability()
        r = tr.overall_regret(hist, 1) + tr.overall_regret(hist, 2)
        assert nc == pytest.approx(r, abs=1e-11)


def test_regret_bounds():
    for g, tr in tiny_games(3, seed0=1000):
        o = oracle.Oracle(g)
        umax = np.abs(g.utility).max()
        delta = 2 * umax
        for T in (10, 100, 1000):
            o.iterate(T - o.state()["iteration"])
            st = o.state()
            nc, _ = o.exploitability()
            # Zinkevich et al. Thm 3: overall regret <= sum of positive immediate cf regrets
            imm = 0.0
            for h in range(tr.H):
                if tr.player[h] != 0:
                    imm += max(st["cum_regret"][tr.qbase[h]:tr.qbase[h] + tr.nact[h]].max(), 0.0) / T
            assert nc <= imm + 1e-12
            # regret-matching bound: NashConv <= Delta * sum_h sqrt|A(h)| / sqrt(T)
            bound = delta * sum(np.sqrt(tr.nact[h]) for h in range(tr.H) if tr.player[h] != 0) / np.sqrt(T)
            assert nc <= bound


# ------------------------------------------------------------------------------------------------
# 5. invariants
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("variant,avg", [(0, 0), (1, 1)])
def test_invariants_every_iteration(variant, avg):
    for g, tr in tiny_games(3, seed0=1100):
        o = oracle.Oracle(g, record=True)
        depth = np.array(tr.depth)
        term = np.array(g.infoset) < 0
        for _ in range(8):
            prev = o.current_strategy().copy()
            rv = o.iterate(1, variant=variant, avg=avg)
            st = o.state()
            nd = o.nodes()
            for h in range(tr.H):
                sl = slice(tr.qbase[h], tr.qbase[h] + tr.nact[h])
                assert st["sigma"][sl].sum() == pytest.approx(1.0, abs=1e-14)
                if tr.player[h] != 0:
                    # sum_a sigma(h,a) r~(h,a) = 0 exactly: sum_a sigma_a (u_a - u) = 0
                    assert np.dot(prev[sl], st["inst_regret"][sl]) == pytest.approx(0.0, abs=1e-12)
            np.testing.assert_allclose(nd["u1"] + nd["u2"], 0.0, atol=1e-13)
            pi = nd["cf1"] * nd["own1"]                 # non-player-1 factors x player-1 factors
            for lvl in range(depth.max() + 1):
                tot = pi[depth == lvl].sum() + pi[(depth < lvl) & term].sum()
                assert tot == pytest.approx(1.0, abs=1e-12)
            assert rv[0] == pytest.approx(float((pi[term] * g.utility[term, 0]).sum()), abs=1e-12)
            if variant == 1:
                assert np.all(st["cum_regret"] >= 0)
        assert o.recall_violations() == 0


def test_general_sum_payoffs_match_definition():
    rng = np.random.default_rng(12)
    for g, tr in tiny_games(3, seed0=1200, general_sum=True):
        o = oracle.Oracle(g, record=True)
        prof = _set_random_strategy(o, tr, rng)
        o.iterate(1)
        np.testing.assert_allclose(o.state()["inst_regret"], tr.inst_regret(prof), atol=1e-12)
        nd = o.nodes()
        assert nd["u2"][tr.root] == pytest.approx(tr.expected_payoff(prof, 2), abs=1e-12)


def test_oracle_rejects_malformed_trees():
    g, _ = hand_game()
    bad = gamegen.GameDesc(g.parent.copy(), g.action.copy(), g.infoset.copy(), g.infoset_player,
                           g.infoset_num_actions, g.chance_prob, g.utility)
    bad.action[4] = 0                                   # two children of n1 with action 0
    with pytest.raises(ValueError):
        oracle.Oracle(bad)
    bad2 = gamegen.GameDesc(g.parent.copy(), g.action.copy(), g.infoset.copy(), g.infoset_player,
                            g.infoset_num_actions, g.chance_prob, g.utility)
    bad2.parent[1] = -1                                 # two roots
    with pytest.raises(ValueError):
        oracle.Oracle(bad2)
