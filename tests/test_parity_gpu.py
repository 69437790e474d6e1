"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

FP64 mode performs the oracle's operations in the oracle's order (no fused multiply-add,
deterministic per-infoset regret reduction in depth-first node order), so its results are compared
at 1e-12 and are in practice bit-identical.  FP32 mode is compared at 1e-5 one step at a time from
the oracle's FP64 state (step parity), with strategies checked as in paritylib.fp32_sigma_check.
"""
import numpy as np
import pytest

import gamegen
import oracle
import paper_2408_14778_gb300 as cfr
from paritylib import TOL32, TOL64, TOL_EXPL, compare_nodes, compare_state, normwise, player_mask

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    cfr.build()


def small_games():
    games = [gamegen.config("bucket3_depth6", seed=1),
             gamegen.public_private(seed=11, num_buckets=3, depth=6, amin=1, amax=4, p_cont=0.7, p_chance=0.3),
             gamegen.public_private(seed=12, num_buckets=4, depth=7, amin=2, amax=3, p_cont=0.6, p_chance=0.2,
                                    payoff_kind=gamegen.PAY_FOLD_SHOWDOWN, first_actor=2),
             gamegen.matrix_game([[0, -1, 1], [1, 0, -1], [-1, 1, 0]]),
             gamegen.matrix_game(np.arange(12.0).reshape(3, 4) - 5)]
    games.append(gamegen.permute_nodes(games[1], seed=99))
    return games


@pytest.mark.parametrize("variant", [cfr.CFR_VANILLA, cfr.CFR_PLUS])
def test_step_by_step_fp64(variant):
    for g in small_games():
        o = oracle.Oracle(g, record=True)
        s = cfr.cfr_load_tree(g, variant=variant, precision=cfr.CFR_FP64)
        for _ in range(5):
            o.iterate(1, variant=variant, avg=variant)
            cfr.cfr_iterate(s, 1)
            compare_state(s, o, TOL64, g)
            compare_nodes(s, o, TOL64, g)
            np.testing.assert_allclose(cfr.cfr_get_state(s)["own_reach"][g.infoset_player > 0],
                                       o.state()["own_reach"][g.infoset_player > 0], atol=1e-15)
        s.close()


def test_trajectory_fp64_vanilla_1000_iterations():
    # bucket3_depth6: 6-way deal of 3 buckets, depth 6, |A| in {2,3}; vanilla CFR in FP64.
    g = gamegen.config("bucket3_depth6", seed=1)
    o = oracle.Oracle(g)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_VANILLA, precision=cfr.CFR_FP64)
    done = 0
    for T in (1, 10, 100, 1000):
        o.iterate(T - done)
        cfr.cfr_iterate(s, T - done)
        done = T
        compare_state(s, o, TOL64, g)
        assert normwise(cfr.cfr_average_strategy(s), o.average_strategy()) <= TOL64
        nc_g, ex_g = cfr.cfr_exploitability(s)
        nc_o, ex_o = o.exploitability()
        assert abs(nc_g - nc_o) <= TOL_EXPL and abs(ex_g - ex_o) <= TOL_EXPL


def test_trajectory_fp64_cfr_plus():
    for g in small_games()[:3]:
        o = oracle.Oracle(g)
        s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP64)
        o.iterate(300, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
        cfr.cfr_iterate(s, 300)
        compare_state(s, o, TOL64, g)
        assert normwise(cfr.cfr_average_strategy(s), o.average_strategy()) <= TOL64
        assert abs(cfr.cfr_exploitability(s)[0] - o.exploitability()[0]) <= TOL_EXPL


def test_fp64_is_bit_identical_to_the_oracle():
    # Same operations in the same order: the FP64 path reproduces the oracle exactly.
    g = gamegen.config("rank13_depth10", seed=2, target_nodes=200_000)
    o = oracle.Oracle(g)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP64)
    o.iterate(50, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
    cfr.cfr_iterate(s, 50)
    gs, os_ = cfr.cfr_get_state(s), o.state()
    for k in ("cum_regret", "strat_sum", "inst_regret"):
        np.testing.assert_array_equal(gs[k], os_[k])
    np.testing.assert_array_equal(cfr.cfr_current_strategy(s), os_["sigma"])


@pytest.mark.parametrize("fuse", [0, 2, 4])
@pytest.mark.parametrize("variant", [cfr.CFR_VANILLA, cfr.CFR_PLUS])
def test_one_iteration_fp32(variant, fuse):
    # fuse: the deepest depths in one kernel (none; the last two by k_tail; four in tiles)
    for g in small_games():
        o = oracle.Oracle(g, record=True)
        s = cfr.cfr_load_tree(g, variant=variant, precision=cfr.CFR_FP32, fuse_levels=fuse, record_nodes=True)
        o.iterate(1, variant=variant, avg=variant)
        cfr.cfr_iterate(s, 1)
        compare_state(s, o, TOL32, g)
        compare_nodes(s, o, TOL32, g)


def test_fp32_nine_to_twelve_actions():
    # 9..12 actions per node at every depth: the streamed kernels' general (more than 8 actions) path on
    # depths of >= 32768 nodes, and the unrolled per-depth kernels' general path on the small ones.
    g = gamegen.public_private(seed=31, num_buckets=13, depth=6, amin=9, amax=12, p_cont=0.45)
    for variant in (cfr.CFR_VANILLA, cfr.CFR_PLUS):
        o = oracle.Oracle(g, record=True)
        s = cfr.cfr_load_tree(g, variant=variant, precision=cfr.CFR_FP32, record_nodes=True)
        o.iterate(1, variant=variant, avg=variant)
        cfr.cfr_iterate(s, 1)
        compare_state(s, o, TOL32, g)
        compare_nodes(s, o, TOL32, g)
        st = o.state()
        cfr.cfr_set_state(s, st["cum_regret"], st["strat_sum"], st["iteration"])
        o.iterate(1, variant=variant, avg=variant)
        cfr.cfr_iterate(s, 1)
        compare_state(s, o, TOL32, g)


def _step_parity(g, variant, Ts, precision, tol, nodes=False, fuse=-1, tail_slots=-1):
    o = oracle.Oracle(g, record=nodes)
    s = cfr.cfr_load_tree(g, variant=variant, precision=precision, fuse_levels=fuse, record_nodes=nodes,
                          tail_slots=tail_slots)
    done = 0
    for T in Ts:
        o.iterate(T - 1 - done, variant=variant, avg=variant)
        done = T - 1
        st = o.state()
        cfr.cfr_set_state(s, st["cum_regret"], st["strat_sum"], st["iteration"])
        assert normwise(cfr.cfr_current_strategy(s), st["sigma"]) <= (TOL64 if precision == cfr.CFR_FP64 else 1e-7)
        o.iterate(1, variant=variant, avg=variant)
        done += 1
        cfr.cfr_iterate(s, 1)
        compare_state(s, o, tol, g)
        if nodes:
            compare_nodes(s, o, tol, g)
    return s, o


@pytest.mark.parametrize("fuse,slots,kernel", [(2, 1, 3), (2, 2, 4), (2, 0, 2), (0, 0, 0)],
                         ids=["tail_slots", "tail_slots_bulk", "tail_stream", "per_depth"])
def test_step_parity_fp32_rank13_depth10(fuse, slots, kernel):
    # ~2e6 nodes, 156-way deal, fold/showdown payoffs, CFR+: one FP32 step from the oracle's FP64
    # state at T = 1, 2, 10, 100 (step parity), with the last two depths fused (slot-dense tiles with
    # staged strategy entries and bulk-reduced regrets, or per-slot loads and atomics) and not.
    g = gamegen.config("rank13_depth10", seed=1)
    s, o = _step_parity(g, cfr.CFR_PLUS, (1, 2, 10, 100), cfr.CFR_FP32, TOL32, nodes=fuse == 2, fuse=fuse,
                        tail_slots=slots)
    info = cfr.cfr_get_info(s)
    assert (info["fused_from_depth"] < info["num_levels"]) == (fuse == 2)
    assert info["tail_kernel"] == kernel
    nc_g, _ = cfr.cfr_exploitability(s)
    nc_o, _ = o.exploitability()
    assert abs(nc_g - nc_o) <= 1e-5 * max(1.0, abs(nc_o))


def test_step_parity_fp64_rank13_depth10():
    g = gamegen.config("rank13_depth10", seed=2)
    s, o = _step_parity(g, cfr.CFR_VANILLA, (1, 5), cfr.CFR_FP64, TOL64, nodes=True)
    assert abs(cfr.cfr_exploitability(s)[0] - o.exploitability()[0]) <= TOL_EXPL


def test_fp32_trajectory_converges_like_the_oracle():
    # Over many iterations FP32 rounding re-decides near-tied regrets, so the trajectories part;
    # the solution quality must not: NashConv of the average strategy tracks the FP64 oracle's.
    g = gamegen.config("rank13_depth10", seed=3, target_nodes=300_000)
    o = oracle.Oracle(g)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32)
    for T in (10, 100, 400):
        o.iterate(T - o.state()["iteration"], variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
        cfr.cfr_iterate(s, T - cfr.cfr_get_info(s)["iteration"])
        nc_g, _ = cfr.cfr_exploitability(s)
        nc_o, _ = o.exploitability()
        assert nc_g <= 1.1 * nc_o + 1e-4, (T, nc_g, nc_o)
        nc_chk, _ = o.exploitability(cfr.cfr_average_strategy(s))      # oracle's BR on the GPU's strategy
        assert abs(nc_chk - nc_g) <= TOL_EXPL


# ---- edge cases ---------------------------------------------------------------------------------

def test_terminal_root():
    g = gamegen.GameDesc(np.array([-1], np.int32), np.array([-1], np.int32), np.array([-1], np.int32),
                         np.zeros(0, np.int8), np.zeros(0, np.int32), np.zeros(0), np.array([[2.0, -2.0]]))
    s = cfr.cfr_load_tree(g, precision=cfr.CFR_FP64)
    cfr.cfr_iterate(s, 3)
    assert cfr.cfr_exploitability(s) == (0.0, 0.0)
    assert cfr.cfr_get_nodes(s)["u1"][0] == 2.0
    assert cfr.cfr_root_value(s) == 2.0
    assert cfr.cfr_get_info(s)["iteration"] == 3


def test_chance_only_tree():
    parent = np.array([-1, 0, 0, 0, 1, 1], np.int32)
    action = np.array([-1, 0, 1, 2, 0, 1], np.int32)
    infoset = np.array([0, 1, -1, -1, -1, -1], np.int32)
    util = np.zeros((6, 2))
    util[:, 0] = [0, 0, 1.0, -3.0, 2.0, 5.0]
    util[:, 1] = -util[:, 0]
    g = gamegen.GameDesc(parent, action, infoset, np.array([0, 0], np.int8), np.array([3, 2], np.int32),
                         np.array([0.5, 0.25, 0.25, 0.1, 0.9]), util)
    s = cfr.cfr_load_tree(g, precision=cfr.CFR_FP64)
    o = oracle.Oracle(g, record=True)
    o.iterate(2)
    cfr.cfr_iterate(s, 2)
    compare_nodes(s, o, TOL64, g)
    assert cfr.cfr_exploitability(s)[0] == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("m,n", [(1, 3), (12, 20), (9, 32), (33, 2), (64, 3), (5, 64), (200, 3), (3, 1326)])
def test_wide_and_single_action_infosets(m, n):
    rng = np.random.default_rng(m * 100 + n)
    g = gamegen.matrix_game(rng.normal(size=(m, n)))
    for precision, tol in ((cfr.CFR_FP64, TOL64), (cfr.CFR_FP32, TOL32)):
        o = oracle.Oracle(g, record=True)
        s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=precision, record_nodes=True)
        o.iterate(1, variant=1, avg=1)
        cfr.cfr_iterate(s, 1)
        compare_state(s, o, tol, g)
        compare_nodes(s, o, tol, g)
        if precision == cfr.CFR_FP64:
            o.iterate(6, variant=1, avg=1)
            cfr.cfr_iterate(s, 6)
            compare_state(s, o, tol, g)


def test_zero_probability_branch():
    g = gamegen.public_private(seed=21, num_buckets=3, depth=5, amin=2, amax=3, p_cont=0.8, p_chance=0.4)
    cp = g.chance_prob.copy()
    cp[:6] = [0.5, 0.5, 0.0, 0.0, 0.0, 0.0]                  # four of six deals never happen
    g = gamegen.GameDesc(g.parent, g.action, g.infoset, g.infoset_player, g.infoset_num_actions, cp, g.utility)
    o = oracle.Oracle(g, record=True)
    s = cfr.cfr_load_tree(g, precision=cfr.CFR_FP64)
    o.iterate(10)
    cfr.cfr_iterate(s, 10)
    compare_state(s, o, TOL64, g)
    compare_nodes(s, o, TOL64, g)
    assert abs(cfr.cfr_exploitability(s)[0] - o.exploitability()[0]) <= TOL_EXPL


def test_multilevel_infoset_iterates_but_br_is_unsupported():
    from test_oracle_pins import multilevel_game

    g = multilevel_game()
    o = oracle.Oracle(g, record=True)
    s = cfr.cfr_load_tree(g, precision=cfr.CFR_FP64)
    assert cfr.cfr_get_info(s)["single_level_infosets"] == 0
    for _ in range(4):
        o.iterate(1)
        cfr.cfr_iterate(s, 1)
        compare_state(s, o, TOL64, g)
        compare_nodes(s, o, TOL64, g)
    with pytest.raises(cfr.CfrError) as e:
        cfr.cfr_exploitability(s)
    assert e.value.status == cfr.CFR_ERR_UNSUPPORTED


def _edge_games():
    from test_oracle_pins import multilevel_game

    g = gamegen.public_private(seed=21, num_buckets=3, depth=5, amin=2, amax=3, p_cont=0.8, p_chance=0.4)
    cp = g.chance_prob.copy()
    cp[:6] = [0.5, 0.5, 0.0, 0.0, 0.0, 0.0]
    zero = gamegen.GameDesc(g.parent, g.action, g.infoset, g.infoset_player, g.infoset_num_actions, cp, g.utility)
    deep = gamegen.public_private(seed=22, num_buckets=3, depth=9, amin=2, amax=3, p_cont=0.7, p_chance=0.2)
    return {"zero_probability_branch": zero, "multilevel_infoset": multilevel_game(), "public_chance_depth9": deep}


@pytest.mark.parametrize("fuse", [2, 8])
@pytest.mark.parametrize("name", ["zero_probability_branch", "multilevel_infoset", "public_chance_depth9"])
def test_fp32_fused_depths_on_edge_games(name, fuse):
    # The fused kernel on chance nodes inside the fused depths, unreachable subtrees, an infoset spanning
    # depths (own reach through the own-sequence chain) and up to 8 fused depths from the root.
    g = _edge_games()[name]
    o = oracle.Oracle(g, record=True)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32, fuse_levels=fuse, record_nodes=True)
    info = cfr.cfr_get_info(s)
    assert info["fused_from_depth"] < info["num_levels"]
    for T in (1, 2, 3):
        o.iterate(1, variant=1, avg=1)
        cfr.cfr_iterate(s, 1)
        compare_state(s, o, TOL32, g)
        compare_nodes(s, o, TOL32, g)
        st = o.state()                                  # next step from the oracle's state (step parity)
        cfr.cfr_set_state(s, st["cum_regret"], st["strat_sum"], st["iteration"])


def test_get_nodes_needs_record_when_fused():
    g = gamegen.config("bucket3_depth6", seed=1)
    s = cfr.cfr_load_tree(g, precision=cfr.CFR_FP32, fuse_levels=2)
    info = cfr.cfr_get_info(s)
    assert info["fused_from_depth"] < info["num_levels"] and info["fused_tiles"] > 0
    cfr.cfr_iterate(s, 1)
    with pytest.raises(cfr.CfrError) as e:
        cfr.cfr_get_nodes(s)
    assert e.value.status == cfr.CFR_ERR_STATE
    cfr.cfr_iterate(s, 1)                                 # still usable
    cfr.cfr_synchronize(s)


def test_state_roundtrip_and_cuda_allocator():
    g = gamegen.config("bucket3_depth6", seed=4)
    a = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP64)
    cfr.cfr_iterate(a, 17)
    st = cfr.cfr_get_state(a)
    b = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP64, allocator="cuda")
    cfr.cfr_set_state(b, st["cum_regret"], st["strat_sum"], st["iteration"])
    np.testing.assert_array_equal(cfr.cfr_current_strategy(a), cfr.cfr_current_strategy(b))
    cfr.cfr_iterate(a, 5)
    cfr.cfr_iterate(b, 5)
    np.testing.assert_array_equal(cfr.cfr_get_state(b)["cum_regret"], cfr.cfr_get_state(a)["cum_regret"])
    assert cfr.cfr_get_info(b)["iteration"] == 22
    mask = player_mask(g)
    assert np.all(cfr.cfr_get_state(b)["cum_regret"][~mask] == 0)


def test_root_value_is_expected_payoff():
    g = gamegen.config("bucket3_depth6", seed=5)
    o = oracle.Oracle(g)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP64)
    for _ in range(3):
        rv = o.iterate(1, variant=1, avg=1)
        cfr.cfr_iterate(s, 1)
        assert cfr.cfr_root_value(s) == rv[0]


def test_root_value_async_matches_the_synchronous_read():
    import torch

    buf = torch.zeros(2, dtype=torch.float64, pin_memory=True)
    g = gamegen.config("bucket3_depth6", seed=5)
    for precision in (cfr.CFR_FP64, cfr.CFR_FP32):
        s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=precision)
        for t in range(4):
            cfr.cfr_iterate(s, 1)
            cfr.cfr_root_value_async(s, buf.data_ptr() + 8 * (t % 2))
            cfr.cfr_synchronize(s)
            assert buf[t % 2].item() == cfr.cfr_root_value(s)
        with pytest.raises(cfr.CfrError):                  # pageable host memory is refused
            cfr.cfr_root_value_async(s, np.zeros(1).ctypes.data)
        s.close()


def test_bad_arguments_raise():
    g = gamegen.config("bucket3_depth6", seed=4)
    s = cfr.cfr_load_tree(g)
    with pytest.raises(cfr.CfrError):
        cfr.cfr_set_state(s, np.zeros(3), np.zeros(3), 0)
    with pytest.raises(cfr.CfrError):
        cfr.cfr_iterate(s, -1)
    L = cfr.lib()
    buf = np.zeros(2)
    assert L.cfr_average_strategy(s.handle, buf.ctypes.data, 2) == cfr.CFR_ERR_INVALID
    cfr.cfr_iterate(s, 2)                                     # still usable after argument errors
    cfr.cfr_synchronize(s)


def _node_depths(g):
    """Depth of every node (root 0), by following parents."""
    d = np.full(g.num_nodes, -1, np.int64)
    d[g.parent < 0] = 0
    while (d < 0).any():
        todo = d < 0
        known = d[g.parent[todo]] >= 0
        idx = np.nonzero(todo)[0][known]
        d[idx] = d[g.parent[idx]] + 1
    return d


@pytest.mark.parametrize("precision,fuse", [(cfr.CFR_FP64, -1), (cfr.CFR_FP32, 0), (cfr.CFR_FP32, -1)])
def test_phase_times_run_a_real_iteration(precision, fuse):
    g = gamegen.config("rank13_depth10", seed=6, target_nodes=None, p_cont=0.6)
    o = oracle.Oracle(g)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=precision, fuse_levels=fuse)
    o.iterate(2, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
    st = o.state()                                            # (FP32 is compared one step from FP64 state)
    cfr.cfr_set_state(s, st["cum_regret"], st["strat_sum"], st["iteration"])
    ph = cfr.cfr_phase_times(s)                               # the third iteration, kernel by kernel
    o.iterate(1, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR)
    compare_state(s, o, TOL64 if precision == cfr.CFR_FP64 else TOL32, g)
    info = cfr.cfr_get_info(s)
    assert info["iteration"] == 3
    assert all(p["us"] > 0 for p in ph)
    assert abs(sum(p["bytes"] for p in ph) - info["bytes_per_iteration"]) <= 1
    L, f = info["num_levels"], info["fused_from_depth"]
    kinds = [p["kind"] for p in ph]
    n_td = f if f < L else max(L - 1, 1)                     # the last depth has no top-down step
    assert kinds == [cfr.CFR_PHASE_OWN] + [cfr.CFR_PHASE_TOPDOWN] * n_td + [cfr.CFR_PHASE_FUSED] * (f < L) + \
        [cfr.CFR_PHASE_BOTTOMUP] * f + [cfr.CFR_PHASE_UPDATE]
    if f == L:
        # every node but the root is some depth's child, and the last depth (no decision children) has no
        # top-down step: the byte model in closed form
        Nd, Nt, Q = info["num_decision"], info["num_terminal"], info["num_q"]
        Hp = int((g.infoset_player > 0).sum())
        dd = _node_depths(g)[g.infoset >= 0]
        last = int((dd == dd.max()).sum()) if L >= 2 else 0
        want = (96 * Nd + 8 * Nt + 56 * Q + 17 * Hp - 24 - 32 * last if precision == cfr.CFR_FP64
                else 56 * Nd + 4 * Nt + 44 * Q + 13 * Hp - 12 - 20 * last)
        assert info["bytes_per_iteration"] == want
    else:
        assert precision == cfr.CFR_FP32 and info["fused_tiles"] > 0


def test_unaligned_device_allocator_is_rejected():
    # A caller's allocator must return 256-byte aligned blocks, as cudaMalloc does: the kernels' bulk copies
    # need 16-byte aligned arrays.  One that returns blocks 16 bytes off fails the load with CFR_ERR_INVALID
    # and gets every block it handed out back.
    import ctypes

    import torch

    lib = cfr.lib()
    d = cfr._Desc(gamegen.config("bucket3_depth6", seed=1))
    c = cfr._Config()
    lib.cfr_config_init(ctypes.byref(c))
    c.precision, c.device = cfr.CFR_FP32, torch.cuda.current_device()
    held = {}

    def alloc(nbytes, ctx):
        p = int(torch.cuda.caching_allocator_alloc(int(nbytes) + 256, c.device))
        held[p + 16] = p
        return p + 16

    def free(ptr, ctx):
        torch.cuda.caching_allocator_delete(held.pop(int(ptr)))

    a, f = cfr._ALLOC_FN(alloc), cfr._FREE_FN(free)
    c.dev_alloc, c.dev_free = a, f
    h = ctypes.c_void_p()
    st = lib.cfr_load_tree(ctypes.byref(d.c), ctypes.byref(c), ctypes.byref(h))
    assert st == cfr.CFR_ERR_INVALID and b"256-byte" in lib.cfr_last_error(None)
    assert not held and not h.value
