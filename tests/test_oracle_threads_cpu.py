"""The oracle's multi-threaded passes (used to time it on all host cores) against its one-thread
passes: the same state bit for bit, for every variant and update mode, on games whose infosets have
one node per root outcome (the deal-structured workloads), several nodes per root outcome (an
infoset spanning two depths), nodes of one infoset under every root child (a matrix game with a
player root), and node ids that are not in depth-first order."""
import numpy as np
import pytest

import gamegen
import oracle
from test_oracle_pins import multilevel_game, tiny_games

KEYS = ("cum_regret", "strat_sum", "inst_regret", "sigma", "own_reach", "cf_reach_sum")


def _games():
    yield "bucket3_depth6", gamegen.config("bucket3_depth6", seed=1)
    yield "rank13_cut", gamegen.first_deals(gamegen.config("rank13_depth10", seed=2, target_nodes=40_000), 20)
    yield "public_chance", tiny_games(count=1, seed0=101)[0][0]
    yield "multilevel", multilevel_game()
    yield "matrix", gamegen.matrix_game(np.array([[0.0, -1.0, 2.0], [1.5, 0.0, -1.0], [-1.0, 1.0, 0.0]]))
    yield "permuted", gamegen.permute_nodes(gamegen.config("bucket3_depth6", seed=4), 9)


RUNS = [(oracle.VANILLA, oracle.AVG_UNIFORM, False), (oracle.CFR_PLUS, oracle.AVG_LINEAR, False),
        (oracle.CFR_PLUS, oracle.AVG_LINEAR, True), (oracle.LINEAR, oracle.AVG_UNIFORM, False),
        (oracle.DISCOUNTED, oracle.AVG_UNIFORM, True)]


@pytest.mark.parametrize("name,game", list(_games()), ids=[n for n, _ in _games()])
@pytest.mark.parametrize("variant,avg,alt", RUNS)
def test_multi_threaded_passes_are_bit_identical(name, game, variant, avg, alt):
    one = oracle.Oracle(game, record=True)
    for threads in (2, 3, 8):
        many = oracle.Oracle(game, record=True)
        rv1 = rv2 = None
        for chunk in (1, 4, 7):
            rv1 = one.iterate(chunk, variant=variant, avg=avg, alternating=alt) if threads == 2 else rv1
            rv2 = many.iterate(chunk, variant=variant, avg=avg, alternating=alt, threads=threads)
        if threads == 2:
            s1, n1, v1 = one.state(), one.nodes(), rv1
        s2, n2 = many.state(), many.nodes()
        assert many.last_threads == threads or oracle.max_threads() == 1
        for k in KEYS:
            np.testing.assert_array_equal(s2[k], s1[k], err_msg=f"{name} {k} threads={threads}")
        assert s2["iteration"] == s1["iteration"]
        for k in n1:
            np.testing.assert_array_equal(n2[k], n1[k], err_msg=f"{name} node {k} threads={threads}")
        np.testing.assert_array_equal(rv2, v1)
        assert many.recall_violations() == one.recall_violations()
        np.testing.assert_array_equal(many.average_strategy(), one.average_strategy())


def test_all_threads_default():
    g = gamegen.config("bucket3_depth6", seed=1)
    o = oracle.Oracle(g)
    o.iterate(2, variant=oracle.CFR_PLUS, avg=oracle.AVG_LINEAR, threads=0)
    assert o.last_threads == oracle.max_threads() >= 1
