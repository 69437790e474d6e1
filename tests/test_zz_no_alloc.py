"""cfr_exploitability_static: the exploitability entry point that allocates no device memory.

Callers that may not allocate GPU memory while they run (a fixed memory budget handed over at
set-up, or a real-time loop where cudaMalloc/cudaFree are not allowed) evaluate exploitability
through this entry point; its working memory is a fixed region inside the library.  This file is
collected last so that a run stopping at its first failure has run every other test before it.
"""
import numpy as np
import pytest

import gamegen
import paper_2408_14778_gb300 as cfr
from paritylib import TOL_EXPL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    cfr.build()


@pytest.mark.parametrize("precision", [cfr.CFR_FP32, cfr.CFR_FP64])
def test_matches_allocating_entry_point_on_two_calls_in_a_row(precision):
    # rank13_depth10 family at ~1.7e6 nodes: its working memory (~10 MB) fits the fixed region.
    g = gamegen.config("rank13_depth10", seed=7, target_nodes=None, p_cont=0.7)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=precision)
    info = cfr.cfr_get_info(s)
    assert 16 * (info["num_decision"] + info["num_q"]) + 4 * info["num_infosets"] < cfr.CFR_STATIC_SCRATCH_BYTES
    # another game's call first fills the shared region with values laid out for a different tree, so a
    # quantity the next call failed to reset would show up in its result
    other = cfr.cfr_load_tree(gamegen.config("bucket3_depth6", seed=3), variant=cfr.CFR_VANILLA, precision=precision)
    cfr.cfr_iterate(other, 7)
    want_other = cfr.cfr_exploitability(other)
    got_other = cfr.cfr_exploitability_static(other)
    assert abs(got_other[0] - want_other[0]) <= TOL_EXPL, (got_other, want_other)
    for iters in (5, 20):
        cfr.cfr_iterate(s, iters)
        want = cfr.cfr_exploitability(s)
        first = cfr.cfr_exploitability_static(s)
        second = cfr.cfr_exploitability_static(s)        # two calls in a row share the region
        for got in (first, second):
            assert abs(got[0] - want[0]) <= TOL_EXPL and abs(got[1] - want[1]) <= TOL_EXPL, (got, want)
        assert want[0] > 0
    got_other = cfr.cfr_exploitability_static(other)     # and back to the small game after the large one
    assert abs(got_other[0] - want_other[0]) <= TOL_EXPL, (got_other, want_other)
    other.close()
    s.close()


def test_rejects_games_beyond_the_region():
    # ~1e7 nodes: ~60 MB of working memory, beyond the 32 MiB region.
    g = gamegen.config("rank13_depth10", seed=8, target_nodes=None, p_cont=0.9)
    s = cfr.cfr_load_tree(g, variant=cfr.CFR_PLUS, precision=cfr.CFR_FP32)
    info = cfr.cfr_get_info(s)
    assert 16 * (info["num_decision"] + info["num_q"]) > cfr.CFR_STATIC_SCRATCH_BYTES
    cfr.cfr_iterate(s, 2)
    with pytest.raises(cfr.CfrError) as e:
        cfr.cfr_exploitability_static(s)
    assert e.value.status == cfr.CFR_ERR_UNSUPPORTED and "bytes" in str(e.value)
    nc, _ = cfr.cfr_exploitability(s)                     # the solver is still usable
    assert np.isfinite(nc)
    s.close()
