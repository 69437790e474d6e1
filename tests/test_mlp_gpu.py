"""The value network's kernels (cfr_mlp_*) against the FP64 oracle (oracle/mlp.py) in its BF16 mode,
which rounds at the same points as the kernels (GPU tests).

Element by element, layer by layer: every product is recomputed by the oracle from the kernels' own
BF16 inputs of that layer (the test hook cfr_mlp_get_intermediate), so each output entry has a
rigorous bound.  The products of BF16 values are exact in FP32, and the FP32 accumulation of K of them
(tensor-core or warp-level, in any order, with round-to-nearest or truncating alignment of the
addends) is within c K 2^-24 sum_k |a_k b_k| of the exact sum; c = 8 leaves a factor of two to four
over the worst case of either accumulation.  The sum of absolute products (|A||B|)_ij is computed by the
oracle on absolute values.  A result that the kernels round to BF16 (hidden activations, masked
gradients) must lie between the roundings of exact - E and exact + E (rounding is monotone); where the
two differ the kernels may round either way (a one-BF16-ulp flip), and such flips must stay rare
(at most 1% of a layer's entries).  An error confined to one tile, one bias row or one column would
break these bounds by orders of magnitude.

The whole network is also compared normwise with the oracle run from the input alone: outputs within
2e-3, gradients within 5e-3 (the flips above propagate), Adam (elementwise FP32) within 1e-5.
"""
import numpy as np
import pytest

import paper_2408_14778_gb300 as cfr
from oracle import mlp

pytestmark = pytest.mark.gpu

LEAF_DIMS = [64 + 2 * 169, 1024, 1024, 1024, 2 * 169]   # public embedding + two ranges -> two value vectors


U32 = 2.0 ** -24
C_ACC = 8.0


def _acc_bound(absprod, k):
    """Bound on |FP32 accumulation - exact| for reductions of length k with absolute-value sum absprod
    (plus one FP32 rounding of the bias addition, folded into k + 1)."""
    return C_ACC * (k + 1) * U32 * absprod


def _check_rounded(got, exact, err, rd, what):
    """got must be rd(v) for some v within err of exact (rd monotone); returns the number of entries
    where got differs from rd(exact)."""
    lo, hi = rd(exact - err), rd(exact + err)
    bad = ~((got >= lo) & (got <= hi))
    assert not bad.any(), (what, int(bad.sum()), np.argwhere(bad)[:5].tolist(),
                           got[bad][:5].tolist(), exact[bad][:5].tolist(), err[bad][:5].tolist())
    flips = int(np.count_nonzero(got != rd(exact)))
    assert flips <= max(3, 0.01 * got.size), (what, flips, got.size)
    return flips


def _check_close(got, exact, err, what):
    bad = np.abs(got - exact) > err
    assert not bad.any(), (what, int(bad.sum()), np.argwhere(bad)[:5].tolist(), got[bad][:5].tolist(),
                           exact[bad][:5].tolist(), err[bad][:5].tolist())


def _layerwise_forward(m, params, x, batch):
    """Every layer's product and epilogue element by element, from the kernels' own layer inputs."""
    a = cfr.cfr_mlp_get_intermediate(m, cfr.CFR_MLP_ACT, 0, batch).astype(np.float64)
    np.testing.assert_array_equal(a, mlp.bf16_round(x))            # the packed input is bf16(x), exactly
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = mlp.dense(a, W, b, bf16=True)
        err = _acc_bound(mlp.dense(np.abs(a), np.abs(W), np.abs(b), bf16=True), a.shape[1])
        if l + 1 < L:
            nxt = cfr.cfr_mlp_get_intermediate(m, cfr.CFR_MLP_ACT, l + 1, batch).astype(np.float64)
            _check_rounded(nxt, z, err, lambda v: mlp.hidden(v, bf16=True), f"hidden {l}")
            a = nxt
        else:
            y = cfr.cfr_mlp_get_intermediate(m, cfr.CFR_MLP_OUT, 0, batch).astype(np.float64)
            _check_close(y, z, err + U32 * np.abs(z), "output")
    return a


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def _net(dims, seed, path=cfr.MLP_PATH_MIXED):
    rng = np.random.default_rng(seed)
    params = mlp.init_params(dims, rng)
    m = cfr.cfr_mlp_create(dims)
    cfr.cfr_mlp_set_tensor_path(m, path)
    cfr.cfr_mlp_set_params(m, mlp.flatten(params).astype(np.float32))
    # the oracle uses the FP32 parameters the network holds
    params = mlp.unflatten(cfr.cfr_mlp_get_params(m).astype(np.float64), dims)
    return m, params, rng


PATHS = pytest.mark.parametrize("path", [cfr.MLP_PATH_MMA_SYNC, cfr.MLP_PATH_TCGEN05, cfr.MLP_PATH_MIXED],
                                ids=["mma_sync", "tcgen05", "mixed"])


@PATHS
@pytest.mark.parametrize("dims,batch", [(LEAF_DIMS, 300), ([5, 7, 3], 1), ([130, 200, 129], 128), ([1, 1], 3),
                                        ([33, 300, 300, 17], 257), ([64, 512, 512, 64], 4096),
                                        ([128, 1024, 256], 9728)])   # the last: 256-wide tcgen05 tiles
def test_forward_matches_oracle(dims, batch, path):
    import torch

    m, params, rng = _net(dims, seed=len(dims) * 1000 + batch, path=path)
    x = rng.normal(size=(batch, dims[0])).astype(np.float32)
    y = cfr.cfr_mlp_forward(m, torch.tensor(x, device="cuda")).cpu().numpy().astype(np.float64)
    cfr.cfr_mlp_synchronize(m)
    _layerwise_forward(m, params, x.astype(np.float64), batch)
    np.testing.assert_array_equal(y, cfr.cfr_mlp_get_intermediate(m, cfr.CFR_MLP_OUT, 0, batch))
    ref, _ = mlp.forward(params, x.astype(np.float64), bf16=True)
    assert _rel(y, ref) <= 2e-3


@PATHS
@pytest.mark.parametrize("dims,batch", [(LEAF_DIMS, 300), ([5, 7, 3], 2), ([130, 200, 129], 128),
                                        ([33, 300, 300, 17], 257)])
def test_gradients_match_oracle(dims, batch, path):
    import torch

    m, params, rng = _net(dims, seed=7 + batch, path=path)
    x = rng.normal(size=(batch, dims[0])).astype(np.float32)
    t = rng.normal(size=(batch, dims[-1])).astype(np.float32)
    loss = cfr.cfr_mlp_backward(m, torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")).item()
    g = mlp.unflatten(cfr.cfr_mlp_get_grads(m).astype(np.float64), dims)
    # element by element, from the kernels' own intermediates of this backward pass
    _layerwise_forward(m, params, x.astype(np.float64), batch)
    y = cfr.cfr_mlp_get_intermediate(m, cfr.CFR_MLP_OUT, 0, batch).astype(np.float64)
    dz = cfr.cfr_mlp_get_intermediate(m, cfr.CFR_MLP_DZ, len(params) - 1, batch).astype(np.float64)
    # dL/dy: the kernels form y - t and scale it in FP32 (two roundings) before rounding to BF16
    v = mlp.output_gradient(y, t.astype(np.float64))
    _check_rounded(dz, v, 4 * U32 * np.abs(v), lambda u: mlp.bf16_round(u), "output gradient")
    Bp = -(-batch // 128) * 128                                      # the kernels' padded batch
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        a = cfr.cfr_mlp_get_intermediate(m, cfr.CFR_MLP_ACT, l, batch).astype(np.float64)
        rW, rb = mlp.layer_gradients(dz, a)
        aW, ab = mlp.layer_gradients(np.abs(dz), np.abs(a))
        _check_close(g[l][0], rW, _acc_bound(aW, Bp) + U32 * np.abs(rW), f"dW {l}")
        _check_close(g[l][1], rb, _acc_bound(ab, Bp) + U32 * np.abs(rb), f"db {l}")
        if l > 0:
            prev = cfr.cfr_mlp_get_intermediate(m, cfr.CFR_MLP_DZ, l - 1, batch).astype(np.float64)
            exact = mlp.masked_product(dz, W, a, bf16=True)
            err = _acc_bound(mlp.masked_product(np.abs(dz), np.abs(W), a, bf16=True), W.shape[0])
            assert not prev[~(a > 0)].any(), f"masked gradient {l - 1}"   # zero where the ReLU output was 0
            _check_rounded(prev, exact, err, lambda u: mlp.bf16_round(u), f"masked gradient {l - 1}")
            dz = prev
    # and the whole network from the input alone, normwise
    ref_loss, ref = mlp.loss_and_grads(params, x.astype(np.float64), t.astype(np.float64), bf16=True)
    assert loss == pytest.approx(ref_loss, rel=1e-3)
    for l, ((gW, gb), (rW, rb)) in enumerate(zip(g, ref)):
        assert _rel(gW, rW) <= 5e-3, l
        assert _rel(gb, rb) <= 5e-3, l


def test_adam_step_matches_oracle():
    import torch

    dims = [40, 64, 10]
    m, params, rng = _net(dims, seed=3)
    state = {}
    for _ in range(3):
        x = rng.normal(size=(50, dims[0])).astype(np.float32)
        t = rng.normal(size=(50, dims[-1])).astype(np.float32)
        cfr.cfr_mlp_backward(m, torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"))
        g = mlp.unflatten(cfr.cfr_mlp_get_grads(m).astype(np.float64), dims)   # the kernels' own gradients
        cfr.cfr_mlp_adam(m, 1e-3, 0.9, 0.999, 1e-8)
        params = mlp.adam_step(params, g, state, lr=1e-3)
        got = cfr.cfr_mlp_get_params(m).astype(np.float64)
        np.testing.assert_allclose(got, mlp.flatten(params), rtol=1e-5, atol=1e-7)
        params = mlp.unflatten(got, dims)


def test_training_fits_a_teacher_network():
    import torch

    dims = [32, 256, 256, 8]
    rng = np.random.default_rng(11)
    teacher = mlp.init_params(dims, rng)
    x = rng.normal(size=(2048, dims[0]))
    t, _ = mlp.forward(teacher, x)
    m = cfr.cfr_mlp_create(dims)
    cfr.cfr_mlp_set_params(m, mlp.flatten(mlp.init_params(dims, rng)).astype(np.float32))
    xd, td = torch.tensor(x, dtype=torch.float32, device="cuda"), torch.tensor(t, dtype=torch.float32, device="cuda")
    first = cfr.cfr_mlp_backward(m, xd, td).item()
    for _ in range(300):
        cfr.cfr_mlp_backward(m, xd, td)
        cfr.cfr_mlp_adam(m, 1e-3)
    last = cfr.cfr_mlp_backward(m, xd, td).item()
    assert last < 0.1 * first, (first, last)


def test_invalid_arguments():
    with pytest.raises(cfr.CfrError) as e:
        cfr.cfr_mlp_create([4])
    assert e.value.status == cfr.CFR_ERR_INVALID
    with pytest.raises(cfr.CfrError):
        cfr.cfr_mlp_create([4, 0, 2])
    m = cfr.cfr_mlp_create([4, 2])
    with pytest.raises(cfr.CfrError):
        cfr.cfr_mlp_set_params(m, np.zeros(3, np.float32))
    with pytest.raises(cfr.CfrError):
        cfr.cfr_mlp_adam(m, 1e-3, beta1=1.0)
