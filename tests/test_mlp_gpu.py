"""The value network's kernels (cfr_mlp_*) against the FP64 oracle (oracle/mlp.py) in its BF16 mode,
which rounds at the same points as the kernels (GPU tests).

Tolerances: the kernels accumulate in FP32 over K <= 1024 products, a relative error near K 2^-24 at
worst (about 1e-4) and far less on average; a hidden activation whose FP32 value differs from the
oracle's by that much can round to the neighbouring BF16 value (one BF16 ulp, 2^-8 relative) - a rare
event that moves a result by about 4e-3 times one term's share.  Normwise, outputs must agree to 2e-3
and gradients to 5e-3; Adam, elementwise FP32 arithmetic, to 1e-5.
"""
import numpy as np
import pytest

import paper_2408_14778_gb300 as cfr
from oracle import mlp

pytestmark = pytest.mark.gpu

LEAF_DIMS = [64 + 2 * 169, 1024, 1024, 1024, 2 * 169]   # public embedding + two ranges -> two value vectors


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
    ref, _ = mlp.forward(params, x.astype(np.float64), bf16=True)
    assert _rel(y, ref) <= 2e-3
    assert np.max(np.abs(y - ref)) <= 2e-2 * np.max(np.abs(ref)) + 1e-6


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
