"""Pins of the CPU value-network oracle (oracle/mlp.py) against facts fixed by mathematics (no GPU).

Checked against something other than itself: central finite differences of the loss (independent of
backpropagation), the least-squares solution of a linear model (numpy's lstsq), Adam's closed-form
first step, positive homogeneity of a bias-free ReLU network, and BF16 rounding against PyTorch's
conversion.
"""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_rounding_matches_a_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-30, 30, size=2000),
                        [0.0, -0.0, 1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, 1.0 + 3 * 2.0 ** -9,
                         65504.0, 3.4e38, -1.0e-40, 1.0e-45]])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), ref)
    # ties go to the even neighbour: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert mlp.bf16_round(1.0 + 2.0 ** -8) == 1.0
    assert mlp.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


def test_gradients_match_central_differences():
    rng = np.random.default_rng(1)
    dims = [5, 7, 6, 3]
    params = mlp.init_params(dims, rng)
    x, t = rng.normal(size=(4, 5)), rng.normal(size=(4, 3))
    _, grads = mlp.loss_and_grads(params, x, t)
    flat, gflat = mlp.flatten(params), mlp.flatten(grads)
    h = 1e-6
    fd = np.zeros_like(flat)
    for i in range(flat.size):
        up, dn = flat.copy(), flat.copy()
        up[i] += h
        dn[i] -= h
        fd[i] = (mlp.loss_and_grads(mlp.unflatten(up, dims), x, t)[0] -
                 mlp.loss_and_grads(mlp.unflatten(dn, dims), x, t)[0]) / (2 * h)
    np.testing.assert_allclose(gflat, fd, rtol=1e-5, atol=1e-8)


def test_loss_of_the_zero_network_is_the_mean_square_target():
    rng = np.random.default_rng(2)
    dims = [3, 4, 2]
    params = [(np.zeros((4, 3)), np.zeros(4)), (np.zeros((2, 4)), np.zeros(2))]
    x, t = rng.normal(size=(6, 3)), rng.normal(size=(6, 2))
    loss, grads = mlp.loss_and_grads(params, x, t)
    assert loss == pytest.approx(np.mean(t ** 2), rel=1e-14)
    np.testing.assert_allclose(grads[1][1], -2 * t.mean(axis=0) / 2, rtol=1e-12)   # d/db of mean (b - t)^2


def test_bias_free_relu_network_is_positively_homogeneous():
    rng = np.random.default_rng(3)
    dims = [6, 9, 9, 4]
    params = [(W, np.zeros_like(b)) for W, b in mlp.init_params(dims, rng)]
    x = rng.normal(size=(5, 6))
    y1, _ = mlp.forward(params, x)
    y2, _ = mlp.forward(params, 3.5 * x)
    np.testing.assert_allclose(y2, 3.5 * y1, rtol=1e-12, atol=1e-12)
    y3, _ = mlp.forward(params, -x)          # a ReLU network is not odd: the negated input differs
    assert not np.allclose(y3, -y1)


def test_adam_first_step_moves_each_parameter_by_the_learning_rate():
    rng = np.random.default_rng(4)
    dims = [4, 5, 3]
    params = mlp.init_params(dims, rng)
    x, t = rng.normal(size=(8, 4)), rng.normal(size=(8, 3))
    _, grads = mlp.loss_and_grads(params, x, t)
    new = mlp.adam_step(params, grads, {}, lr=1e-3, eps=1e-12)
    step = mlp.flatten(params) - mlp.flatten(new)
    g = mlp.flatten(grads)
    nz = np.abs(g) > 1e-9
    np.testing.assert_allclose(step[nz], 1e-3 * np.sign(g[nz]), rtol=1e-6)


def test_adam_fits_a_linear_model_to_the_least_squares_solution():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(64, 3))
    t = x @ rng.normal(size=(3, 2)) + rng.normal(size=2) + 0.1 * rng.normal(size=(64, 2))
    params = [(np.zeros((2, 3)), np.zeros(2))]
    state = {}
    for k in range(4000):
        _, g = mlp.loss_and_grads(params, x, t)
        params = mlp.adam_step(params, g, state, lr=0.02 if k < 3000 else 0.002)
    X1 = np.hstack([x, np.ones((64, 1))])
    sol, *_ = np.linalg.lstsq(X1, t, rcond=None)
    np.testing.assert_allclose(params[0][0], sol[:3].T, atol=2e-4)
    np.testing.assert_allclose(params[0][1], sol[3], atol=2e-4)


def test_bf16_mode_stays_within_bf16_accuracy_of_fp64():
    rng = np.random.default_rng(6)
    dims = [16, 32, 32, 8]
    params = mlp.init_params(dims, rng)
    x = rng.normal(size=(20, 16))
    y64, _ = mlp.forward(params, x)
    y16, _ = mlp.forward(params, x, bf16=True)
    rel = np.linalg.norm(y16 - y64) / np.linalg.norm(y64)
    assert 1e-5 < rel < 2e-2
