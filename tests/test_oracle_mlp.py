"""Pins of the warm-start network reference (oracle/mlp.py): finite differences, bf16 rounding."""
import numpy as np
import pytest

from oracle import mlp


def test_parameter_count():
    assert mlp.N_PARAMS == 9603
    p = mlp.init_params(1)
    np.testing.assert_array_equal(mlp.flatten(mlp.unflatten(mlp.flatten(p))), mlp.flatten(p))


def test_bf16_round_matches_library_conversion():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).normal(scale=3.0, size=10000)
    x = np.concatenate([x, [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0, 1e-30]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), ref)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    p = mlp.init_params(2)
    p["W4"] = p["W4"] * 10.0
    for k in ("b1", "b2", "b3", "b4"):
        p[k] = rng.normal(scale=0.1, size=p[k].shape)
    X = rng.normal(size=(40, 16))
    T = rng.normal(size=(40, 3))
    mask = rng.random(40) < 0.8
    loss, g, _ = mlp.loss_and_grad(p, X, T, mask)
    theta = mlp.flatten(p)
    gflat = mlp.flatten(g)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        lp, _, _ = mlp.loss_and_grad(mlp.unflatten(tp), X, T, mask)
        lm, _, _ = mlp.loss_and_grad(mlp.unflatten(tm), X, T, mask)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gflat[i])


def test_silu_derivative():
    z = np.linspace(-6, 6, 101)
    e = 1e-6
    np.testing.assert_allclose(mlp.dsilu(z), (mlp.silu(z + e) - mlp.silu(z - e)) / (2 * e), rtol=1e-7, atol=1e-9)
