"""Pins of the warm-start network reference (oracle/mlp.py): finite differences, bf16 rounding,
a hand-wired network with closed-form activations."""
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


def test_forward_of_a_hand_wired_network():
    """A network wired by hand through one unit per layer, with pre-activations set to ln k
    where SiLU has the closed form silu(ln k) = ln k * k / (k + 1).  This pins the layer
    order, the orientation of each W (out x in), the bias of every layer, SiLU on the hidden
    layers only and the linear output, independently of the formula in the oracle."""
    p = {name: np.zeros(shp) for name, shp in mlp.SHAPES}
    ln3, ln7, ln15 = np.log(3.0), np.log(7.0), np.log(15.0)
    p["W1"][0, 5] = 1.0                        # hidden unit 0 reads input 5
    p["W2"][1, 0] = 2.0                        # unit 1 of layer 2 reads unit 0 of layer 1
    p["b2"][1] = ln7 - 2.0 * 0.75 * ln3
    p["W3"][2, 1] = 1.0
    p["b3"][2] = ln15 - 0.875 * ln7
    p["W4"][:, 2] = [1.0, 2.0, 3.0]
    p["b4"][:] = [0.5, -1.0, 2.0]
    X = np.random.default_rng(4).normal(size=(6, 16))
    X[:, 5] = ln3
    y, cache = mlp.forward(p, X)
    a3 = 15.0 / 16.0 * ln15
    want = np.array([a3 + 0.5, 2.0 * a3 - 1.0, 3.0 * a3 + 2.0])
    np.testing.assert_allclose(y, np.broadcast_to(want, y.shape), rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(cache["a1"][:, 0], 0.75 * ln3, rtol=1e-14)
    np.testing.assert_allclose(cache["a2"][:, 1], 0.875 * ln7, rtol=1e-14)
    # every other hidden unit has a zero pre-activation, and silu(0) = 0
    assert np.count_nonzero(cache["a1"]) == 6 and np.count_nonzero(cache["a3"]) == 6
