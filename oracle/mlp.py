"""Per-particle MLP of the learned warm start, float64 reference (test infrastructure only).

Network: 16 -> 64 -> 64 -> 64 -> 3 with SiLU (x sigmoid(x)) on the hidden layers
and a linear output; 9,603 parameters:
    W1 [64,16] b1 [64]  W2 [64,64] b2 [64]  W3 [64,64] b3 [64]  W4 [3,64] b4 [3]
Loss: mean over the masked rows of |y - t|^2 (sum over the 3 outputs).

The GPU computes with bfloat16 operands and float32 accumulation: it rounds the
inputs, the weights and each hidden activation (post-SiLU) to bfloat16 before
they enter a product, and in the backward pass it rounds each backpropagated
gradient to bfloat16 before it enters a product.  ``forward``/``backward`` can
mimic those rounding points (``bf16=True``) so the comparison isolates
accumulation order; with ``bf16=False`` they are the exact float64 network,
pinned by finite differences.
"""
import numpy as np

SHAPES = [("W1", (64, 16)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 64)), ("b3", (64,)),
          ("W4", (3, 64)), ("b4", (3,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16_round(x):
    """Round float64 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def unflatten(theta):
    theta = np.asarray(theta, np.float64)
    out, k = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[k:k + n].reshape(shp)
        k += n
    return out


def flatten(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def init_params(seed=0):
    """He-style uniform initialisation (biases zero)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            fan_in = shp[1]
            lim = np.sqrt(3.0 / fan_in)
            p[name] = rng.uniform(-lim, lim, size=shp)
        else:
            p[name] = np.zeros(shp)
    p["W4"] *= 0.1      # small output layer: the first warm start is close to v^n
    return p


def forward(p, X, bf16=False):
    """Returns y [n,3] and the cache (pre-activations z, inputs of each layer a)."""
    r = bf16_round if bf16 else (lambda v: np.asarray(v, np.float64))
    W = {k: r(v) if k.startswith("W") else np.asarray(v, np.float64) for k, v in p.items()}
    a0 = r(X)
    z1 = a0 @ W["W1"].T + p["b1"]
    a1 = r(silu(z1))
    z2 = a1 @ W["W2"].T + p["b2"]
    a2 = r(silu(z2))
    z3 = a2 @ W["W3"].T + p["b3"]
    a3 = r(silu(z3))
    y = a3 @ W["W4"].T + p["b4"]
    return y, dict(a0=a0, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3, a3=a3, W=W)


def loss_and_grad(p, X, T, mask=None, bf16=False):
    """MSE loss over masked rows and its gradient with respect to every parameter."""
    r = bf16_round if bf16 else (lambda v: np.asarray(v, np.float64))
    y, c = forward(p, X, bf16)
    m = np.ones(len(X)) if mask is None else np.asarray(mask, np.float64)
    cnt = max(m.sum(), 1.0)
    diff = (y - T) * m[:, None]
    loss = float((diff * diff).sum() / cnt)
    W = c["W"]
    d4 = 2.0 * diff / cnt                   # dL/dy
    g = {"W4": r(d4).T @ c["a3"], "b4": d4.sum(0)}
    da3 = r(d4) @ W["W4"]
    d3 = da3 * dsilu(c["z3"])
    g["W3"] = r(d3).T @ c["a2"]
    g["b3"] = d3.sum(0)
    da2 = r(d3) @ W["W3"]
    d2 = da2 * dsilu(c["z2"])
    g["W2"] = r(d2).T @ c["a1"]
    g["b2"] = d2.sum(0)
    da1 = r(d2) @ W["W2"]
    d1 = da1 * dsilu(c["z1"])
    g["W1"] = r(d1).T @ c["a0"]
    g["b1"] = d1.sum(0)
    return loss, g, y
