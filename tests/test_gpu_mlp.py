"""Warm-start network on tensor cores against the float64 oracle (same bf16 rounding points)."""
import numpy as np
import pytest

import scenes
from oracle import features as ofeat, mlp as omlp, neighbors as onb, operator as oop
from sph_testutil import lib_build, params_for, torch_cuda

pytestmark = pytest.mark.gpu


def _problem(m=777, seed=0):
    rng = np.random.default_rng(seed)
    p = omlp.init_params(seed)
    p["W4"] = p["W4"] * 10.0
    for k in ("b1", "b2", "b3", "b4"):
        p[k] = rng.normal(scale=0.1, size=p[k].shape)
    X = omlp.bf16_round(rng.normal(size=(m, 16)))
    T = rng.normal(size=(m, 3))
    mask = (rng.random(m) < 0.85).astype(np.uint8)
    return p, X, T, mask


def _dev(torch, X, T, mask):
    xb = torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).cuda().view(torch.int16).contiguous()
    t4 = np.zeros((len(T), 4), np.float32)
    t4[:, :3] = T
    return xb, torch.from_numpy(t4).cuda(), torch.from_numpy(mask).cuda()


def test_forward_matches_oracle():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    p, X, T, mask = _problem()
    net = binding.Mlp(omlp.flatten(p).astype(np.float32))
    xb, _, _ = _dev(torch, X, T, mask)
    out = torch.empty((len(X), 4), dtype=torch.float32, device="cuda")
    net.forward(xb, out)
    y = out.cpu().numpy()
    p32 = omlp.unflatten(omlp.flatten(p).astype(np.float32).astype(np.float64))
    ref, _ = omlp.forward(p32, X, bf16=True)
    # the same bf16 rounding points as the oracle: what differs is the float32 accumulation
    # order before each rounding, which flips an occasional activation by one bf16 ulp
    assert np.linalg.norm(y[:, :3] - ref) <= 2e-3 * np.linalg.norm(ref)
    np.testing.assert_array_equal(y[:, 3], 0.0)


def test_gradient_matches_oracle():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    p, X, T, mask = _problem(seed=1)
    theta = omlp.flatten(p).astype(np.float32)
    net = binding.Mlp(theta)
    xb, tt, mk = _dev(torch, X, T, mask)
    g = torch.empty(binding.MLP_NPARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    net.grad(xb, tt, mk, int(mask.sum()), g, loss)
    torch.cuda.synchronize()
    p32 = omlp.unflatten(theta.astype(np.float64))
    l_ref, g_ref, _ = omlp.loss_and_grad(p32, X, T, mask, bf16=True)
    g_ref = omlp.flatten(g_ref)
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - l_ref) <= 1e-4 * l_ref
    assert np.linalg.norm(gg - g_ref) <= 1e-3 * np.linalg.norm(g_ref)
    # every parameter block is exercised (a transposed fragment would scramble one of them)
    off = 0
    for name, shp in omlp.SHAPES:
        k = int(np.prod(shp))
        blk, ref = gg[off:off + k], g_ref[off:off + k]
        assert np.linalg.norm(blk - ref) <= 2e-3 * np.linalg.norm(ref) + 1e-7, name
        off += k


@pytest.mark.parametrize("m", [128, 129, 152 * 128 * 3 + 77])
def test_gradient_over_many_tiles_matches_oracle_and_repeats_exactly(m):
    """One 128-row tile, a tile plus one row, and more tiles than SMs (each CTA then
    accumulates several tiles' weight gradients in tensor memory): the gradient
    matches the oracle's, and a second call returns the same bits (fixed summation
    order)."""
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    p, X, T, mask = _problem(m=m, seed=3)
    theta = omlp.flatten(p).astype(np.float32)
    net = binding.Mlp(theta)
    xb, tt, mk = _dev(torch, X, T, mask)
    g = torch.empty(binding.MLP_NPARAMS, dtype=torch.float32, device="cuda")
    g2 = torch.empty_like(g)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    net.grad(xb, tt, mk, int(mask.sum()), g, loss)
    net.grad(xb, tt, mk, int(mask.sum()), g2, loss)
    torch.cuda.synchronize()
    assert torch.equal(g, g2)
    l_ref, g_ref, _ = omlp.loss_and_grad(omlp.unflatten(theta.astype(np.float64)), X, T, mask, bf16=True)
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - l_ref) <= 1e-4 * l_ref
    off = 0
    for name, shp in omlp.SHAPES:
        k = int(np.prod(shp))
        blk, ref = gg[off:off + k], omlp.flatten(g_ref)[off:off + k]
        assert np.linalg.norm(blk - ref) <= 2e-3 * np.linalg.norm(ref) + 1e-7, name
        off += k
    net.close()


def test_training_reduces_loss():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    rng = np.random.default_rng(4)
    teacher = omlp.init_params(9)
    teacher["W4"] = teacher["W4"] * 10.0
    X = omlp.bf16_round(rng.normal(size=(4096, 16)))
    T, _ = omlp.forward(teacher, X)
    net = binding.Mlp(omlp.flatten(omlp.init_params(10)).astype(np.float32))
    xb, tt, mk = _dev(torch, X, T, np.ones(len(X), np.uint8))
    losses = [net.train_step(xb, tt, mk, len(X), 3e-3) for _ in range(400)]
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])
    assert np.all(np.isfinite(net.params()))


@pytest.mark.parametrize("make", [lambda: scenes.couette(2), lambda: scenes.lava_box(3, n=10),
                                  lambda: scenes.slope_subset(1, nx=12, ny=8, nz=12),
                                  lambda: scenes.lava_box(4, n=10, layers=4, kernel=scenes.KERNEL_GAUSSIAN)])
def test_features_match_oracle(make):
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = make()
    nb, t = lib_build(s, max_neighbors=512 if s.kernel == scenes.KERNEL_GAUSSIAN else 128)
    vel = torch.from_numpy(s.vel).cuda()
    f = torch.empty((s.n, 16), dtype=torch.int16, device="cuda")
    U = binding.mlp_features(nb, params_for(s), vel, f)
    F = f.view(torch.bfloat16).float().cpu().numpy().astype(np.float64)
    off, idx = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h, kernel_id=s.kernel)
    A = oop.assemble(s, off, idx)
    Fr, Ur = ofeat.features(s, off, idx, A)
    assert abs(U - Ur) <= 1e-6 * Ur
    err = np.abs(F - Fr) / np.maximum(1.0, np.abs(Fr))
    assert err.max() <= 1e-2, (np.unravel_index(err.argmax(), err.shape), err.max())
