"""sph_visc_apply_noalloc: the allocation-free apply agrees with sph_visc_apply.

Collected last on purpose (file name), so a failure here never hides another test.
Callers that cannot allocate device memory at call time (a plugin inside a
framework that owns the device memory pool, or a loop that forbids allocation)
use this entry point after setting the coefficients up once.
"""
import numpy as np
import pytest

import scenes
from sph_testutil import lib_build, params_for, torch_cuda

pytestmark = pytest.mark.gpu


def _vec(torch, n, seed):
    v = np.zeros((n, 4), np.float32)
    v[:, :3] = np.random.default_rng(seed).normal(size=(n, 3))
    return torch.from_numpy(v).cuda()


def test_noalloc_apply_matches_apply_on_two_calls():
    torch = torch_cuda()
    s = scenes.couette(3)
    nb, _ = lib_build(s)
    p = params_for(s)
    nb.setup(p)
    for seed in (11, 12):        # two calls in a row: the second must not see the first's data
        v = _vec(torch, s.n, seed)
        y_ref = torch.empty_like(v)
        y_na = torch.full_like(v, float("nan"))
        nb.apply(p, v, y_ref)
        nb.apply_noalloc(p, v, y_na)
        torch.cuda.synchronize()
        ref = y_ref.cpu().numpy()[:, :3].astype(np.float64)
        got = y_na.cpu().numpy()[:, :3].astype(np.float64)
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_noalloc_apply_matches_the_oracle_and_leaves_device_memory_unchanged():
    """Against the oracle's assembled A(dt) (float64), on two calls in a row; the
    device's free memory is the same before and after the calls (the scratch is
    the library's static array, present since the library loaded)."""
    torch = torch_cuda()
    from oracle import operator as oop
    from sph_testutil import oracle_system

    s = scenes.lava_box(5, n=12)
    nb, _ = lib_build(s)
    p = params_for(s)
    nb.setup(p)
    off, idx, A = oracle_system(s)
    v0 = _vec(torch, s.n, 21)
    y0 = torch.empty_like(v0)
    nb.apply_noalloc(p, v0, y0)                    # first call: the symbol address look-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for seed in (22, 23):
        v = _vec(torch, s.n, seed)
        y = torch.full_like(v, float("nan"))
        nb.apply_noalloc(p, v, y)
        torch.cuda.synchronize()
        ref = A @ v.cpu().numpy()[:, :3].astype(np.float64)
        got = y.cpu().numpy()[:, :3].astype(np.float64)
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_apply_rejects_overlapping_buffers():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = scenes.couette(5)
    nb, _ = lib_build(s)
    p = params_for(s)
    nb.setup(p)
    buf = torch.zeros((s.n + 1, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(binding.SphError) as e:       # y starts one row after v: the ranges overlap
        nb.apply_noalloc(p, buf[:s.n], buf[1:])
    assert e.value.status == 1


def test_noalloc_apply_rejects_missing_setup_and_oversize():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = scenes.couette(4)
    nb, _ = lib_build(s)
    v = _vec(torch, s.n, 1)
    y = torch.empty_like(v)
    with pytest.raises(binding.SphError) as e:       # coefficients never set up
        nb.apply_noalloc(params_for(s), v, y)
    assert e.value.status == 1
    big = scenes.periodic_lattice(66)                 # 287,496 rows > SPH_NOALLOC_MAX_ROWS
    assert big.n > binding.SPH_NOALLOC_MAX_ROWS
    nbb, _ = lib_build(big)
    pb = params_for(big)
    nbb.setup(pb)
    vb = _vec(torch, big.n, 2)
    with pytest.raises(binding.SphError) as e:
        nbb.apply_noalloc(pb, vb, torch.empty_like(vb))
    assert e.value.status == 1
