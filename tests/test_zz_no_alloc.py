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
