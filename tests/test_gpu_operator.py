"""GPU operator apply and float64 residual against the oracle's assembled A(dt)."""
import numpy as np
import pytest

from oracle import operator as oop
from sph_testutil import SCENES_SMALL, lib_build, oracle_system, params_for, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

APPLY_RTOL = 1e-5   # relative L2 of the float32 apply (its error bound is ~ a few float32 ulps)


@pytest.mark.parametrize("name", sorted(SCENES_SMALL))
def test_apply_matches_oracle(name):
    torch = torch_cuda()
    s = SCENES_SMALL[name]()
    nb, _ = lib_build(s)
    off, idx, A = oracle_system(s)
    rng = np.random.default_rng(7)
    for v_np in (rng.normal(size=(s.n, 3)), s.x0, np.ones((s.n, 3))):
        v = np.zeros((s.n, 4), np.float32)
        v[:, :3] = v_np
        vt = torch.from_numpy(v).cuda()
        yt = torch.empty_like(vt)
        nb.apply(params_for(s), vt, yt)
        y = yt.cpu().numpy()[:, :3]
        ref = A @ v[:, :3].astype(np.float64)
        assert rel_l2(y, ref) < APPLY_RTOL, rel_l2(y, ref)


@pytest.mark.parametrize("name", sorted(SCENES_SMALL))
def test_apply_otf_matches_oracle(name):
    """The on-the-fly form (coefficients recomputed per pair in float32) gives the same
    A v as the assembled float64 matrix, within the float32 apply tolerance."""
    torch = torch_cuda()
    s = SCENES_SMALL[name]()
    nb, _ = lib_build(s)
    off, idx, A = oracle_system(s)
    rng = np.random.default_rng(8)
    for v_np in (rng.normal(size=(s.n, 3)), s.x0, np.ones((s.n, 3))):
        v = np.zeros((s.n, 4), np.float32)
        v[:, :3] = v_np
        vt = torch.from_numpy(v).cuda()
        yt = torch.empty_like(vt)
        nb.apply_otf(params_for(s), vt, yt)
        y = yt.cpu().numpy()
        ref = A @ v[:, :3].astype(np.float64)
        assert rel_l2(y[:, :3], ref) < APPLY_RTOL, rel_l2(y[:, :3], ref)
        np.testing.assert_array_equal(y[:, 3], 0.0)


def test_apply_otf_follows_dt_and_viscosity():
    torch = torch_cuda()
    s = SCENES_SMALL["random_box_mu_mass"]()
    nb, t = lib_build(s)
    v = np.zeros((s.n, 4), np.float32)
    v[:, :3] = np.random.default_rng(2).normal(size=(s.n, 3))
    vt = torch.from_numpy(v).cuda()
    yt = torch.empty_like(vt)
    off, idx, _ = oracle_system(s)
    for dt, scale in ((1e-4, 1.0), (3e-4, 1.0), (3e-4, 7.0)):
        mu = (np.asarray(s.mu, np.float32) * np.float32(scale)).astype(np.float32)
        nb.set_viscosity(torch.from_numpy(mu).cuda())
        A = oop.assemble(s, off, idx, dt=dt, mu=mu)
        nb.apply_otf(params_for(s, dt), vt, yt)
        ref = A @ v[:, :3].astype(np.float64)
        assert rel_l2(yt.cpu().numpy()[:, :3], ref) < APPLY_RTOL


@pytest.mark.parametrize("name", ["couette_dummy", "random_box_mu_mass", "lava_box_12"])
def test_residual_f64_matches_oracle(name):
    torch = torch_cuda()
    s = SCENES_SMALL[name]()
    nb, _ = lib_build(s)
    off, idx, A = oracle_system(s)
    rng = np.random.default_rng(3)
    x = rng.normal(size=(s.n, 3))
    xt = torch.from_numpy(x).cuda()
    bt = torch.from_numpy(s.b).cuda()
    rt = torch.empty_like(xt)
    nb.residual(params_for(s), xt, bt, rt)
    r = rt.cpu().numpy()
    ref = s.b - A @ x
    scale = np.linalg.norm(s.b) + np.linalg.norm(abs(A) @ abs(x))
    assert np.linalg.norm(r - ref) < 1e-12 * scale


def test_dt_change_recomputes_coefficients():
    torch = torch_cuda()
    s = SCENES_SMALL["couette_dummy"]()
    nb, _ = lib_build(s)
    v = np.zeros((s.n, 4), np.float32)
    v[:, :3] = np.random.default_rng(1).normal(size=(s.n, 3))
    vt = torch.from_numpy(v).cuda()
    yt = torch.empty_like(vt)
    for dt in (1e-4, 3e-4):
        off, idx, A = oracle_system(s)
        A = oop.assemble(s, off, idx, dt=dt)
        nb.apply(params_for(s, dt), vt, yt)
        assert rel_l2(yt.cpu().numpy()[:, :3], A @ v[:, :3].astype(np.float64)) < APPLY_RTOL
