"""The truncated Gaussian kernel (paper Sec. 5.2, support radius 3h, ~250 neighbours at
h = 1.3 dx) through the GPU path: neighbour lists, A(dt), the solve and the
Papanastasiou pass against the oracle evaluated with the same kernel."""
import numpy as np
import pytest

import scenes
from oracle import neighbors as onb, operator as oop, rheology, solvers as osv
from sph_testutil import gpu_solve, lib_build, oracle_system, params_for, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

G = scenes.KERNEL_GAUSSIAN
MAXNB = 512

GAUSS_SCENES = {
    "periodic_lattice_jitter": lambda: scenes.periodic_lattice(12, jitter=0.1, mu_spread=4.0, seed=5, kernel=G),
    "random_box": lambda: scenes.random_box(9, nf=1800, mu_spread=3.0, kernel=G),
    "lava_box_10_4layers": lambda: scenes.lava_box(6, n=10, layers=4, kernel=G),
    "lava_box_10_dynamic": lambda: scenes.lava_box(7, n=10, layers=4, kernel=G, boundary=scenes.BC_DYNAMIC),
}


@pytest.mark.parametrize("name", sorted(GAUSS_SCENES))
def test_gaussian_lists_equal_oracle(name):
    s = GAUSS_SCENES[name]()
    nb, _ = lib_build(s, max_neighbors=MAXNB)
    off, idx = nb.export()
    off_o, idx_o = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h, kernel_id=G)
    np.testing.assert_array_equal(off.cpu().numpy(), off_o)
    np.testing.assert_array_equal(idx.cpu().numpy(), idx_o)
    assert np.diff(off_o).max() > 200


@pytest.mark.parametrize("name", sorted(GAUSS_SCENES))
def test_gaussian_apply_and_solve_match_oracle(name):
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = GAUSS_SCENES[name]()
    nb, _ = lib_build(s, max_neighbors=MAXNB)
    off, idx, A = oracle_system(s)
    rng = np.random.default_rng(3)
    for v_np in (rng.normal(size=(s.n, 3)), np.ones((s.n, 3))):
        v = np.zeros((s.n, 4), np.float32)
        v[:, :3] = v_np
        vt = torch.from_numpy(v).cuda()
        yt = torch.empty_like(vt)
        nb.apply(params_for(s), vt, yt)
        assert rel_l2(yt.cpu().numpy()[:, :3], A @ v[:, :3].astype(np.float64)) < 1e-5
    x, rep = gpu_solve(nb, s)
    assert rep["status"] == 0, rep
    assert oop.true_residual(A, x, s.b)[0] <= 1e-6
    x7, rep7 = gpu_solve(nb, s, binding.solve_opts(rtol=1e-7))
    assert rep7["status"] == 0 and rel_l2(x7, osv.reference_solution(A, s.b, s.x0)) <= 1e-5
    if s.boundary == scenes.BC_DYNAMIC:                 # the rotated CG with the wider kernel
        xc, repc = gpu_solve(nb, s, binding.solve_opts(method=binding.SPH_SOLVER_CG))
        assert repc["status"] == 0 and oop.true_residual(A, xc, s.b)[0] <= 1e-6


def test_gaussian_mu_pass_matches_oracle():
    torch = torch_cuda()
    s = scenes.slope_subset(2, nx=20, ny=12, nz=20).copy()
    s.kernel = G
    nb, _ = lib_build(s, max_neighbors=MAXNB)
    off, idx = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h, kernel_id=G)
    mu_ref, D = rheology.mu_pass(s, off, idx)
    vel = torch.from_numpy(s.vel).cuda()
    wv = torch.from_numpy(s.wall_vel).cuda()
    out = torch.empty(s.n, dtype=torch.float32, device="cuda")
    tau0, mu0, m = s.rheology
    nb.mu_papanastasiou(vel, wv, tau0, mu0, m, out, set_handle=True)
    fl = s.ptype == scenes.FLUID
    err = np.abs(out.cpu().numpy().astype(np.float64)[fl] - mu_ref[fl]) / mu_ref[fl]
    assert err.max() < 1e-4, err.max()


def test_gaussian_rejections_and_capacity():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = GAUSS_SCENES["random_box"]()
    with pytest.raises(binding.SphError) as e:           # ~250 neighbours do not fit 128
        lib_build(s, max_neighbors=128)
    assert e.value.status == 3
    nb, t = lib_build(s, max_neighbors=MAXNB)
    v = torch.zeros((s.n, 4), dtype=torch.float32, device="cuda")
    y = torch.empty_like(v)
    with pytest.raises(binding.SphError):
        nb.apply_otf(params_for(s), v, y)
    # the warm-start network takes Wendland scenes only (its features run on either kernel)
    import numpy as np

    net = binding.Mlp(np.zeros(binding.MLP_NPARAMS, np.float32))
    b = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    x0 = torch.empty_like(b)
    with pytest.raises(binding.SphError):
        binding.warm_start(nb, params_for(s), net, v, t["ptype"], b, x0)
    feats = torch.empty((s.n, 16), dtype=torch.int16, device="cuda")
    binding.mlp_features(nb, params_for(s), v, feats)
    net.close()
