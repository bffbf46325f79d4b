"""The diagonal preconditioner scale on top of Jacobi (S D^-1 from the left): the row
norms and the closed-form wall scale against the oracle, and scaled solves that keep
the oracle's solution and true residual."""
import numpy as np
import pytest

import scenes
from oracle import operator as oop, solvers as osv
from sph_testutil import gpu_solve, lib_build, oracle_system, params_for, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

CASES = {
    "couette_dummy": lambda: scenes.couette(0),
    "couette_dynamic": lambda: scenes.couette(1, boundary=scenes.BC_DYNAMIC),
    "lava_box_12": lambda: scenes.lava_box(2, n=12),
    "slope_papanastasiou": lambda: scenes.slope_subset(4, nx=12, ny=8, nz=12),
}


def _dev_f32(torch, n):
    return torch.empty(n, dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("name", sorted(CASES))
def test_row_norms_and_wall_scale_match_oracle(name):
    torch = torch_cuda()
    s = CASES[name]()
    nb, _ = lib_build(s)
    _, _, A = oracle_system(s)
    out = _dev_f32(torch, s.n)
    nb.row_norms(params_for(s), out)
    want = oop.row_norms2(A)
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=2e-6)
    for factor, power in ((1.0, 0.0), (1.0, 3.0), (0.125, 0.0), (0.5, 2.0)):
        nb.wall_row_scale(params_for(s), factor, power, out)
        np.testing.assert_allclose(out.cpu().numpy(), oop.wall_row_scale(s, A, power, factor), rtol=2e-5)
    nb.close()


def test_unit_scale_leaves_the_solve_bit_identical():
    """s = 1 multiplies every row's invD by 1.0f: the iterates, and the result, are
    those of the solve without a scale, bit for bit."""
    torch = torch_cuda()
    s = scenes.lava_box(2, n=12)
    nb, _ = lib_build(s)
    x0, rep0 = gpu_solve(nb, s)
    nb.set_row_scale(torch.ones(s.n, dtype=torch.float32, device="cuda"))
    x1, rep1 = gpu_solve(nb, s)
    assert rep0["iters"] == rep1["iters"] and rep0["refinements"] == rep1["refinements"]
    np.testing.assert_array_equal(x0, x1)
    nb.set_row_scale(None)
    x2, _ = gpu_solve(nb, s)
    np.testing.assert_array_equal(x0, x2)
    nb.close()


@pytest.mark.parametrize("name", ["lava_box_12", "couette_dummy", "slope_papanastasiou"])
def test_wall_scaled_solve_keeps_the_oracle_solution(name):
    """The scaled system has the solution of A x = b: the 1e-6 solve passes the
    oracle's residual and a 1e-8 solve lies within 1e-5 of the oracle's solution."""
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = CASES[name]()
    nb, _ = lib_build(s)
    _, _, A = oracle_system(s)
    sc = _dev_f32(torch, s.n)
    nb.wall_row_scale(params_for(s), 1.0, 3.0, sc)
    nb.set_row_scale(sc)
    x, rep = gpu_solve(nb, s)
    assert rep["status"] == 0, rep
    res, _ = oop.true_residual(A, x, s.b)
    assert res <= 1e-6
    x8, rep8 = gpu_solve(nb, s, binding.solve_opts(rtol=1e-8))
    assert rep8["status"] == 0
    assert rel_l2(x8, osv.reference_solution(A, s.b, s.x0)) <= 1e-5
    nb.close()


@pytest.mark.parametrize("factor,power", [(1.0, 3.0), (0.125, 0.0)])
def test_wall_scale_cuts_iterations_on_a_box(factor, power):
    """On a stiff lava box weighting the wall rows down shortens the inner iteration
    (the float64 study: about a fifth fewer iterations with norm2^-3, about a third with
    a constant 1/8, at 15k-90k rows)."""
    torch = torch_cuda()
    s = scenes.lava_box(5, n=24)
    nb, _ = lib_build(s)
    _, rep0 = gpu_solve(nb, s)
    sc = _dev_f32(torch, s.n)
    nb.wall_row_scale(params_for(s), factor, power, sc)
    nb.set_row_scale(sc)
    _, rep1 = gpu_solve(nb, s)
    assert rep0["status"] == 0 and rep1["status"] == 0
    assert rep1["iters"] < 0.95 * rep0["iters"], (rep0["iters"], rep1["iters"])
    nb.close()


def test_scale_follows_an_operator_rebuild_and_the_cg():
    """The scale stays with the handle when dt changes (the scaled diagonals are
    rebuilt for the new operator), and the conjugate gradient takes it too (dynamic
    walls: S D^-1 stays symmetric positive definite as a preconditioner)."""
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = scenes.couette(1, boundary=scenes.BC_DYNAMIC)
    nb, _ = lib_build(s)
    sc = torch.from_numpy(np.random.default_rng(3).uniform(0.5, 2.0, s.n).astype(np.float32)).cuda()
    nb.set_row_scale(sc)
    for dt in (s.dt, 3 * s.dt):
        s2 = s.copy()
        s2.dt = dt
        _, _, A = oracle_system(s2)
        for method in (binding.SPH_SOLVER_BICGSTAB, binding.SPH_SOLVER_CG):
            x, rep = gpu_solve(nb, s2, binding.solve_opts(method=method, rtol=1e-8))
            assert rep["status"] == 0, (dt, method, rep)
            assert rel_l2(x, osv.reference_solution(A, s2.b, s2.x0)) <= 1e-5
    nb.close()


def test_bad_scales_and_unsupported_solves_are_refused():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = scenes.couette(0)
    nb, _ = lib_build(s)
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        v = torch.ones(s.n, dtype=torch.float32, device="cuda")
        v[s.n // 2] = bad
        with pytest.raises(RuntimeError):
            nb.set_row_scale(v)
    nb.set_row_scale(torch.full((s.n,), 0.5, dtype=torch.float32, device="cuda"))
    with pytest.raises(RuntimeError):
        gpu_solve(nb, s, binding.solve_opts(precision=binding.SPH_PREC_FP64))
    for factor, power in ((1.0, -1.0), (0.0, 1.0), (float("nan"), 0.0)):
        with pytest.raises(RuntimeError):
            nb.wall_row_scale(params_for(s), factor, power, torch.empty(s.n, dtype=torch.float32, device="cuda"))
    nb.set_row_scale(None)
    x, rep = gpu_solve(nb, s, binding.solve_opts(precision=binding.SPH_PREC_FP64))
    assert rep["status"] == 0
    nb.close()


def test_batched_solve_takes_each_scenes_scale():
    """The batched solve with the wall scale on some scenes: each scene reaches the
    oracle's residual and solution; changing a scale after the batch was made is
    refused."""
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    ss = [scenes.lava_box(2, n=12), scenes.couette(0), scenes.lava_box(7, n=10)]
    nbs, bs, xs, As = [], [], [], []
    for k, s in enumerate(ss):
        nb, _ = lib_build(s)
        if k != 1:
            sc = _dev_f32(torch, s.n)
            nb.wall_row_scale(params_for(s), 1.0, 3.0, sc)
            nb.set_row_scale(sc)
        nbs.append(nb)
        bs.append(torch.from_numpy(s.b).cuda())
        xs.append(torch.from_numpy(s.x0).cuda())
        As.append(oracle_system(s)[2])
    batch = binding.Batch(nbs, [params_for(s) for s in ss])
    st, reps = batch.solve(binding.solve_opts(rtol=1e-8), bs, xs)
    assert st == 0
    for k, s in enumerate(ss):
        x = xs[k].cpu().numpy()
        assert oop.true_residual(As[k], x, s.b)[0] <= 1e-8 * 1.01
        assert rel_l2(x, osv.reference_solution(As[k], s.b, s.x0)) <= 1e-5
    nbs[1].set_row_scale(torch.ones(ss[1].n, dtype=torch.float32, device="cuda"))
    with pytest.raises(RuntimeError):
        batch.solve(binding.solve_opts(), bs, xs)
    batch.close()
    for nb in nbs:
        nb.close()


def test_scale_targets_match_the_oracle_closed_form():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = scenes.lava_box(3, n=10)
    nb, _ = lib_build(s)
    _, _, A = oracle_system(s)
    tgt = torch.empty((s.n, 4), dtype=torch.float32, device="cuda")
    mask = torch.empty(s.n, dtype=torch.uint8, device="cuda")
    for factor, power in ((1.0, 4.0), (0.125, 0.0), (0.25, 1.5)):
        binding.mlp_scale_targets(nb, params_for(s), factor, power, tgt, mask)
        t = tgt.cpu().numpy()
        np.testing.assert_allclose(t[:, 0], np.log(oop.wall_row_scale(s, A, power, factor)), rtol=0, atol=2e-5)
    np.testing.assert_array_equal(t[:, 1:], 0.0)
    np.testing.assert_array_equal(mask.cpu().numpy(), (s.ptype != scenes.FLUID).astype(np.uint8))
    nb.close()


def _scale_net():
    import os

    from paper_2206_14780_gb300 import binding

    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2206_14780_gb300",
                        "weights", "scale_head_mlp.npz")
    z = np.load(path)
    return binding.Mlp(z["params"]), z["params"]


def test_learned_scale_is_the_networks_first_output_on_wall_rows():
    """sph_mlp_row_scale = exp(y_0) of the network on the handle's features on wall
    rows, 1 on fluid rows; and against the oracle's float64 features and network with
    the same bf16 rounding points (feature roundings may flip, so loosely)."""
    torch = torch_cuda()
    from oracle import features as ofeat, mlp as omlp, neighbors as onb
    from paper_2206_14780_gb300 import binding

    net, theta = _scale_net()
    s = scenes.lava_box(4, n=12)
    nb, _ = lib_build(s)
    p = params_for(s)
    vel = torch.from_numpy(s.vel).cuda()
    sc = torch.empty(s.n, dtype=torch.float32, device="cuda")
    binding.mlp_row_scale(nb, p, net, vel, sc)
    f = torch.empty((s.n, 16), dtype=torch.int16, device="cuda")
    binding.mlp_features(nb, p, vel, f)
    y = torch.empty((s.n, 4), dtype=torch.float32, device="cuda")
    net.forward(f, y)
    wall = s.ptype != scenes.FLUID
    got = sc.cpu().numpy()
    np.testing.assert_array_equal(got[~wall], 1.0)
    want = np.exp(np.clip(y.cpu().numpy()[:, 0].astype(np.float64), -8.0, 2.0))
    np.testing.assert_allclose(got[wall], want[wall], rtol=1e-6)
    off, idx = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    Fr, _ = ofeat.features(s, off, idx, oop.assemble(s, off, idx))
    yr, _ = omlp.forward(omlp.unflatten(theta.astype(np.float64)), omlp.bf16_round(Fr), bf16=True)
    d = np.abs(np.log(got[wall]) - np.clip(yr[wall, 0], -8.0, 2.0))
    assert np.median(d) <= 0.01 and d.max() <= 0.15, (np.median(d), d.max())
    nb.close()


def test_learned_scale_cuts_iterations_on_an_unseen_full_size_box():
    """The committed head on a 1.16M-particle lava box it never saw (seed 11): fewer
    iterations than Jacobi alone and than the closed-form norm2^-3 scale, from the same
    start (v^n with the wall closure); installing the scale directly (no output array)
    gives the same solve bit for bit."""
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    net, _ = _scale_net()
    s = scenes.lava_box(11, n=100)
    t = binding.scene_tensors(s, torch.device("cuda", 0))
    vel = torch.from_numpy(s.vel).cuda()
    nb = binding.build_neighbors(t["pos"], t["rho"], t["mu"], t["ptype"], s.lo, s.hi, s.periodic, s.h)
    p = params_for(s)
    b = torch.from_numpy(s.b).cuda()
    its, xs = {}, {}
    for name in ("jacobi", "wall_p3", "learned", "learned_installed"):
        sc = torch.empty(s.n, dtype=torch.float32, device="cuda")
        if name == "jacobi":
            nb.set_row_scale(None)
        elif name == "wall_p3":
            nb.wall_row_scale(p, 1.0, 3.0, sc)
            nb.set_row_scale(sc)
        elif name == "learned":
            binding.mlp_row_scale(nb, p, net, vel, sc)
            nb.set_row_scale(sc)
        else:
            nb.set_row_scale(None)
            binding.mlp_row_scale(nb, p, net, vel, None)
        x = torch.empty_like(b)
        binding.warm_start(nb, p, None, vel, t["ptype"], b, x)
        rep = nb.solve(p, binding.solve_opts(), b, x)
        assert rep["status"] == 0 and rep["true_rel_res"] <= 1e-6
        its[name] = rep["iters"]
        xs[name] = x
    assert its["learned"] < 0.8 * its["jacobi"] and its["learned"] < its["wall_p3"], its
    assert its["learned_installed"] == its["learned"] and torch.equal(xs["learned_installed"], xs["learned"])
    nb.close()


def test_rebuild_keeps_the_scale_for_the_same_particles_and_drops_it_otherwise():
    """A neighbour rebuild of the same particles (moved) keeps the caller-order scale and
    the solve still meets the oracle; a rebuild with another particle count clears it
    (the float64 solve, which refuses a scaled handle, then runs)."""
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = scenes.lava_box(2, n=10)
    nb, t = lib_build(s)
    sc = _dev_f32(torch, s.n)
    nb.wall_row_scale(params_for(s), 0.125, 0.0, sc)
    nb.set_row_scale(sc)
    s2 = s.copy()
    s2.pos = s.pos.copy()
    s2.pos[s2.ptype == scenes.FLUID, :3] += np.float32(0.05 * s.dx)   # fluid shifted, same particles
    pos2 = torch.from_numpy(s2.pos).cuda()
    nb.rebuild(pos2, t["rho"], t["mu"], t["ptype"], s2.lo, s2.hi, s2.periodic, s2.h)
    with pytest.raises(RuntimeError):                   # still scaled
        gpu_solve(nb, s2, binding.solve_opts(precision=binding.SPH_PREC_FP64))
    _, _, A2 = oracle_system(s2)
    x, rep = gpu_solve(nb, s2, binding.solve_opts(rtol=1e-8))
    assert rep["status"] == 0 and rel_l2(x, osv.reference_solution(A2, s2.b, s2.x0)) <= 1e-5
    s3 = scenes.lava_box(3, n=9)
    t3 = binding.scene_tensors(s3, torch.device("cuda", 0))
    nb.rebuild(t3["pos"], t3["rho"], t3["mu"], t3["ptype"], s3.lo, s3.hi, s3.periodic, s3.h)
    x3, rep3 = gpu_solve(nb, s3, binding.solve_opts(precision=binding.SPH_PREC_FP64))
    assert rep3["status"] == 0
    nb.close()


def test_learned_scale_entry_points_take_either_kernel_and_refuse_bad_arguments():
    """The learned scale runs on a truncated-Gaussian handle too (its features use the
    handle's kernel): positive finite scales, 1 on fluid rows; the target builder checks
    factor and power like the closed form does."""
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    net, _ = _scale_net()
    g = scenes.lava_box(3, n=10, layers=4, kernel=scenes.KERNEL_GAUSSIAN)
    nb, t = lib_build(g, max_neighbors=512)
    sc = torch.empty(g.n, dtype=torch.float32, device="cuda")
    binding.mlp_row_scale(nb, params_for(g), net, torch.from_numpy(g.vel).cuda(), sc)
    v = sc.cpu().numpy()
    assert np.all(np.isfinite(v)) and np.all(v > 0)
    np.testing.assert_array_equal(v[g.ptype == scenes.FLUID], 1.0)
    nb.close()
    s = scenes.couette(0)
    nb, _ = lib_build(s)
    tgt = torch.empty((s.n, 4), dtype=torch.float32, device="cuda")
    mask = torch.empty(s.n, dtype=torch.uint8, device="cuda")
    for factor, power in ((0.0, 1.0), (1.0, 65.0), (float("inf"), 0.0)):
        with pytest.raises(RuntimeError):
            binding.mlp_scale_targets(nb, params_for(s), factor, power, tgt, mask)
    nb.close()
