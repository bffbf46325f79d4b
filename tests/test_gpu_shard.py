"""One system solved over several sub-domains (paper Sec. 7 and Sec. 7.1) on the GPU.

sph_shard_* partitions a built system into slabs of cell layers with their own
operator rows, vectors and halos, exchanges p and r* before each apply and
reduces dots as per-layer partials summed in layer order.  The iterates must not
depend on the number of sub-domains (bit for bit), and the solution must meet the
oracle as the single-domain solve does."""
import numpy as np
import pytest

import scenes
from oracle import operator as oop, solvers as osv
from sph_testutil import SCENES_SMALL, gpu_solve, lib_build, oracle_system, params_for, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def layers_of(nb, s):
    from paper_2206_14780_gb300 import binding

    sh = binding.Shard(nb, params_for(s), 1)
    nl = sh.info()["layers"]
    sh.close()
    return nl


def shard_solve(nb, s, ranks, opts=None, b=None, x0=None, striped=True):
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    sh = binding.Shard(nb, params_for(s), ranks)
    sh.set_striping(striped)
    bt = torch.from_numpy(np.ascontiguousarray(s.b if b is None else b, np.float64)).cuda()
    xt = torch.from_numpy(np.ascontiguousarray(s.x0 if x0 is None else x0, np.float64)).cuda()
    rep = sh.solve(opts or binding.solve_opts(), bt, xt)
    torch.cuda.synchronize()
    info = sh.info()
    sh.close()
    return xt.cpu().numpy(), rep, info


SHARD_SCENES = {
    "lava_box_20": lambda: scenes.lava_box(4, n=20),                           # open box, stiff
    "couette_dummy": SCENES_SMALL["couette_dummy"],                            # periodic slab axis (wrap halo)
    "random_box_mu_mass": SCENES_SMALL["random_box_mu_mass"],
    "periodic_lattice": SCENES_SMALL["periodic_lattice"],                      # periodic on every axis
}


@pytest.mark.parametrize("name", sorted(SHARD_SCENES))
def test_iterates_do_not_depend_on_the_number_of_subdomains(name):
    s = SHARD_SCENES[name]()
    nb, _ = lib_build(s)
    runs = {}
    nl = layers_of(nb, s)
    for k in (1, 2, 3, 4):
        if k > nl:
            continue
        for striped in (True, False):
            x, rep, info = shard_solve(nb, s, k, striped=striped)
            assert rep["status"] == 0, (k, striped, rep)
            runs[(k, striped)] = (x, rep, info)
    x1, r1, i1 = runs[(1, True)]
    assert i1["halo"] == [0] and i1["exchanged"] == 0
    # striping (the exchange overlapped with the interior slices) changes no bit either
    for (k, striped), (x, rep, info) in runs.items():
        np.testing.assert_array_equal(x, x1, err_msg=f"{name}: {k} sub-domains, striped {striped}")
        assert rep["iters"] == r1["iters"] and rep["refinements"] == r1["refinements"]
        assert rep["true_rel_res"] == r1["true_rel_res"]
        if k > 1:
            assert all(h > 0 for h in info["halo"]) and info["exchanged"] == sum(info["halo"])
            assert all(o % 32 == 0 for o in info["owned"]) and sum(info["owned"]) >= s.n


@pytest.mark.parametrize("name", sorted(SHARD_SCENES))
@pytest.mark.parametrize("ranks", [2, 4])
def test_sharded_solution_matches_oracle(name, ranks):
    from paper_2206_14780_gb300 import binding

    s = SHARD_SCENES[name]()
    nb, _ = lib_build(s)
    off, idx, A = oracle_system(s)
    if ranks > layers_of(nb, s):
        pytest.skip("fewer cell layers than sub-domains")
    x, rep, info = shard_solve(nb, s, ranks)
    assert rep["status"] == 0, rep
    res, _ = oop.true_residual(A, x, s.b)
    assert res <= 1e-6, (res, rep)
    assert abs(rep["true_rel_res"] - res) <= 1e-9 + 1e-2 * res
    x7, rep7, _ = shard_solve(nb, s, ranks, binding.solve_opts(rtol=1e-7))
    assert rep7["status"] == 0
    assert rel_l2(x7, osv.reference_solution(A, s.b, s.x0)) <= 1e-5


def test_one_subdomain_agrees_with_the_single_domain_solver():
    """Same method, different summation order (layer-ordered sums against the solver's
    grid-stride sums): the same iteration count within a few and both at the oracle."""
    s = SHARD_SCENES["lava_box_20"]()
    nb, _ = lib_build(s)
    off, idx, A = oracle_system(s)
    xs, rs, _ = shard_solve(nb, s, 1)
    xp, rp = gpu_solve(nb, s)
    assert rs["status"] == 0 and rp["status"] == 0
    assert abs(rs["iters"] - rp["iters"]) <= max(8, rp["iters"] // 10)
    assert oop.true_residual(A, xs, s.b)[0] <= 1e-6


def test_shard_rejects_other_solver_options_and_a_changed_operator():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = SHARD_SCENES["lava_box_20"]()
    nb, _ = lib_build(s)
    sh = binding.Shard(nb, params_for(s), 2)
    b = torch.from_numpy(s.b).cuda()
    x = torch.from_numpy(s.x0).cuda()
    for opts in (binding.solve_opts(merged_reductions=1), binding.solve_opts(precision=binding.SPH_PREC_FP64),
                 binding.solve_opts(method=binding.SPH_SOLVER_CG), binding.solve_opts(jacobi=0)):
        with pytest.raises(binding.SphError) as e:
            sh.solve(opts, b, x)
        assert e.value.status == 1
    nb.setup(params_for(s, dt=s.dt * 0.5))                 # a new A(dt): the shard's copy is stale
    with pytest.raises(binding.SphError):
        sh.solve(binding.solve_opts(), b, x)
    sh.close()
    with pytest.raises(binding.SphError):
        binding.Shard(nb, params_for(s), 65)


def test_striping_switch_takes_only_zero_or_one():
    import ctypes

    from paper_2206_14780_gb300 import binding

    s = SHARD_SCENES["couette_dummy"]()
    nb, _ = lib_build(s)
    sh = binding.Shard(nb, params_for(s), 2)
    lib = binding.load()
    assert lib.sph_shard_set_striping(sh.handle, 2) == 1
    assert lib.sph_shard_set_striping(sh.handle, 1) == 0
    assert lib.sph_shard_set_striping(None, 1) == 1
    sh.close()
    nb.close()
