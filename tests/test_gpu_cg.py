"""The rotated conjugate gradient (Sec. 4.1, second listing) on the GPU, for the symmetric
dynamic-boundary systems of Sec. 4, against the oracle."""
import numpy as np
import pytest

import scenes
from oracle import operator as oop, solvers as osv
from sph_testutil import gpu_solve, lib_build, oracle_system, params_for, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

CG_SCENES = {
    # moving top wall: the full matrix is not symmetric, the fluid block is
    "couette_dynamic": lambda: scenes.couette(1, boundary=scenes.BC_DYNAMIC),
    # no walls: symmetric, viscosity spread over a decade
    "periodic_lattice_mu": lambda: scenes.periodic_lattice(10, jitter=0.1, mu_spread=10.0, seed=4),
    # irregular positions over a moving floor, harmonic and arithmetic means
    "random_box_dynamic": lambda: scenes.random_box(6, nf=500, boundary=scenes.BC_DYNAMIC, mu_spread=5.0),
    "random_box_dynamic_arith": lambda: scenes.random_box(7, nf=400, boundary=scenes.BC_DYNAMIC,
                                                          mean=scenes.MEAN_ARITHMETIC, periodic=(0, 0, 0)),
    # the stiff box (dt sum c ~ 670) with dynamic walls, several tiles
    "lava_box_16_dynamic": lambda: scenes.lava_box(3, n=16, boundary=scenes.BC_DYNAMIC),
}


def _dynamic(s):
    # a periodic lattice has no walls: the dynamic and dummy matrices coincide
    s = s.copy()
    s.boundary = scenes.BC_DYNAMIC
    return s


@pytest.mark.parametrize("name", sorted(CG_SCENES))
@pytest.mark.parametrize("jacobi", [1, 0])
def test_cg_solution_matches_oracle(name, jacobi):
    from paper_2206_14780_gb300 import binding

    s = _dynamic(CG_SCENES[name]())
    nb, _ = lib_build(s)
    off, idx, A = oracle_system(s)
    x_ref = osv.reference_solution(A, s.b, s.x0)
    opts = dict(method=binding.SPH_SOLVER_CG, jacobi=jacobi)
    x, rep = gpu_solve(nb, s, binding.solve_opts(**opts))
    assert rep["status"] == 0, rep
    assert rep["stalled_any"] == [0, 0, 0]
    res, _ = oop.true_residual(A, x, s.b)
    assert res <= 1e-6, (res, rep)
    x7, rep7 = gpu_solve(nb, s, binding.solve_opts(rtol=1e-7, **opts))
    assert rep7["status"] == 0 and rel_l2(x7, x_ref) <= 1e-5
    # the oracle's own rotated CG (Jacobi-preconditioned, wall rows started at b)
    wall = s.ptype == scenes.WALL
    x0 = s.x0.copy()
    x0[wall] = s.b[wall]
    x_cg, _, st, _ = osv.cg_rotated(A, s.b, x0, eps=1e-12, jacobi=True, record=True)
    assert np.all(st == osv.CONVERGED)
    assert rel_l2(x7, x_cg) <= 1e-5


@pytest.mark.parametrize("form", [1, 2, 3, 4])
def test_cg_every_register_form(form):
    from paper_2206_14780_gb300 import binding

    s = CG_SCENES["lava_box_16_dynamic"]()
    nb, _ = lib_build(s)
    off, idx, A = oracle_system(s)
    x, rep = gpu_solve(nb, s, binding.solve_opts(method=binding.SPH_SOLVER_CG, apply_form=form))
    assert rep["status"] == 0, rep
    res, _ = oop.true_residual(A, x, s.b)
    assert res <= 1e-6


def test_cg_needs_fewer_operator_applies_than_bicgstab():
    """One apply per CG iteration against two per BiCGSTAB iteration, on the stiff box
    with dynamic walls: the CG solve applies the operator fewer times in all."""
    from paper_2206_14780_gb300 import binding

    s = CG_SCENES["lava_box_16_dynamic"]()
    nb, _ = lib_build(s)
    _, rep_cg = gpu_solve(nb, s, binding.solve_opts(method=binding.SPH_SOLVER_CG))
    _, rep_bi = gpu_solve(nb, s, binding.solve_opts())
    assert rep_cg["status"] == 0 and rep_bi["status"] == 0
    assert rep_cg["iters"] < 2 * rep_bi["iters"], (rep_cg, rep_bi)


def test_invalid_method_combinations_are_rejected():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = scenes.couette(2)                          # dummy walls: not symmetric
    nb, _ = lib_build(s)
    for opts in (binding.solve_opts(method=binding.SPH_SOLVER_CG),
                 binding.solve_opts(jacobi=0),
                 binding.solve_opts(method=2),
                 binding.solve_opts(method=binding.SPH_SOLVER_CG, precision=binding.SPH_PREC_FP64)):
        b = torch.from_numpy(s.b).cuda()
        x = torch.from_numpy(s.x0).cuda()
        with pytest.raises(binding.SphError) as e:
            nb.solve(params_for(s), opts, b, x)
        assert e.value.status == 1
    sd = CG_SCENES["couette_dynamic"]()
    nbd, _ = lib_build(sd)
    with pytest.raises(binding.SphError):
        gpu_solve(nbd, sd, binding.solve_opts(method=binding.SPH_SOLVER_CG, apply_form=5))
