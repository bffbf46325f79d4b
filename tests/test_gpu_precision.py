"""Precision study on the Papanastasiou slope (mu from the GPU mu pass: 1e3..1e5 Pa s with the
plastic viscosity mu0 = 1e3 Pa s, about 2..7e4 Pa s with mu0 = 1 Pa s and a faster shear
profile): mixed float32/float64 and all-float64 solves against the float64 oracle on the
57,500-particle subset."""
import numpy as np
import pytest

import scenes
from oracle import neighbors as onb, operator as oop, solvers as osv
from sph_testutil import lib_build, params_for, rel_l2, torch_cuda

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.parametrize("mu0,U,span", [(1e3, 0.1, 50.0), (1.0, 3.3, 1e4)])
def test_slope_subset_mixed_and_fp64_against_oracle(mu0, U, span):
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = scenes.slope_subset(0, mu0=mu0, U=U)
    nb, _ = lib_build(s)
    mu = torch.empty(s.n, dtype=torch.float32, device="cuda")
    nb.mu_papanastasiou(torch.from_numpy(s.vel).cuda(), torch.from_numpy(s.wall_vel).cuda(), *s.rheology, mu,
                        set_handle=True)
    mu_np = mu.cpu().numpy()
    fl = s.ptype == scenes.FLUID
    assert mu_np[fl].max() / mu_np[fl].min() > span           # two decades, or four
    s.mu = mu_np                                              # the oracle uses the same float32 mu
    off, idx = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    A = oop.assemble(s, off, idx)
    x_ref = osv.reference_solution(A, s.b, s.x0, rtol=1e-13)
    out = {}
    for name, prec in (("mixed", binding.SPH_PREC_MIXED), ("fp64", binding.SPH_PREC_FP64)):
        b = torch.from_numpy(s.b).cuda()
        x = torch.from_numpy(s.x0).cuda()
        rtol = 1e-6 if prec == binding.SPH_PREC_MIXED else 1e-10
        rep = nb.solve(params_for(s), binding.solve_opts(rtol=rtol, precision=prec), b, x)
        xg = x.cpu().numpy()
        res, _ = oop.true_residual(A, xg, s.b)
        out[name] = (rep, res, rel_l2(xg, x_ref))
    rep, res, err = out["mixed"]
    assert rep["status"] == 0 and res <= 1e-6 and err <= 1e-5, out["mixed"]
    rep, res, err = out["fp64"]
    assert rep["status"] == 0 and res <= 1e-10 and err <= 1e-8, out["fp64"]
