"""sph_visc_solve_host: the one-call solve from host buffers (scene, v^n, b in; x out)
against the oracle, with its staging reused across calls and both starts."""
import numpy as np
import pytest

import scenes
from oracle import operator as oop, solvers as osv, warmstart as ows
from sph_testutil import SCENES_SMALL, oracle_system, params_for, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def _host(s, torch):
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return dict(pos=pin(np.asarray(s.pos, np.float32)), rho=pin(np.asarray(s.rho, np.float32)),
                mu=pin(np.asarray(s.mu, np.float32)), ptype=pin(np.asarray(s.ptype, np.uint8)),
                vel=pin(np.asarray(s.vel, np.float32)), b=pin(np.asarray(s.b, np.float64)))


@pytest.mark.parametrize("name", ["couette_dummy", "lava_box_12"])
def test_host_solve_matches_oracle(name):
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = SCENES_SMALL[name]()
    off, idx, A = oracle_system(s)
    h = _host(s, torch)
    geo = (s.lo, s.hi, s.periodic, s.h)
    x = torch.empty((s.n, 3), dtype=torch.float64).pin_memory()
    opts = binding.solve_opts(rtol=1e-7)
    rep, nb = binding.solve_host(h["pos"], h["rho"], h["mu"], h["ptype"], *geo, params_for(s), opts, h["vel"],
                                 h["b"], x)
    assert rep["status"] == 0, rep
    xn = x.numpy().copy()
    res, _ = oop.true_residual(A, xn, s.b)
    assert res <= 1e-7 * 1.01, res
    x0 = ows.start(A, s.b, s.vel, None, s.ptype, 1.0)
    assert rel_l2(xn, osv.reference_solution(A, s.b, x0)) <= 1e-5
    # second call on the same handle and staging, now from x (vel = None): starts at the
    # solution, so it needs no pass and returns it unchanged up to the residual check
    rep2, nb2 = binding.solve_host(h["pos"], h["rho"], h["mu"], h["ptype"], *geo, params_for(s), opts, None,
                                   h["b"], x, nb=nb)
    assert nb2 is nb and rep2["status"] == 0 and rep2["iters"] == 0, rep2
    np.testing.assert_array_equal(x.numpy(), xn)
    nb.close()


def test_host_solve_rejects_null_and_bad_scene():
    torch = torch_cuda()
    from paper_2206_14780_gb300 import binding

    s = SCENES_SMALL["couette_dummy"]()
    h = _host(s, torch)
    x = torch.empty((s.n, 3), dtype=torch.float64)
    with pytest.raises(binding.SphError):
        binding.solve_host(h["pos"], h["rho"], h["mu"], h["ptype"], s.lo, s.hi, s.periodic, -1.0,
                           params_for(s), binding.solve_opts(), h["vel"], h["b"], x)
