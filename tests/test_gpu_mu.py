"""GPU Papanastasiou viscosity pass against the oracle (float64)."""
import numpy as np
import pytest

import scenes
from oracle import neighbors as onb, rheology
from sph_testutil import lib_build, torch_cuda

pytestmark = pytest.mark.gpu

MU_RTOL = 1e-4   # float32 gradient sums over ~80 neighbours; mu is 1-Lipschitz in log D


def test_mu_pass_matches_oracle():
    torch = torch_cuda()
    s = scenes.slope_subset(2, nx=20, ny=12, nz=20)
    nb, _ = lib_build(s)
    off, idx = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    mu_ref, D = rheology.mu_pass(s, off, idx)
    vel = torch.from_numpy(s.vel).cuda()
    wv = torch.from_numpy(s.wall_vel).cuda()
    out = torch.empty(s.n, dtype=torch.float32, device="cuda")
    tau0, mu0, m = s.rheology
    nb.mu_papanastasiou(vel, wv, tau0, mu0, m, out, set_handle=True)
    mu = out.cpu().numpy().astype(np.float64)
    fl = s.ptype == scenes.FLUID
    err = np.abs(mu[fl] - mu_ref[fl]) / mu_ref[fl]
    assert err.max() < MU_RTOL, err.max()
    # both regimes of Ybar occur: the series (m D < 0.5) and the direct formula
    x = m * D[fl]
    assert (x < 0.5).any() and (x >= 0.5).any()
