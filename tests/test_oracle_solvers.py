"""Pins of the solvers of paper Sec. 4 against LU, elimination and the stated semantics."""
import numpy as np
import pytest
import scipy.sparse as sp

import scenes
from oracle import neighbors, operator, rheology, solvers


def _tiny(seed=0, nf=80, **kw):
    s = scenes.random_box(seed, nf=nf, **kw)
    off, idx = neighbors.bruteforce(s.pos, s.lo, s.hi, s.periodic, s.h)
    return s, operator.assemble(s, off, idx)


@pytest.mark.parametrize("seed", [0, 1])
def test_all_solvers_agree_with_lu(seed):
    s, A = _tiny(seed, mu_spread=5.0)
    xl = solvers.dense_solve(A, s.b)
    xg = solvers.gauss_elim(A, s.b)
    np.testing.assert_allclose(xg, xl, rtol=1e-12, atol=1e-12)
    xp = solvers.bicgstab_paper(A, s.b, s.x0, eps=1e-14).x
    xt, _ = solvers.bicgstab_textbook(A, s.b, s.x0, eps=1e-14, jacobi=True)
    xr = solvers.reference_solution(A, s.b, s.x0)
    for x in (xp, xt, xr):
        np.testing.assert_allclose(x, xl, rtol=0, atol=1e-10 * np.abs(xl).max())


def test_rotated_cg_on_symmetric_system():
    s = scenes.periodic_lattice(8, jitter=0.1, seed=1)
    off, idx = neighbors.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    A = operator.assemble(s, off, idx)
    x, its = solvers.cg_rotated(A, s.b, s.x0, eps=1e-13)
    xr = solvers.reference_solution(A, s.b, s.x0)
    np.testing.assert_allclose(x, xr, atol=1e-10)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_restructured_equals_textbook_iterates(k):
    # Sec. 4.2: beta_i = alpha'_{i-1}/omega_{i-1}; the two listings produce the same
    # iterates in exact arithmetic, so in float64 they agree to round-off
    s, A = _tiny(2, nf=150)
    b = s.b[:, :1]
    x0 = s.x0[:, :1]
    xp = solvers.bicgstab_paper(A, b, x0, eps=1e-30, maxit=k).x
    xt, _ = solvers.bicgstab_textbook(A, b, x0, eps=1e-30, maxit=k, jacobi=True)
    np.testing.assert_allclose(xp, xt, rtol=0, atol=1e-11 * np.abs(xt).max())


def test_merged_reductions_match_direct_dots():
    s, A = _tiny(3, nf=150)
    r1 = solvers.bicgstab_paper(A, s.b, s.x0, eps=1e-30, maxit=6, record=True)
    r2 = solvers.bicgstab_paper(A, s.b, s.x0, eps=1e-30, maxit=6, merged=True, record=True)
    for (x1, rr1, _), (x2, rr2, _) in zip(r1.history, r2.history):
        np.testing.assert_allclose(x1, x2, rtol=0, atol=1e-9 * np.abs(x1).max())
        np.testing.assert_allclose(rr1, rr2, rtol=1e-6)


def test_stall_when_delta_is_zero():
    # skew-symmetric A: r0^ . A r0 = 0 exactly, so delta = 0 in the first iteration;
    # alpha = alpha' = beta = 0, the component is reported stalled, single exit
    A = sp.csr_matrix(np.array([[0.0, 1.0], [-1.0, 0.0]]))
    b = np.array([[1.0], [0.0]])
    res = solvers.bicgstab_paper(A, b, np.zeros((2, 1)), jacobi=False)
    assert res.iters == 1
    assert res.state[0] == solvers.STALLED
    np.testing.assert_array_equal(res.x, 0.0)


def test_zero_rhs_component_is_converged_untouched():
    s, A = _tiny(4)
    b = s.b.copy()
    b[:, 2] = 0.0
    x0 = s.x0.copy()
    x0[:, 2] = 0.0
    res = solvers.bicgstab_paper(A, b, x0, eps=1e-12, freeze_done=True)
    assert res.state[2] == solvers.CONVERGED
    np.testing.assert_array_equal(res.x[:, 2], 0.0)
    assert np.all(res.state == solvers.CONVERGED)


def test_tolerance_floor_is_flt_min_not_squared():
    assert solvers.tau2(1e-40, 2.0 ** -23) == 2.0 ** -126
    assert solvers.tau2(1.0, 2.0 ** -23) == 2.0 ** -46


def test_float32_vectors_converge_on_couette():
    s = scenes.couette(0)
    off, idx = neighbors.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    A = operator.assemble(s, off, idx)
    xr = solvers.reference_solution(A, s.b, s.x0)
    res = solvers.bicgstab_paper(A, s.b, s.x0, eps=2.0 ** -23, dtype=np.float32)
    assert np.all(res.state != solvers.PROGRESSING)
    assert np.abs(res.x - xr).max() < 2e-5


def test_merged_and_direct_reductions_on_channel_and_slope():
    """The paper-exact direct gamma' = r0^.r against the merged recurrence, with float64 and
    with float32 vectors (float64 dots), at the paper's eps = 2^-23: the small Couette channel
    and the 57.5k slope subset with its Papanastasiou viscosity.  Every run converges without
    a stall; on the stiff slope the float32 recursion stops at a true residual near 1e-3
    (what the float64 refinement corrects) and the merged form needs more iterations there
    (165 against 131 when measured)."""
    counts = {}
    for name, s in (("couette", scenes.couette(0)), ("slope", scenes.slope_subset(0))):
        off, idx = neighbors.build(s.pos, s.lo, s.hi, s.periodic, s.h)
        mu = rheology.mu_pass(s, off, idx)[0] if s.rheology is not None else None
        A = operator.assemble(s, off, idx, mu=mu)
        for dtype in (np.float64, np.float32):
            for merged in (False, True):
                r = solvers.bicgstab_paper(A, s.b, s.x0, eps=2.0 ** -23, dtype=dtype, merged=merged, maxit=3000)
                assert np.all(r.state == solvers.CONVERGED), (name, dtype, merged, r.state)
                res = np.linalg.norm(s.b - A @ r.x) / np.linalg.norm(s.b)
                assert res < (1e-7 if dtype is np.float64 else 2e-3), (name, dtype, merged, res)
                counts[name, dtype, merged] = r.iters
    assert counts["couette", np.float32, True] == counts["couette", np.float32, False]
    assert counts["slope", np.float32, True] > counts["slope", np.float32, False]
