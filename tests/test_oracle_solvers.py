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
    for h1, h2 in zip(r1.history, r2.history):
        np.testing.assert_allclose(h1["x"], h2["x"], rtol=0, atol=1e-9 * np.abs(h1["x"]).max())
        np.testing.assert_allclose(h1["rr"], h2["rr"], rtol=1e-6)


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


# ---- breakdown safeguards of Sec. 4.2 ("Stopping criterion"), reading X8, derived by hand ----

C, S, P = solvers.CONVERGED, solvers.STALLED, solvers.PROGRESSING


@pytest.mark.parametrize("freeze", [False, True])
def test_two_by_two_iterates_by_hand(freeze):
    """A = diag(1, 2), b = [e1, (1, 1)], x0 = 0, no Jacobi, worked out in exact arithmetic.

    Column 0: p = r0 = e1, A p = e1, delta = 1, alpha = 1, r* = 0, A r* = 0, so omega
    cannot be formed (0/0) and is zero; r.r = 0 < tau^2: converged after one iteration
    with x = e1.  Column 1: gamma0 = 2, A p = (1, 2), delta = 3, alpha = 2/3,
    r* = (1/3, -1/3), A r* = (1/3, -2/3), omega = (1/3)/(5/9) = 3/5, r = (2/15, 1/15),
    x = (13/15, 7/15), gamma' = 1/5, alpha' = 1/15, beta = 1/9; then p = (8/45, 2/45),
    delta = 4/15, alpha = 3/4 and r* = 0: x = (1, 1/2), converged after two.  Without
    freezing, column 0 runs the second iteration too: p = 0 gives delta = 0 (a stall),
    but r.r = 0 < tau^2 is checked first, so it stays converged and x is unchanged."""
    A = sp.csr_matrix(np.diag([1.0, 2.0]))
    b = np.array([[1.0, 1.0], [0.0, 1.0]])
    res = solvers.bicgstab_paper(A, b, np.zeros((2, 2)), eps=1e-12, jacobi=False, freeze_done=freeze,
                                 record=True)
    assert res.iters == 2
    np.testing.assert_array_equal(res.state, [C, C])
    np.testing.assert_array_equal(res.stalled_any, [False, False])
    h1, h2 = res.history
    tol = dict(rtol=4e-16, atol=4e-16)
    np.testing.assert_allclose(h1["x"], [[1.0, 13 / 15], [0.0, 7 / 15]], **tol)
    np.testing.assert_allclose(h1["delta"], [1.0, 3.0], **tol)
    np.testing.assert_allclose(h1["alpha"], [1.0, 2 / 3], **tol)
    np.testing.assert_allclose(h1["omega"], [0.0, 3 / 5], **tol)
    np.testing.assert_allclose(h1["gam_n"], [0.0, 1 / 5], **tol)
    np.testing.assert_allclose(h1["alpha_p"], [0.0, 1 / 15], **tol)
    np.testing.assert_allclose(h1["beta"], [0.0, 1 / 9], **tol)
    np.testing.assert_array_equal(h1["state"], [C, P])
    np.testing.assert_allclose(h2["delta"][1], 4 / 15, **tol)
    np.testing.assert_allclose(h2["alpha"][1], 3 / 4, **tol)
    np.testing.assert_allclose(res.x, [[1.0, 1.0], [0.0, 0.5]], rtol=0, atol=1e-15)
    assert h2["alpha"][0] == 0.0 and h2["omega"][0] == 0.0
    np.testing.assert_array_equal(h2["live"], [not freeze, True])


def test_omega_zero_on_identity_is_converged():
    """A = I: one iteration gives alpha = 1, r* = 0 and A r* = 0, so omega = 0; r.r = 0
    makes the component converged (not stalled) with x = b exactly."""
    A = sp.identity(3, format="csr")
    b = np.array([[1.0], [2.0], [3.0]])
    res = solvers.bicgstab_paper(A, b, np.zeros((3, 1)), record=True)
    assert res.iters == 1 and res.state[0] == C and not res.stalled_any[0]
    assert res.history[0]["omega"][0] == 0.0 and res.history[0]["alpha"][0] == 1.0
    np.testing.assert_array_equal(res.x, b)


def test_omega_from_an_overflowing_denominator_is_zero_and_stalls():
    """A = diag(1e200, 1), b = (1, 1): delta = 1e200 + 1, alpha = 2/delta, r* = (-1, 1)
    to rounding, A r* = (-1e200, 1) so Ar*.Ar* overflows to +inf: omega = 0, r = r*
    with r.r = 2 > tau^2, hence stalled after one iteration with x = alpha (1, 1)."""
    A = sp.csr_matrix(np.diag([1e200, 1.0]))
    b = np.ones((2, 1))
    res = solvers.bicgstab_paper(A, b, np.zeros((2, 1)), jacobi=False, record=True)
    h = res.history[0]
    assert res.iters == 1 and res.state[0] == S and res.stalled_any[0]
    assert np.isinf(h["AA"][0]) and h["omega"][0] == 0.0
    assert h["alpha_p"][0] == 0.0 and h["beta"][0] == 0.0
    np.testing.assert_allclose(res.x[:, 0], 2e-200, rtol=1e-15)
    np.testing.assert_allclose(h["rr"][0], 2.0, rtol=1e-15)


def test_nonfinite_alpha_stalls():
    """A = (1e-320) (a subnormal), b = 1: gamma = 1, delta = 1e-320 and gamma/delta
    overflows: alpha = 0 and the component stalls with x = x0 = 0."""
    A = sp.csr_matrix(np.array([[1e-320]]))
    res = solvers.bicgstab_paper(A, np.ones((1, 1)), np.zeros((1, 1)), jacobi=False, record=True)
    assert res.iters == 1 and res.state[0] == S
    assert res.history[0]["alpha"][0] == 0.0
    np.testing.assert_array_equal(res.x, 0.0)


def test_scalar_steps_on_chosen_values():
    """Each branch of the scalar steps on hand-chosen dots (reading X8)."""
    live = np.ones(4, bool)
    a, st = solvers.scalar_after_delta([0.0, np.nan, np.inf, 2.0], [1.0, 1.0, 1.0, 4.0], live)
    np.testing.assert_array_equal(a, [0.0, 0.0, 0.0, 2.0])
    np.testing.assert_array_equal(st, [True, True, True, False])
    a, st = solvers.scalar_after_delta([1e-310, 3.0], [1e10, 1.0], np.array([True, False]))
    np.testing.assert_array_equal(a, [0.0, 0.0])          # 1e10 / 1e-310 overflows; a frozen one stays 0
    np.testing.assert_array_equal(st, [True, False])
    om = solvers.scalar_after_omega([1.0, 1.0, 1.0, np.nan, 3.0, 1e300], [0.0, -1.0, np.inf, 2.0, 1.5, 1e-300],
                                    np.ones(6, bool))
    np.testing.assert_array_equal(om, [0.0, 0.0, 0.0, 0.0, 2.0, 0.0])
    # update: converged first, then stalled (stall now / omega = 0 / r.r not finite), else progressing
    state = np.array([P, P, P, P, P, P, C])
    stall = np.array([True, False, False, False, False, False, False])
    omega = np.array([0.5, 0.0, 0.5, 0.5, 0.5, 1e-300, 0.5])
    delta = np.array([2.0, 2.0, 2.0, 2.0, 4.0, 1e-300, 2.0])
    gam = np.full(7, 9.0)
    gam_n = np.array([1.0, 1.0, 1.0, 1.0, 2.0, 1e10, 1.0])
    rr = np.array([1.0, 1.0, 1e-30, np.nan, 1.0, 1.0, 1.0])
    t2 = np.full(7, 1e-20)
    live = np.array([True] * 6 + [False])
    ap, be, g, s = solvers.scalar_after_update(state, stall, omega, delta, gam, gam_n, rr, t2, live)
    np.testing.assert_array_equal(s, [S, S, C, S, P, P, C])
    np.testing.assert_array_equal(ap, [0.0, 0.0, 0.5, 0.5, 0.5, 0.0, 0.0])
    np.testing.assert_array_equal(be, [0.0, 0.0, 1.0, 1.0, 1.0, 0.0, 0.0])  # 1e10/1e-300 overflows: both 0
    np.testing.assert_array_equal(g, [1.0, 1.0, 1.0, 1.0, 2.0, 1e10, 9.0])


# ---- rotated CG (Sec. 4.1, second listing), by hand and against LU ----

def test_rotated_cg_iterates_by_hand():
    """A = [[2, 1], [1, 3]], b = (1, 2), x0 = 0, no preconditioner: r0 = p0 = (1, 2),
    A p0 = (4, 7), alpha0 = 5/18, x1 = (5/18, 5/9), r1 = (-1/9, 1/18),
    beta1 = (5/324)/5 = 1/324, p1 = (-35/324, 20/324), alpha1 = 18/25 and
    x2 = (1/5, 3/5), the exact solution, after two iterations."""
    A = sp.csr_matrix(np.array([[2.0, 1.0], [1.0, 3.0]]))
    x, its, st, hist = solvers.cg_rotated(A, np.array([1.0, 2.0]), eps=1e-12, record=True)
    assert its[0] == 2 and st[0] == solvers.CONVERGED
    np.testing.assert_allclose(hist[0][0], [5 / 18, 5 / 9], rtol=4e-16)
    np.testing.assert_allclose(hist[0][1], [0.2, 0.6], rtol=1e-15)


def test_jacobi_cg_solves_a_diagonal_system_in_one_iteration():
    """With z = D^-1 r on A = D: p = z is the exact error, A p = r, alpha = 1."""
    A = sp.diags([2.0, 5.0, 7.0]).tocsr()
    b = np.array([[1.0, -2.0], [3.0, 0.5], [4.0, 1.0]])
    x0 = np.array([[0.5, 0.0], [0.0, 1.0], [1.0, 0.0]])
    x, its, st, _ = solvers.cg_rotated(A, b, x0, eps=1e-14, jacobi=True, record=True)
    np.testing.assert_array_equal(its, [1, 1])
    np.testing.assert_allclose(x, b / np.array([[2.0], [5.0], [7.0]]), rtol=1e-15)


def test_cg_stalls_when_alpha_is_zero():
    """A skew matrix gives p.Ap = 0 in the first iteration: alpha = 0, a stall, x = x0."""
    A = sp.csr_matrix(np.array([[0.0, 1.0], [-1.0, 0.0]]))
    x, its, st, _ = solvers.cg_rotated(A, np.array([1.0, 0.0]), record=True)
    assert its[0] == 1 and st[0] == solvers.STALLED
    np.testing.assert_array_equal(x, 0.0)


@pytest.mark.parametrize("jacobi", [False, True])
def test_cg_on_the_dynamic_wall_channel_matches_lu(jacobi):
    """Dynamic walls with a moving top wall: the full matrix is not symmetric (fluid rows
    see the walls, wall rows are the identity), but with the wall rows of x0 at their
    exact value b the residual vanishes on the walls and CG runs on the symmetric
    fluid block (the reduced system of Sec. 4); it reaches the LU solution."""
    s = scenes.couette(5, nx=8, ny=6, nz=6, boundary=scenes.BC_DYNAMIC)
    off, idx = neighbors.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    A = operator.assemble(s, off, idx)
    wall = s.ptype == scenes.WALL
    x0 = s.x0.copy()
    x0[wall] = s.b[wall]
    x, its, st, _ = solvers.cg_rotated(A, s.b, x0, eps=1e-13, jacobi=jacobi, record=True)
    xl = solvers.dense_solve(A, s.b)
    assert np.all(st == solvers.CONVERGED)
    np.testing.assert_allclose(x, xl, rtol=0, atol=1e-9 * np.abs(xl).max())
    if jacobi:
        _, its_plain = solvers.cg_rotated(A, s.b, x0, eps=1e-13)
        assert np.all(its <= its_plain)
