"""The breakdown safeguards of the restructured BiCGSTAB on the GPU (Sec. 4.2, "Stopping
criterion"; reading X8), against the oracle's scalar steps.

sph_bicgstab_replay runs the solver's own device code for the three scalar steps
(after delta, after omega, after gamma' and r.r) on dots chosen here; the
expected tables come from the oracle's ``scalar_after_*`` functions sequenced the
way the oracle's restructured BiCGSTAB sequences them (frozen components, a
single exit when nothing progresses or the cap is reached), and from traces of
oracle solves whose matrices drive each branch.  Full solves through
sph_visc_solve then exercise omega = 0 and per-component states on real scenes.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import scenes
from oracle import operator as oop, solvers as osv
from sph_testutil import gpu_solve, lib_build, oracle_system, rel_l2

pytestmark = pytest.mark.gpu

C, S, P = osv.CONVERGED, osv.STALLED, osv.PROGRESSING


def oracle_table(gamma0, eps, maxit, dots):
    """The [k + 1][20] table of sph_bicgstab_replay from the oracle's scalar steps."""
    gamma0 = np.asarray(gamma0, np.float64)
    t2 = osv.tau2(gamma0, eps)
    state = np.where((gamma0 == 0.0) | (gamma0 < t2), C, P)
    gam = gamma0.copy()
    zeros = np.zeros(3)
    alpha = omega = alpha_p = beta = zeros
    stalled_any = np.zeros(3, bool)
    it = 0
    done = not np.any(state == P)
    rows = []

    def row():
        rows.append(np.concatenate([alpha, omega, alpha_p, beta, state, stalled_any, [it, float(done)]]))

    row()
    for d in np.asarray(dots, np.float64).reshape(-1, 15):
        if not done:
            live = state == P
            alpha, stall = osv.scalar_after_delta(d[0:3], gam, live)
            omega = osv.scalar_after_omega(d[3:6], d[6:9], live)
            alpha_p, beta, gam, state = osv.scalar_after_update(state, stall, omega, d[0:3], gam, d[9:12],
                                                                d[12:15], t2, live)
            stalled_any = stalled_any | (state == S)
            it += 1
            done = (not np.any(state == P)) or it >= maxit
        row()
    return np.array(rows, np.float64)


def gpu_table(gamma0, eps, maxit, dots):
    from paper_2206_14780_gb300 import binding

    return binding.bicgstab_replay(gamma0, eps, maxit, np.asarray(dots, np.float64).reshape(-1, 15))


def assert_tables_equal(got, want):
    # the same float64 divisions and comparisons on both sides: bit for bit
    np.testing.assert_array_equal(got, want)


def _d(delta, sA, AA, gn, rr):
    return np.concatenate([np.broadcast_to(np.asarray(v, np.float64), (3,)) for v in (delta, sA, AA, gn, rr)])


CHOSEN = {
    # one normal iteration, then delta = 0 on component 0, NaN on 1, +inf on 2
    "delta_zero_nan_inf": (
        [4.0, 4.0, 4.0], 1e-6, 50,
        [_d(2.0, 1.0, 2.0, 1.0, 1.0), _d([0.0, np.nan, np.inf], 1.0, 2.0, 1.0, 1.0)]),
    # omega: denominator 0, negative, +inf, numerator NaN (component-wise), later iterations keep frozen
    "omega_branches": (
        [1.0, 2.0, 3.0], 1e-6, 50,
        [_d(1.0, [1.0, 1.0, np.nan], [0.0, -1.0, 2.0], 0.5, 0.5),
         _d(1.0, 1.0, [np.inf, 1.0, 1.0], 0.5, 0.5),
         _d(1.0, 1.0, 1.0, 0.5, 0.5)]),
    # converged is checked before stalled: delta = 0 but r.r below tau^2
    "converged_before_stalled": (
        [1.0, 1.0, 1.0], 1e-3, 50,
        [_d([0.0, 1.0, 1.0], 1.0, 1.0, 1.0, [1e-8, 1e-8, 0.5]), _d(1.0, 1.0, 1.0, 1.0, 1e-9)]),
    # r.r or gamma' not finite, and alpha' / beta overflowing to infinity
    "nonfinite_update": (
        [1.0, 1.0, 1.0], 1e-6, 50,
        [_d([1.0, 1.0, 1e-300], 1.0, 1.0, [np.nan, 1.0, 1e10], [1.0, np.inf, 1.0]),
         _d(1.0, 1.0, 1.0, 1.0, 1.0)]),
    # gamma / delta overflows: alpha = 0 and a stall
    "alpha_overflow": ([1e10, 1.0, 1.0], 1e-6, 50, [_d([1e-310, 1.0, 1.0], 1.0, 1.0, 1.0, 1.0)]),
    # a zero right-hand side component is converged from the start and never moves;
    # the cap stops the pass after two iterations
    "zero_rhs_and_cap": (
        [0.0, 1.0, 1.0], 1e-9, 2,
        [_d(1.0, 1.0, 2.0, 0.5, 0.5), _d(1.0, 1.0, 2.0, 0.5, 0.25), _d(1.0, 1.0, 2.0, 0.5, 0.1)]),
    # tau^2 floor: eps^2 gamma0 below FLT_MIN uses FLT_MIN (not squared)
    "flt_min_floor": ([1e-40, 1e-30, 1.0], 1e-12, 50, [_d(1.0, 1.0, 1.0, 1.0, [1e-39, 1e-37, 1.0])]),
}


@pytest.mark.parametrize("name", sorted(CHOSEN))
def test_replay_matches_oracle_on_chosen_dots(name):
    g0, eps, maxit, dots = CHOSEN[name]
    want = oracle_table(g0, eps, maxit, dots)
    got = gpu_table(g0, eps, maxit, dots)
    assert_tables_equal(got, want)


def test_chosen_dots_give_the_documented_states():
    """The outcomes the reading of Sec. 4.2 fixes, written out: a stall on delta = 0,
    NaN or inf; omega = 0 for a non-positive or infinite denominator and a NaN
    numerator; converged before stalled; a non-finite r.r is a stall; a NaN gamma'
    or an overflowing alpha' zeroes alpha' and beta (the NaN gamma' then stalls the
    component at the next delta step)."""
    t = gpu_table(*CHOSEN["delta_zero_nan_inf"])
    np.testing.assert_array_equal(t[2, 12:15], [S, S, S])
    np.testing.assert_array_equal(t[2, 0:3], 0.0)
    assert t[2, 19] == 1.0 and t[2, 18] == 2.0
    t = gpu_table(*CHOSEN["omega_branches"])
    np.testing.assert_array_equal(t[1, 3:6], 0.0)
    np.testing.assert_array_equal(t[1, 12:15], [S, S, S])
    t = gpu_table(*CHOSEN["converged_before_stalled"])
    np.testing.assert_array_equal(t[1, 12:15], [C, C, P])
    np.testing.assert_array_equal(t[1, 15:18], [0, 0, 0])
    t = gpu_table(*CHOSEN["nonfinite_update"])
    np.testing.assert_array_equal(t[1, 12:15], [P, S, P])
    assert t[1, 6] == 0.0 and t[1, 9] == 0.0           # gamma' NaN: alpha' = beta = 0
    assert t[1, 8] == 0.0 and t[1, 11] == 0.0          # alpha' = 1e10 / 1e-300 overflows: both 0
    np.testing.assert_array_equal(t[2, 12:15], [S, S, P])
    t = gpu_table(*CHOSEN["zero_rhs_and_cap"])
    assert t[0, 12] == C and t[-1, 18] == 2.0 and t[-1, 19] == 1.0
    np.testing.assert_array_equal(t[:, 0], 0.0)
    t = gpu_table(*CHOSEN["flt_min_floor"])
    np.testing.assert_array_equal(t[1, 12:15], [C, P, P])


def _trace_dots(res):
    return np.array([np.concatenate([h["delta"], h["sA"], h["AA"], h["gam_n"], h["rr"]]) for h in res.history])


def _trace_table(res):
    stalled = np.zeros(3, bool)
    rows = []
    for i, h in enumerate(res.history):
        stalled |= h["state"] == S
        done = (not np.any(h["state"] == P)) or i + 1 == len(res.history)
        rows.append(np.concatenate([h["alpha"], h["omega"], h["alpha_p"], h["beta"], h["state"], stalled,
                                    [i + 1, float(done)]]))
    return np.array(rows)


def _systems():
    rng = np.random.default_rng(5)
    M = sp.csr_matrix(np.eye(12) * 4.0 + rng.normal(size=(12, 12)))
    yield "nonsymmetric_12", M, rng.normal(size=(12, 3)), True
    yield "two_by_two", sp.csr_matrix(np.diag([1.0, 2.0])), np.array([[1.0, 1.0, 0.0], [0.0, 1.0, 0.0]]), False
    yield "identity", sp.identity(4, format="csr"), rng.normal(size=(4, 3)), True
    yield "skew_delta_zero", sp.csr_matrix(np.array([[0.0, 1.0], [-1.0, 0.0]])), \
        np.array([[1.0, 1.0, 2.0], [0.0, 1.0, 0.0]]), False
    yield "overflowing_omega", sp.csr_matrix(np.diag([1e200, 1.0])), np.ones((2, 3)), False
    yield "subnormal_delta", sp.csr_matrix(np.array([[1e-320]])), np.ones((1, 3)), False


@pytest.mark.parametrize("case", range(6))
def test_replay_matches_oracle_solve_traces(case):
    """Oracle solves (float64, frozen components as on the GPU) whose matrices drive
    normal progress, a zero right-hand side column, omega = 0 at convergence,
    delta = 0, an overflowing omega denominator and an overflowing alpha: their
    per-iteration dots replayed on the GPU give the oracle's scalars and states."""
    name, A, b, jacobi = list(_systems())[case]
    res = osv.bicgstab_paper(A, b, np.zeros_like(b), eps=1e-10, maxit=40, jacobi=jacobi, freeze_done=True,
                             record=True)
    bs = b / A.diagonal()[:, None] if jacobi else b
    gamma0 = np.einsum("ij,ij->j", bs, bs)
    got = gpu_table(gamma0, 1e-10, 40, _trace_dots(res))
    want = _trace_table(res)
    np.testing.assert_array_equal(got[1:], want, err_msg=name)
    np.testing.assert_array_equal(got[-1, 12:15], res.state, err_msg=name)


def test_identity_system_solve_omega_zero_is_converged():
    """Every particle a dynamic wall: A = I.  Each refinement pass converges in one
    iteration (r = r* - omega A r* vanishes), no component is ever stalled, and the
    refined x equals b to the requested residual.  (omega = 0 itself, which float32
    rounding of delta against gamma avoids here, is driven by the replay tests.)"""
    from paper_2206_14780_gb300 import binding

    s = scenes.random_box(21, nf=500).copy()
    s.ptype[:] = scenes.WALL
    s.boundary = scenes.BC_DYNAMIC
    rng = np.random.default_rng(3)
    s.b = rng.normal(size=(s.n, 3))
    s.x0 = rng.normal(size=(s.n, 3))
    nb, _ = lib_build(s)
    x, rep = gpu_solve(nb, s, binding.solve_opts(rtol=1e-12, eps_inner=1e-6))
    assert rep["status"] == 0, rep
    assert rep["state"] == [C, C, C] and rep["stalled_any"] == [0, 0, 0]
    assert rep["iters"] == rep["refinements"]                 # one iteration per pass
    assert rel_l2(x, s.b) <= 1e-12


def test_component_states_with_a_zero_rhs_component_and_one_exact():
    """Component 1 has b = 0 and x0 = 0 (converged from the start, x untouched),
    component 2 starts at the oracle's solution (converged from the start), component 0
    progresses to the oracle's solution; no component is reported stalled."""
    from paper_2206_14780_gb300 import binding

    s = scenes.random_box(22, nf=400, mu_spread=10.0)
    nb, _ = lib_build(s)
    off, idx, A = oracle_system(s)
    b = s.b.copy()
    b[:, 1] = 0.0
    x_ref = osv.reference_solution(A, b, s.x0, rtol=1e-14)
    x0 = s.x0.copy()
    x0[:, 1] = 0.0
    x0[:, 2] = x_ref[:, 2]
    x, rep = gpu_solve(nb, s, binding.solve_opts(rtol=1e-7), b=b, x0=x0)
    assert rep["status"] == 0, rep
    assert rep["state"] == [C, C, C] and rep["stalled_any"] == [0, 0, 0]
    np.testing.assert_array_equal(x[:, 1], 0.0)
    res, per = oop.true_residual(A, x, b)
    assert res <= 1e-7
    assert rel_l2(x[:, 0], x_ref[:, 0]) <= 1e-5 and rel_l2(x[:, 2], x_ref[:, 2]) <= 1e-6
