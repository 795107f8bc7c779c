"""Pins of the oracle's tabulated (piecewise-linear) property laws.

Section 3.1.6 gives rho, c and k at two temperatures; a table with more
points makes each law piecewise linear.  The pins: numpy's own interpolation
inside the table, hand-computed values outside it, the linear laws for a
two-point or collinear table, the discrete steady state of a Dirichlet bar
(equal element fluxes with Eq. 13's average of k), the closed-form relaxation
of a uniform perfused block, and the critical-step scale against brute force."""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import Oracle, critical_dt, piecewise_linear
from oracle.critical_dt import td_scale
from synth.meshes import box_face_nodes, hex_box, kuhn_tet_box
from synth.problem import Material, Perfusion, Problem

H = 1e-3
# liver-like values with kinks at 42 and 50 degC (rho, c falling, k rising)
TAB = dict(T=(30.0, 42.0, 50.0, 70.0),
           rho=(1060.0, 1050.0, 1030.0, 1000.0),
           c=(3600.0, 3700.0, 3500.0, 3300.0),
           k=(0.50, 0.56, 0.70, 0.74))


def _tab():
    return Material.tabulated(TAB["T"], TAB["rho"], TAB["c"], TAB["k"])


def test_piecewise_linear_inside_is_numpy_interp():
    T = np.linspace(30.0, 70.0, 1001)
    for key in ("rho", "c", "k"):
        np.testing.assert_allclose(piecewise_linear(TAB["T"], TAB[key], T), np.interp(T, TAB["T"], TAB[key]),
                                   rtol=1e-14, atol=0)
    # at the points: the table values
    np.testing.assert_allclose(piecewise_linear(TAB["T"], TAB["k"], np.array(TAB["T"])), TAB["k"], rtol=1e-15)


def test_piecewise_linear_extends_the_end_intervals():
    # below 30: slope of [30, 42] for k is 0.06 / 12 = 0.005 per K
    assert piecewise_linear(TAB["T"], TAB["k"], 20.0) == pytest.approx(0.50 - 0.05, rel=1e-14)
    # above 70: slope of [50, 70] for rho is -30 / 20 = -1.5 per K
    assert piecewise_linear(TAB["T"], TAB["rho"], 80.0) == pytest.approx(1000.0 - 15.0, rel=1e-14)
    # the right end point itself and just past a kink
    assert piecewise_linear(TAB["T"], TAB["c"], 50.0) == pytest.approx(3500.0, rel=1e-15)
    assert piecewise_linear(TAB["T"], TAB["c"], 51.0) == pytest.approx(3490.0, rel=1e-14)


def test_two_point_and_collinear_tables_are_the_linear_laws():
    lin = Material.from_two_points(37.0, 65.0, (1040.0, 1000.0), (3600.0, 3700.0), (0.5, 0.6))
    two = Material.tabulated((37.0, 65.0), (1040.0, 1000.0), (3600.0, 3700.0), (0.5, 0.6))
    Ts = np.array([20.0, 37.0, 41.5, 64.0, 90.0])
    sl = (65.0 - 37.0)
    line = lambda v0, v1, T: v0 + (v1 - v0) / sl * (T - 37.0)   # noqa: E731
    col = Material.tabulated((37.0, 44.0, 51.0, 65.0), tuple(line(1040.0, 1000.0, t) for t in (37.0, 44.0, 51.0, 65.0)),
                             tuple(line(3600.0, 3700.0, t) for t in (37.0, 44.0, 51.0, 65.0)),
                             tuple(line(0.5, 0.6, t) for t in (37.0, 44.0, 51.0, 65.0)))
    m = kuhn_tet_box(4, 3, 3, H)
    runs = []
    for mat in (lin, two, col):
        p = Problem(m.elem_type, m.xyz, m.conn, mat, dirichlet_nodes=box_face_nodes(m, ("x0",)),
                    dirichlet_T=np.full(len(box_face_nodes(m, ("x0",))), 60.0), T0=37.0)
        orc = Oracle(p)
        np.testing.assert_allclose(orc.k_of(Ts), line(0.5, 0.6, Ts), rtol=1e-13)
        runs.append(orc.run(0.9 * critical_dt(orc, 30.0, 70.0), 300))
    np.testing.assert_allclose(runs[1], runs[0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(runs[2], runs[0], rtol=0, atol=1e-12)


def test_tabulated_bar_has_equal_element_fluxes_at_steady_state():
    """A Dirichlet bar, insulated elsewhere, reaches a steady state in which
    every element carries the same heat: with Eq. 13's average over the
    element's nodes, (k(T_i) + k(T_i+1)) / 2 * (T_i+1 - T_i) is the same for
    every element.  The temperatures cross both kinks of the k table."""
    n = 8
    m = hex_box(n, 1, 1, H)
    left, right = box_face_nodes(m, ("x0",)), box_face_nodes(m, ("x1",))
    p = Problem(m.elem_type, m.xyz, m.conn, _tab(), dirichlet_nodes=np.concatenate([left, right]),
                dirichlet_T=np.concatenate([np.full(4, 37.0), np.full(4, 65.0)]), T0=40.0)
    orc = Oracle(p)
    T = orc.run(0.9 * critical_dt(orc, 30.0, 70.0), 6000)
    ix = m.grid_index[:, 0]
    Tx = np.array([T[ix == i].mean() for i in range(n + 1)])
    assert np.all(np.array([np.ptp(T[ix == i]) for i in range(n + 1)]) < 1e-12)
    assert Tx[0] < 42.0 and Tx[n] > 50.0 and np.any((Tx > 42.0) & (Tx < 50.0))   # both kinks inside the bar
    kx = np.interp(Tx, TAB["T"], TAB["k"])
    flux = 0.5 * (kx[1:] + kx[:-1]) * np.diff(Tx)
    np.testing.assert_allclose(flux, flux.mean(), rtol=1e-10)


def test_tabulated_capacity_relaxation_follows_the_separated_ode():
    """Uniform and insulated, each node obeys rho(T) c(T) dT/dt = w_b c_b (T_a - T),
    so t = 1/(w_b c_b) int_T0^T rho c / (T_a - s) ds, in closed form on each
    piece where rho c is a quadratic; both laws have a kink at 42 degC on
    the way from 37 to 45.  Explicit Euler is first order:
    Richardson's 2 T(dt/2) - T(dt) hits the closed form to O(dt^2)."""
    m = hex_box(2, 1, 1, H)
    pf = Perfusion(w_b=26.6, c_b=3617.0, T_a=45.0)
    p = Problem(m.elem_type, m.xyz, m.conn, _tab(), perfusion=pf, T0=37.0)
    t_end, dt = 80.0, 0.02
    T1 = Oracle(p).run(dt, int(round(t_end / dt)))
    T2 = Oracle(p).run(dt / 2, int(round(t_end / dt * 2)))

    from numpy.polynomial import Polynomial as P

    def piece(lo, hi):   # rho(s) c(s) on one table interval, as a polynomial in s
        i = int(np.searchsorted(TAB["T"], lo, side="right") - 1)
        T0, T1 = TAB["T"][i], TAB["T"][i + 1]
        r = P([TAB["rho"][i], (TAB["rho"][i + 1] - TAB["rho"][i]) / (T1 - T0)])
        c = P([TAB["c"][i], (TAB["c"][i + 1] - TAB["c"][i]) / (T1 - T0)])
        return (r * c)(P([-T0, 1.0]))

    def integral(a, b):
        """int_a^b p(s) / (T_a - s) ds in closed form: p = q (T_a - s) + p(T_a)."""
        p = piece(a, b)
        q, rem = divmod(p, P([pf.T_a, -1.0]))
        Q = q.integ()
        return (Q(b) - Q(a)) - rem.coef[0] * (np.log(pf.T_a - b) - np.log(pf.T_a - a))

    def t_of(T):
        return (integral(37.0, min(T, 42.0)) + (integral(42.0, T) if T > 42.0 else 0.0)) / (pf.w_b * pf.c_b)

    exact = brentq(lambda T: t_of(T) - t_end, 37.0, pf.T_a - 1e-9, xtol=1e-14)
    assert exact > 43.0                                  # the kink was crossed
    assert np.max(np.abs(2 * T2 - T1 - exact)) < 1e-6
    assert np.max(np.abs(T2 - exact)) > 1e-5


@pytest.mark.parametrize("lo,hi", [(30.0, 70.0), (37.0, 48.0), (43.0, 69.0), (20.0, 80.0)])
def test_critical_step_scale_bounds_the_table_by_brute_force(lo, hi):
    """s = max(1, max k / k0) * max(1, rho0 c0 / min rho c) over [lo, hi], with
    k0, rho0, c0 the first point: against a dense sample (own extension
    outside the table), equal to within the sampling step."""
    mat = _tab()
    T = np.linspace(lo, hi, 400001)
    Tp = np.array(TAB["T"])

    def ext(v):
        v = np.array(v)
        out = np.interp(T, Tp, v)
        out = np.where(T < Tp[0], v[0] + (v[1] - v[0]) / (Tp[1] - Tp[0]) * (T - Tp[0]), out)
        return np.where(T > Tp[-1], v[-1] + (v[-1] - v[-2]) / (Tp[-1] - Tp[-2]) * (T - Tp[-1]), out)

    k, rc = ext(TAB["k"]), ext(TAB["rho"]) * ext(TAB["c"])
    brute = max(1.0, k.max() / TAB["k"][0]) * max(1.0, TAB["rho"][0] * TAB["c"][0] / rc.min())
    s = td_scale(mat, lo, hi)
    assert s >= brute * (1 - 1e-14)
    assert s == pytest.approx(brute, rel=1e-8)


def test_table_rejects_bad_points():
    with pytest.raises(ValueError):
        Material.tabulated((37.0,), (1000.0,), (3600.0,), (0.5,))
    with pytest.raises(ValueError):
        Material.tabulated((37.0, 37.0), (1000.0, 1000.0), (3600.0, 3600.0), (0.5, 0.5))
    with pytest.raises(ValueError):
        Material.tabulated(tuple(range(9)), (1.0,) * 9, (1.0,) * 9, (1.0,) * 9)
