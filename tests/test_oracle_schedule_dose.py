"""Pins of the oracle's time-varying sources (Algorithm 1's per-step load
update; the two-stage heating and relaxation of Section 3.1.5) and of its
CEM43 thermal dose (the treatment-planning use of Section 5; the published
Sapareto-Dewey definition), against discrete closed forms."""
import copy

import numpy as np
import pytest

from oracle import Oracle, cem43_increment
from synth.meshes import hex_box
from synth.problem import GaussianSource, Material, Perfusion, Problem
from synth.scenarios import cube_hex_fp64


def _insulated_box(Q0=2e6, T0=37.0, schedule=None):
    m = hex_box(3, 2, 2, 1e-3)
    p = Problem(elem_type=8, xyz=m.xyz, conn=m.conn, material=Material.constant(1000.0, 4000.0, 0.5),
                perfusion=Perfusion(), q_r=np.full(len(m.xyz), Q0), T0=T0, T_lo=0.0, T_hi=200.0)
    if schedule is not None:
        p.schedule_end = np.asarray(schedule[0], dtype=np.float64)
        p.schedule_factor = np.asarray(schedule[1], dtype=np.float64)
    return p


def test_schedule_of_ones_equals_no_schedule_and_zeros_equal_no_sources():
    w = cube_hex_fp64()
    p = w.problem
    dt = 0.5
    ref = Oracle(p).run(dt, 60)
    p1 = copy.copy(p)
    p1.schedule_end, p1.schedule_factor = np.array([10.0, 1e9]), np.array([1.0, 1.0])
    T1 = Oracle(p1).run(dt, 60)
    assert np.max(np.abs(T1 - ref)) <= 1e-12 * np.max(np.abs(ref))
    p0 = copy.copy(p)
    p0.schedule_end, p0.schedule_factor = np.array([1e9]), np.array([0.0])
    pn = copy.copy(p)
    pn.sources = []
    assert np.array_equal(Oracle(p0).run(dt, 60), Oracle(pn).run(dt, 60))


@pytest.mark.parametrize("t1,dt,n", [(3.0, 0.01, 2000), (0.255, 0.1, 7)])
def test_two_stage_heating_of_an_insulated_block_is_the_discrete_closed_form(t1, dt, n):
    """Uniform source Q0 for t < t1, then none; insulated, no perfusion,
    constant properties: every node follows T_n = T0 + (dt Q0 / (rho c)) *
    #{k < n : k dt < t1} (Euler with the load of the step's start time)."""
    Q0, T0 = 2e6, 37.0
    p = _insulated_box(Q0, T0, schedule=([t1, 1e9], [1.0, 0.0]))
    T = Oracle(p).run(dt, n)
    n_heat = sum(1 for k in range(n) if k * dt < t1)
    expect = T0 + dt * Q0 / (1000.0 * 4000.0) * n_heat
    assert np.max(np.abs(T - expect)) <= 1e-11 * expect


@pytest.mark.parametrize("Tc,ratio", [(43.0, 1.0), (45.0, 4.0), (41.0, 1.0 / 16.0), (37.0, 0.25 ** 6)])
def test_cem43_of_a_constant_field(Tc, ratio):
    """At a constant temperature the dose after n steps is n dt / 60 R^(43 - T)."""
    w = cube_hex_fp64()
    p = copy.copy(w.problem)
    p.sources = []
    p.T0 = Tc
    p.dirichlet_T = np.full(len(p.dirichlet_nodes), Tc)
    p.perfusion = Perfusion(w_b=p.perfusion.w_b, c_b=p.perfusion.c_b, T_a=Tc, Q_m=0.0)
    dt, n = 0.7, 50
    T, D = Oracle(p).run(dt, n, dose=True)
    assert np.all(T == Tc)
    assert np.allclose(D, n * dt / 60.0 * ratio, rtol=1e-13, atol=0)


def test_cem43_during_linear_heating_is_a_geometric_series():
    """Insulated uniform heating: T_k = T0 + k a.  Below 43 degC the dose is
    (dt/60) 4^-(43 - T0) sum_k 4^(k a) = (dt/60) 4^-(43 - T0) (4^(n a) - 1) / (4^a - 1);
    after the crossing the terms use base 2."""
    Q0, T0, dt, n = 4e6, 40.0, 0.05, 400
    p = _insulated_box(Q0, T0)
    T, D = Oracle(p).run(dt, n, dose=True)
    a = dt * Q0 / (1000.0 * 4000.0)
    k = np.arange(n)
    Tk = T0 + k * a
    below = Tk < 43.0
    nb = int(below.sum())
    q4 = 4.0 ** a
    s_below = 0.25 ** (43.0 - T0) * (q4 ** nb - 1.0) / (q4 - 1.0)
    T_first_above = T0 + nb * a
    q2 = 2.0 ** a
    s_above = 2.0 ** (T_first_above - 43.0) * (q2 ** (n - nb) - 1.0) / (q2 - 1.0)
    expect = dt / 60.0 * (s_below + s_above)
    assert nb > 0 and nb < n
    assert np.max(np.abs(D - expect)) <= 1e-10 * expect
    assert np.allclose(T, T0 + n * a, rtol=1e-12)


def test_cem43_increment_switches_base_at_43():
    d = cem43_increment(np.array([42.999999, 43.0, 43.000001]), 60.0)
    assert d[1] == 1.0
    assert d[0] == pytest.approx(0.25 ** 1e-6, rel=1e-12) and d[2] == pytest.approx(0.5 ** -1e-6, rel=1e-12)


# --- Arrhenius damage integral (Henriques and Moritz) -----------------------
# liver coagulation parameters often used with this model
A_LIVER, EA_LIVER = 7.39e39, 2.577e5


def test_arrhenius_during_linear_heating_meets_the_exponential_integral():
    """Insulated uniform heating at a constant rate h: T(t) = T0 + h t, so
    Omega(t) = (A / h) [F(theta_1) - F(theta_0)] with theta = T + 273.15 K,
    b = Ea / R and F(theta) = theta exp(-b / theta) - b E1(b / theta) (the
    exponential integral).  The oracle sums the rate at each step's start
    temperature, a first-order rule, so Richardson's 2 Omega(dt/2) - Omega(dt)
    meets the closed form to O(dt^2)."""
    from scipy.special import exp1
    from oracle.global_form import GAS_CONSTANT
    Q0, T0, t_end, dt = 4e6, 40.0, 20.0, 0.1
    p = _insulated_box(Q0, T0)
    h = Q0 / (1000.0 * 4000.0)                          # K/s
    _, D1 = Oracle(p).run(dt, int(round(t_end / dt)), dose=("arrhenius", A_LIVER, EA_LIVER))
    T2, D2 = Oracle(p).run(dt / 2, int(round(2 * t_end / dt)), dose=("arrhenius", A_LIVER, EA_LIVER))
    assert np.allclose(T2, T0 + h * t_end, rtol=1e-12)  # 40 -> 60 degC
    b = EA_LIVER / GAS_CONSTANT

    def F(theta):
        return theta * np.exp(-b / theta) - b * exp1(b / theta)

    exact = A_LIVER / h * (F(T0 + h * t_end + 273.15) - F(T0 + 273.15))
    assert 0.1 < exact < 100.0                            # coagulation (Omega = 1) is crossed
    assert np.max(np.abs(2 * D2 - D1 - exact)) <= 1e-4 * exact
    assert np.max(np.abs(D2 - exact)) >= 1e-3 * exact     # the step is coarse enough to be informative


def test_arrhenius_of_a_constant_field_and_its_rate_ratio():
    """At constant T the damage after n steps is n dt A exp(-Ea / (R T_K)),
    and one kelvin more multiplies the rate by exp(b / (T_K (T_K + 1)))."""
    from oracle.global_form import GAS_CONSTANT
    w = cube_hex_fp64()
    out = []
    for Tc in (50.0, 51.0):
        p = copy.copy(w.problem)
        p.sources = []
        p.T0 = Tc
        p.dirichlet_T = np.full(len(p.dirichlet_nodes), Tc)
        p.perfusion = Perfusion(w_b=p.perfusion.w_b, c_b=p.perfusion.c_b, T_a=Tc, Q_m=0.0)
        T, D = Oracle(p).run(0.5, 40, dose=("arrhenius", A_LIVER, EA_LIVER))
        assert np.all(T == Tc) and np.ptp(D) == 0.0
        out.append(D[0])
    b = EA_LIVER / GAS_CONSTANT
    assert out[1] / out[0] == pytest.approx(np.exp(b / (323.15 * 324.15)), rel=1e-12)
    assert out[0] == pytest.approx(40 * 0.5 * A_LIVER * np.exp(-b / 323.15), rel=1e-13)
