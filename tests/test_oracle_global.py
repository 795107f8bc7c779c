"""Pins of the oracle's assembled step (Eq. 7-8, 11, 13, 19) against closed
forms, exact discrete solutions and conservation laws."""
import copy

import numpy as np
import pytest

from oracle import Oracle, critical_dt
from oracle.global_form import lumped_face_areas
from synth.meshes import box_face_nodes, hex_box, kuhn_tet_box
from synth.problem import GaussianSource, Material, Perfusion, Problem
from synth.scenarios import PERFUSION, TISSUE_CONST, TISSUE_TD, cube_hex_fp64

H = 1e-3


def _problem(mesh, material=TISSUE_CONST, **kw):
    return Problem(mesh.elem_type, mesh.xyz, mesh.conn, material, **kw)


# --- assembly ----------------------------------------------------------------

def test_kuhn_grid_assembles_to_seven_point_stencil():
    """P1 elements on the Kuhn split of a uniform grid give exactly the
    7-point Laplacian (h * [6, -1 x 6]) at interior nodes."""
    n = 4
    m = kuhn_tet_box(n, n, n, H)
    orc = Oracle(_problem(m, Material.constant(1000.0, 4000.0, 1.0)))
    K = orc.assemble_K(np.ones(len(m.conn))).toarray()
    g = m.grid_index
    interior = np.nonzero(np.all((g > 0) & (g < n), axis=1))[0]
    for i in interior:
        row = K[i]
        d = np.abs(g - g[i]).sum(axis=1)
        assert row[i] == pytest.approx(6 * H, rel=1e-12)
        np.testing.assert_allclose(row[d == 1], -H, rtol=1e-12)
        np.testing.assert_allclose(row[d > 1], 0.0, atol=1e-15 * H)


def test_hex_grid_interior_stencil():
    """One-point hex8 on a uniform grid: diagonal 3h/2, face neighbours h/4,
    edge neighbours -h/8, corner neighbours -3h/16 (8 shared-element sums of
    h s_i.s_j / 16)."""
    n = 4
    m = hex_box(n, n, n, H)
    orc = Oracle(_problem(m, Material.constant(1000.0, 4000.0, 1.0)))
    K = orc.assemble_K(np.ones(len(m.conn))).toarray()
    g = m.grid_index
    i = int(np.nonzero(np.all(g == 2, axis=1))[0][0])
    off = np.abs(g - g[i])
    d = off.sum(axis=1)
    near = np.all(off <= 1, axis=1)
    assert K[i, i] == pytest.approx(1.5 * H, rel=1e-12)
    np.testing.assert_allclose(K[i, near & (d == 1)], H / 4, rtol=1e-12)
    np.testing.assert_allclose(K[i, near & (d == 2)], -H / 8, rtol=1e-12)
    np.testing.assert_allclose(K[i, near & (d == 3)], -3 * H / 16, rtol=1e-12)
    assert np.count_nonzero(np.abs(K[i]) > 1e-18) == 27


# --- invariants ----------------------------------------------------------------

@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_uniform_field_is_bit_unchanged(kind):
    m = hex_box(4, 3, 5, H) if kind == "hex" else kuhn_tet_box(3, 4, 3, H)
    faces = np.array([[a, b, c] for a, b, c in m.conn[:6, :3]], dtype=np.int32) if kind == "tet" else \
        m.conn[:4, 4:8]
    dn = box_face_nodes(m, ("x0",))
    p = _problem(m, TISSUE_TD, perfusion=Perfusion(w_b=6.784, c_b=3600.0, T_a=41.5),
                 dirichlet_nodes=dn, dirichlet_T=np.full(len(dn), 41.5),
                 conv_faces=faces, conv_h=10.0, conv_T_inf=41.5, T0=41.5)
    orc = Oracle(p)
    T = orc.run(0.1, 40)
    assert np.all(T == 41.5)


@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_energy_is_conserved_when_insulated(kind):
    rng = np.random.default_rng(5)
    m = hex_box(5, 4, 3, H) if kind == "hex" else kuhn_tet_box(4, 3, 3, H)
    T0 = 37.0 + 5.0 * rng.random(len(m.xyz))
    # temperature-independent: sum C_i T_i is constant
    orc = Oracle(_problem(m, TISSUE_CONST, T0=T0))
    dt = 0.5 * critical_dt(orc, 30.0, 45.0)
    C = orc.capacitance(T0)
    T = orc.run(dt, 200)
    assert np.sum(C * T) == pytest.approx(np.sum(C * T0), rel=1e-13)
    assert np.ptp(T) < np.ptp(T0)
    # temperature-dependent: sum_i C_i(T^n) (T^{n+1}_i - T^n_i) = 0 each step
    orc = Oracle(_problem(m, TISSUE_TD, T0=T0))
    dt = 0.5 * critical_dt(orc, 30.0, 45.0)
    T = orc.initial_field()
    for _ in range(50):
        Tn = orc.step(T, dt)
        C = orc.capacitance(T)
        dE = C * (Tn - T)
        # floor: each T^{n+1} is rounded to an ulp of |T|, weighted by C_i
        assert abs(dE.sum()) <= 4 * np.finfo(float).eps * np.abs(T).max() * C.sum()
        T = Tn


def test_perfusion_and_metabolism_closed_form():
    """Insulated, uniform start, no conduction gradient: every node follows
    T^n = T_eq + (T0 - T_eq)(1 - dt w_b c_b / (rho c))^n, T_eq = T_a + Q_m/(w_b c_b)."""
    m = kuhn_tet_box(3, 3, 2, H)
    pf = Perfusion(w_b=26.6, c_b=3617.0, T_a=39.0, Q_m=33800.0)
    mat = Material.constant(1060.0, 3700.0, 0.518)
    orc = Oracle(_problem(m, mat, perfusion=pf, T0=37.0))
    dt, n = 0.01, 3000
    T = orc.run(dt, n)
    T_eq = pf.T_a + pf.Q_m / (pf.w_b * pf.c_b)
    expect = T_eq + (37.0 - T_eq) * (1 - dt * pf.w_b * pf.c_b / (1060.0 * 3700.0)) ** n
    np.testing.assert_allclose(T, expect, rtol=0, atol=1e-12)


@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_linear_slab_is_a_fixed_point_and_the_limit(kind):
    m = hex_box(6, 2, 2, H) if kind == "hex" else kuhn_tet_box(6, 2, 2, H)
    x = m.xyz[:, 0]
    L = x.max()
    left, right = box_face_nodes(m, ("x0",)), box_face_nodes(m, ("x1",))
    dn = np.concatenate([left, right])
    dT = np.concatenate([np.full(len(left), 30.0), np.full(len(right), 50.0)])
    lin = 30.0 + 20.0 * x / L
    # constant k: with k(T) the linear profile is not steady (see the Kirchhoff pin)
    p = _problem(m, TISSUE_CONST, dirichlet_nodes=dn, dirichlet_T=dT, T0=lin)
    orc = Oracle(p)
    dt = 0.5 * critical_dt(orc, 25.0, 55.0)
    np.testing.assert_allclose(orc.run(dt, 100), lin, rtol=0, atol=1e-12)
    p.T0 = 40.0
    np.testing.assert_allclose(Oracle(p).run(dt, 3000), lin, rtol=0, atol=1e-9)


def test_pennes_bar_exact_discrete_steady_state():
    """A one-element-thick hex bar with Dirichlet ends and perfusion settles
    on the exact solution of the discrete equations,
    T_i = T_a + [u0 sinh(th (n - i)) + un sinh(th i)] / sinh(th n),
    cosh th = 1 + m^2 h^2 / 2, m^2 = w_b c_b / k."""
    n = 10
    m = hex_box(n, 1, 1, H)
    pf = PERFUSION
    left, right = box_face_nodes(m, ("x0",)), box_face_nodes(m, ("x1",))
    T1, T2 = 45.0, 38.0
    p = _problem(m, TISSUE_CONST, perfusion=pf, dirichlet_nodes=np.concatenate([left, right]),
                 dirichlet_T=np.concatenate([np.full(4, T1), np.full(4, T2)]), T0=37.0)
    orc = Oracle(p)
    dt = 0.9 * critical_dt(orc, 30.0, 50.0)
    T = orc.run(dt, 4000)
    m2 = pf.w_b * pf.c_b / TISSUE_CONST.k0
    th = np.arccosh(1 + m2 * H * H / 2)
    i = m.grid_index[:, 0]
    u0, un = T1 - pf.T_a, T2 - pf.T_a
    expect = pf.T_a + (u0 * np.sinh(th * (n - i)) + un * np.sinh(th * i)) / np.sinh(th * n)
    np.testing.assert_allclose(T, expect, rtol=0, atol=1e-10)
    # and the continuous profile is within O(h^2) of it
    mm = np.sqrt(m2)
    cont = pf.T_a + (u0 * np.sinh(mm * (n - i) * H) + un * np.sinh(mm * i * H)) / np.sinh(mm * n * H)
    assert np.max(np.abs(cont - expect)) < 1e-2


def test_temperature_dependent_bar_follows_kirchhoff_transform():
    """With k linear in T and Eq. 13's element average, the steady state of a
    Dirichlet bar has Phi(T_i) = int k dT linear in x_i -- the exact
    Kirchhoff-transform solution at the nodes."""
    n = 8
    m = hex_box(n, 1, 1, H)
    mat = Material(T_ref=37.0, rho0=1060.0, drho=-1.4286, c0=3600.0, dc=7.14286, k0=0.53, dk=0.02)
    left, right = box_face_nodes(m, ("x0",)), box_face_nodes(m, ("x1",))
    T1, T2 = 37.0, 65.0
    p = _problem(m, mat, dirichlet_nodes=np.concatenate([left, right]),
                 dirichlet_T=np.concatenate([np.full(4, T1), np.full(4, T2)]), T0=40.0)
    orc = Oracle(p)
    dt = 0.9 * critical_dt(orc, 30.0, 70.0)
    T = orc.run(dt, 6000)

    def phi(t):
        u = t - mat.T_ref
        return mat.k0 * u + 0.5 * mat.dk * u * u

    s = m.grid_index[:, 0] / n
    target = phi(T1) + (phi(T2) - phi(T1)) * s
    # invert the quadratic Phi for u = T - T_ref
    u = (-mat.k0 + np.sqrt(mat.k0 ** 2 + 2 * mat.dk * target)) / mat.dk
    np.testing.assert_allclose(T, mat.T_ref + u, rtol=0, atol=1e-10)


def test_film_condition_on_single_cube_decays_geometrically():
    """One hex of edge h with a film condition on all six faces: each node
    gets 3 h^2/4 of area and h^3/8 of volume, so a uniform field follows
    T^n = T_inf + (T0 - T_inf)(1 - 6 dt h_c / (h rho c))^n."""
    m = hex_box(1, 1, 1, H)
    faces = m.conn[0][[[0, 3, 2, 1], [4, 5, 6, 7], [0, 1, 5, 4], [1, 2, 6, 5], [2, 3, 7, 6], [3, 0, 4, 7]]]
    hc, Tinf = 150.0, 20.0
    p = _problem(m, TISSUE_CONST, conv_faces=faces.astype(np.int32), conv_h=hc, conv_T_inf=Tinf, T0=37.0)
    orc = Oracle(p)
    np.testing.assert_allclose(lumped_face_areas(m.xyz, faces, 8), 0.75 * H * H, rtol=1e-13)
    dt, n = 0.5, 500
    T = orc.run(dt, n)
    rc = TISSUE_CONST.rho0 * TISSUE_CONST.c0
    expect = Tinf + (37.0 - Tinf) * (1 - 6 * dt * hc / (H * rc)) ** n
    np.testing.assert_allclose(T, expect, rtol=0, atol=1e-12)


def test_sources_integrate_to_the_gaussian_mass_and_enter_the_energy_balance():
    """On a uniform hex grid the lumped volumes are trapezoidal weights, so
    sum_i V_i Q_r(x_i) is the integral peak (2 pi sigma^2)^(3/2) to round-off
    when the box covers +-8 sigma; with insulation and constant properties
    sum C_i T_i then grows by dt * (that + sum of nodal fluxes) per step."""
    sigma = 2.5 * H
    n = 40
    m = hex_box(n, n, n, H)
    c = n * H / 2
    src = GaussianSource((c, c, c), sigma, 4e6)
    p = _problem(m, TISSUE_CONST, sources=[src], flux_nodes=np.array([5, 17], np.int32),
                 flux_q=np.array([0.25, 0.5]), T0=37.0)
    orc = Oracle(p)
    mass = src.peak * (2 * np.pi * sigma ** 2) ** 1.5
    assert orc.Q.sum() == pytest.approx(mass + 0.75, rel=1e-10)
    T0 = orc.initial_field()
    dt = 0.2
    T = orc.run(dt, 5)
    C = orc.capacitance(T0)
    assert np.sum(C * (T - T0)) == pytest.approx(5 * dt * (mass + 0.75), rel=1e-10)


def test_cube_problem_is_stable_and_heats_at_the_source():
    w = cube_hex_fp64()
    orc = Oracle(w.problem)
    dt = 0.5 * critical_dt(orc)
    T = orc.run(dt, 300)
    centre = np.argmin(np.sum((w.problem.xyz - 5e-3) ** 2, axis=1))
    assert T[centre] == T.max() and 40.0 < T.max() < 60.0
    assert np.all(T >= 37.0 - 1e-12)
    q = copy.copy(w.problem)
    q.sources = []
    assert np.all(Oracle(q).run(dt, 50) == 37.0)


def test_temperature_dependent_capacity_converges_to_the_ode_solution():
    """Uniform and insulated, each node obeys rho c(T) dT/dt = w_b c_b (T_a - T).
    With c linear in T this separates: with u = T_a - T and
    a = c0 + dc (T_a - T_ref),  t = rho/(w_b c_b) [a ln(u0/u) + dc (u - u0)].
    Explicit Euler is first order, so Richardson's 2 T(dt/2) - T(dt) must hit
    the closed form to O(dt^2)."""
    from scipy.optimize import brentq
    m = hex_box(2, 1, 1, H)
    mat = Material(T_ref=37.0, rho0=1060.0, drho=0.0, c0=3600.0, dc=-40.0, k0=0.5, dk=0.0)
    pf = Perfusion(w_b=26.6, c_b=3617.0, T_a=45.0)
    p = _problem(m, mat, perfusion=pf, T0=37.0)
    t_end, dt = 30.0, 0.02
    T1 = Oracle(p).run(dt, int(round(t_end / dt)))
    T2 = Oracle(p).run(dt / 2, int(round(t_end / dt * 2)))
    a = mat.c0 + mat.dc * (pf.T_a - mat.T_ref)
    u0 = pf.T_a - 37.0
    tau = mat.rho0 / (pf.w_b * pf.c_b)
    u = brentq(lambda u: tau * (a * np.log(u0 / u) + mat.dc * (u - u0)) - t_end, 1e-9, u0)
    exact = pf.T_a - u
    assert np.max(np.abs(2 * T2 - T1 - exact)) < 1e-6
    assert np.max(np.abs(T2 - exact)) > 1e-5   # the step is coarse enough to be informative


def test_uniform_lumping_reproduces_the_papers_per_node_values():
    """Sections 3.1.3-3.1.4 give every node the share V / N of the liver's
    volume: with their w_b, c_b, Q_m, V and N that is the printed film
    coefficient (per 1 m^2) and nodal heat flow."""
    import json
    import os
    from oracle.global_form import uniform_share
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    pf, mt = g["perfusion_as_film_sec_3_1_3"], g["metabolic_as_nodal_flux_sec_3_1_4"]
    assert pf["w_b"] * pf["c_b"] * uniform_share(pf["V"], pf["n_nodes"]) == pytest.approx(pf["h_printed"], rel=2e-3)
    assert mt["Q_m"] * uniform_share(mt["V"], mt["n_nodes"]) == pytest.approx(mt["q_printed"], rel=5e-3)


def test_uniform_lumping_on_a_uniform_grid_block():
    """On a single hex every node's element share is V / 8 = V / N, so the two
    lumpings coincide; on a larger block the uniform one moves perfusion from
    interior to boundary nodes but keeps its total w_b c_b V, and a uniform
    field at T_a with Q_m = 0 stays exactly unchanged."""
    m1 = hex_box(1, 1, 1, H)
    pf = Perfusion(w_b=26.6, c_b=3617.0, T_a=39.0, Q_m=33800.0)
    base = _problem(m1, TISSUE_CONST, perfusion=pf, T0=37.0)
    uni = copy.copy(base)
    uni.lumping = "uniform"
    np.testing.assert_allclose(Oracle(uni).run(0.05, 200), Oracle(base).run(0.05, 200), rtol=0, atol=1e-13)
    m = hex_box(4, 3, 2, H)
    p = _problem(m, TISSUE_CONST, perfusion=pf, T0=37.0)
    p.lumping = "uniform"
    orc = Oracle(p)
    assert np.ptp(orc.beta) == 0.0 and orc.beta.sum() == pytest.approx(pf.w_b * pf.c_b * orc.V.sum(), rel=1e-13)
    assert orc.Q.sum() == pytest.approx(pf.Q_m * orc.V.sum(), rel=1e-13)
    q = copy.copy(p)
    q.perfusion = Perfusion(w_b=26.6, c_b=3617.0, T_a=37.0, Q_m=0.0)
    assert np.all(Oracle(q).run(0.05, 50) == 37.0)
