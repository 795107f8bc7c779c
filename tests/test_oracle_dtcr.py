"""Pins of the oracle's critical step (Eq. 9) against closed forms."""
import numpy as np
import pytest

from oracle import Oracle, critical_dt, element_bound_dt, td_scale
from synth.meshes import HEX8_CORNERS, hex_box
from synth.problem import Material, Problem
from synth.scenarios import TISSUE_CONST, TISSUE_TD, cube_hex_fp64


def test_cube_closed_form_from_the_one_point_hex_symbol():
    """10^3 cube, Dirichlet on all faces: the one-point hexahedron's discrete
    operator on the interior 9^3 nodes is diagonalised by sine modes
    theta_d = m pi / 10, m = 1..9, with eigenvalue
    (4 alpha / h^2) sum_d sin^2(theta_d/2) prod_{d' != d} cos^2(theta_d'/2)
    plus the perfusion rate w_b c_b / (rho c)."""
    w = cube_hex_fp64()
    p = w.problem
    h = 1e-3
    alpha = p.material.k0 / (p.material.rho0 * p.material.c0)
    th = np.arange(1, 10) * np.pi / 10
    s2, c2 = np.sin(th / 2) ** 2, np.cos(th / 2) ** 2
    S = (s2[:, None, None] * c2[None, :, None] * c2[None, None, :]
         + c2[:, None, None] * s2[None, :, None] * c2[None, None, :]
         + c2[:, None, None] * c2[None, :, None] * s2[None, None, :])
    lam = 4 * alpha / h ** 2 * S.max() + p.perfusion.w_b * p.perfusion.c_b / (p.material.rho0 * p.material.c0)
    assert S.max() == pytest.approx(0.9295351, abs=1e-7)
    assert critical_dt(p) == pytest.approx(2.0 / lam, rel=1e-10)
    assert 2.0 / lam == pytest.approx(3.958280, abs=1e-6)


@pytest.mark.parametrize("h", [1.0, 2e-3])
def test_single_free_elements(h):
    """One free element, no perfusion.  Unit cube: A has eigenvalue h/2 and
    each node h^3/8 of volume, so lambda_max = 4 alpha / h^2.  Right
    tetrahedron of legs h: 6A/h has eigenvalues {0, 1, 1, 4}, each node
    carries h^3/24, so lambda_max = 16 alpha / h^2."""
    mat = Material.constant(1000.0, 4000.0, 0.5)
    alpha = 0.5 / 4e6
    cube = Problem(8, HEX8_CORNERS.astype(float) * h, np.arange(8, dtype=np.int32)[None], mat)
    assert critical_dt(cube, 30, 40) == pytest.approx(2.0 / (4 * alpha / h ** 2), rel=1e-12)
    tet = Problem(4, np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * h,
                  np.arange(4, dtype=np.int32)[None], mat)
    assert critical_dt(tet, 30, 40) == pytest.approx(2.0 / (16 * alpha / h ** 2), rel=1e-12)


def test_td_scale_bounds_the_property_ratios():
    """s = max(1, max k/k0) * max(1, max rho0 c0/(rho c)) checked against a
    dense scan of the range."""
    for mat, lo, hi in [(TISSUE_TD, 25.0, 400.0), (TISSUE_TD, 20.0, 100.0),
                        (Material(37.0, 1040.0, -1.4286, 3600.0, 7.14286, 0.53, 0.0014286), 30.0, 90.0),
                        (Material(37.0, 1000.0, -2.0, 3600.0, 9.0, 0.5, -0.001), 0.0, 150.0),
                        (TISSUE_CONST, 30.0, 40.0)]:
        T = np.linspace(lo, hi, 200001)
        k = mat.k0 + mat.dk * (T - mat.T_ref)
        rc = (mat.rho0 + mat.drho * (T - mat.T_ref)) * (mat.c0 + mat.dc * (T - mat.T_ref))
        brute = max(1.0, k.max() / mat.k0) * max(1.0, (mat.rho0 * mat.c0 / rc).max())
        assert td_scale(mat, lo, hi) == pytest.approx(brute, rel=1e-9)
    assert td_scale(TISSUE_CONST, 30.0, 40.0) == 1.0


def test_element_bound_is_conservative():
    w = cube_hex_fp64()
    orc = Oracle(w.problem)
    assert element_bound_dt(orc) <= critical_dt(orc, 37.0, 37.0)
    m = hex_box(3, 2, 2, 1e-3)
    p = Problem(8, m.xyz * np.array([1.0, 1.7, 0.6]), m.conn, TISSUE_CONST)
    orc = Oracle(p)
    assert element_bound_dt(orc) <= critical_dt(orc, 37.0, 37.0)


def test_explicit_scheme_is_stable_below_and_unstable_above():
    """The defining property of dt_cr: just below it the explicit map is a
    contraction, just above it the top mode grows."""
    m = hex_box(4, 4, 4, 1e-3)
    rng = np.random.default_rng(2)
    p = Problem(8, m.xyz, m.conn, TISSUE_CONST, T0=37.0 + rng.random(len(m.xyz)))
    orc = Oracle(p)
    dt = critical_dt(orc, 37.0, 37.0)
    T0 = orc.initial_field()
    dev0 = np.abs(T0 - T0.mean()).max()
    Tb = orc.run(0.98 * dt, 400)
    Ta = orc.run(1.02 * dt, 400)
    assert np.abs(Tb - Tb.mean()).max() < dev0
    assert np.abs(Ta - Ta.mean()).max() > 10 * dev0


def test_full_hex_critical_step_is_the_tensor_product_symbol():
    """With exact integration the trilinear stiffness on a uniform grid is
    K1 x M1 x M1 + M1 x K1 x M1 + M1 x M1 x K1 (1-D stiffness K1 and consistent
    mass M1), whose Dirichlet modes sin(j pi i / n) have eigenvalues
    (4/h) sin^2(theta/2) and (h/3)(2 + cos theta); with the lumped C = rho c h^3
    and beta = w_b c_b h^3 the largest mode gives dt_cr = 2 / lambda_max."""
    import copy
    p = copy.copy(cube_hex_fp64().problem)
    p.hex_rule = "full"
    m, pf = p.material, p.perfusion
    assert m.dk == 0.0 and m.dc == 0.0 and m.drho == 0.0
    n, h = 10, 1e-3
    th = np.arange(1, n) * np.pi / n
    S = (4.0 / h) * np.sin(th / 2) ** 2
    Mv = (h / 3.0) * (2.0 + np.cos(th))
    lam_K = (S[:, None, None] * Mv[None, :, None] * Mv[None, None, :] + Mv[:, None, None] * S[None, :, None] *
             Mv[None, None, :] + Mv[:, None, None] * Mv[None, :, None] * S[None, None, :])
    lam = (m.k0 * lam_K + pf.w_b * pf.c_b * h ** 3) / (m.rho0 * m.c0 * h ** 3)
    assert critical_dt(Oracle(p)) == pytest.approx(2.0 / lam.max(), rel=1e-12)


def test_uniform_lumping_shifts_the_cube_spectrum_by_a_constant():
    """Uniform lumping gives every free node of the 10^3 cube the perfusion
    w_b c_b V/N with V = (10 h)^3 and N = 11^3, while C stays rho c h^3 on
    every free (interior) node: the one-point symbol of the test above is
    shifted by w_b c_b (V/N) / (rho c h^3) instead of w_b c_b / (rho c)."""
    import copy
    p = copy.copy(cube_hex_fp64().problem)
    p.lumping = "uniform"
    h = 1e-3
    m, pf = p.material, p.perfusion
    alpha = m.k0 / (m.rho0 * m.c0)
    th = np.arange(1, 10) * np.pi / 10
    s2, c2 = np.sin(th / 2) ** 2, np.cos(th / 2) ** 2
    S = (s2[:, None, None] * c2[None, :, None] * c2[None, None, :]
         + c2[:, None, None] * s2[None, :, None] * c2[None, None, :]
         + c2[:, None, None] * c2[None, :, None] * s2[None, None, :])
    share = (10 * h) ** 3 / 11 ** 3
    lam = 4 * alpha / h ** 2 * S.max() + pf.w_b * pf.c_b * share / (m.rho0 * m.c0 * h ** 3)
    assert critical_dt(p) == pytest.approx(2.0 / lam, rel=1e-10)


@pytest.mark.parametrize("n", [3, 5, 8, 11])
def test_box_spectrum_equals_dense_eigenvalue(n):
    """Separation of variables (sine modes in x and y, a tridiagonal problem in
    z) gives the same lambda_max as the dense eigenvalue solver on the
    assembled matrices of the film-topped, five-face-Dirichlet hex box."""
    from oracle.box_spectrum import critical_dt_hex_box
    from synth.scenarios import cube_hex_td_convective
    p = cube_hex_td_convective(n=n).problem
    assert critical_dt_hex_box(p, n, 1e-3) == pytest.approx(critical_dt(p), rel=1e-12)


def test_box_spectrum_without_film_or_perfusion_approaches_the_symbol_maximum():
    """Without film or perfusion the largest eigenvalue grows with n towards
    the one-point hex symbol's supremum 4 alpha / h^2 (the symbol
    (4 alpha / h^2) sum_d sin^2(theta_d / 2) prod_{d' != d} cos^2(theta_d' / 2)
    reaches 1 at theta = (pi, 0, 0), which the Dirichlet box never quite
    samples), staying below it."""
    from oracle.box_spectrum import lambda_max_hex_box
    k0, rc, h = 0.5, 4.0e6, 1e-3
    top = 4.0 * k0 / rc / h ** 2
    prev = 0.0
    for n in (8, 16, 32, 64):
        lam = lambda_max_hex_box(n, h, k0, rc, 0.0, 0.0)
        assert prev < lam < top
        prev = lam
    assert prev > 0.99 * top
