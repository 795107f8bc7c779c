"""Pins of the oracle's element matrices (Eq. 14-17) against closed forms.

Each pin is a fact of the finite-element mathematics, not a retyping of the
oracle's formula: exact values on reference elements, exact gradient energy
for affine fields, the rigid null space, the one-point hexahedron's hourglass
null space, and tetrahedral volumes summing to the cube they tile.
"""
import numpy as np
import pytest

from oracle.elements import HEX8_NATURAL, element_matrices, hex8_reduced, tet4_linear
from synth.meshes import KUHN_TETS


def test_unit_right_tet_matches_closed_form():
    xe = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    A, det, V = tet4_linear(xe)
    expect = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    assert V == pytest.approx(1.0 / 6.0, rel=1e-15)
    np.testing.assert_allclose(A, expect, rtol=0, atol=1e-15)


@pytest.mark.parametrize("h", [1.0, 1e-3, 0.37])
def test_unit_cube_hex_matches_sign_outer_product(h):
    xe = (HEX8_NATURAL + 1.0) / 2.0 * h
    A, det, V = hex8_reduced(xe)
    s = HEX8_NATURAL
    # cube of edge h: J = (h/2) I, B = s/(4h)^T ... A_ij = h s_i.s_j / 16
    np.testing.assert_allclose(A, h * (s @ s.T) / 16.0, rtol=1e-14, atol=1e-18 * h)
    assert V == pytest.approx(h ** 3, rel=1e-14)
    ev = np.linalg.eigvalsh(A)
    np.testing.assert_allclose(ev[:5], 0.0, atol=1e-14 * h)
    np.testing.assert_allclose(ev[5:], h / 2.0, rtol=1e-13)


def _random_affine(rng):
    M = rng.normal(size=(3, 3))
    if np.linalg.det(M) < 0:
        M[:, 0] *= -1
    return M, rng.normal(size=3)


def test_affine_fields_exact_energy_and_rigid_nullspace():
    rng = np.random.default_rng(7)
    for _ in range(20):
        M, c = _random_affine(rng)
        # parallelepiped hexahedron: image of the reference cube [-1, 1]^3
        xe = HEX8_NATURAL @ M.T + c
        A, det, V = hex8_reduced(xe)
        assert V == pytest.approx(8.0 * abs(np.linalg.det(M)), rel=1e-12)
        a = rng.normal(size=3)
        T = xe @ a + rng.normal()
        assert T @ A @ T == pytest.approx(V * a @ a, rel=1e-11)
        np.testing.assert_allclose(A @ np.ones(8), 0.0, atol=1e-12 * np.abs(A).max())
        # tetrahedron: image of the unit right tetrahedron
        xt = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) @ M.T + c
        At, dt_, Vt = tet4_linear(xt)
        Tt = xt @ a + 0.3
        assert Vt == pytest.approx(abs(np.linalg.det(M)) / 6.0, rel=1e-12)
        assert Tt @ At @ Tt == pytest.approx(Vt * a @ a, rel=1e-11)
        np.testing.assert_allclose(At @ np.ones(4), 0.0, atol=1e-12 * np.abs(At).max())


def test_kuhn_tets_tile_the_parallelepiped():
    """The six Kuhn tetrahedra of a voxel have total volume equal to the
    voxel's, under any affine map (volumes from Eq. 15's V_tet)."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        M, c = _random_affine(rng)
        xs = KUHN_TETS.astype(float) @ M.T + c
        _, _, V = tet4_linear(xs)
        assert np.all(V > 0)
        assert V.sum() == pytest.approx(abs(np.linalg.det(M)), rel=1e-12)


def test_hex_one_point_hourglass_modes_are_zero_energy():
    """With one integration point the four hourglass patterns s_x s_y,
    s_y s_z, s_z s_x, s_x s_y s_z carry no energy (Eq. 14 has no hourglass
    control), for any parallelepiped."""
    rng = np.random.default_rng(11)
    s = HEX8_NATURAL
    hg = np.stack([s[:, 0] * s[:, 1], s[:, 1] * s[:, 2], s[:, 2] * s[:, 0], s[:, 0] * s[:, 1] * s[:, 2]], axis=1)
    for _ in range(5):
        M, c = _random_affine(rng)
        A, _, _ = hex8_reduced(s @ M.T + c)
        np.testing.assert_allclose(A @ hg, 0.0, atol=1e-12 * np.abs(A).max())
        assert np.linalg.matrix_rank(A, tol=1e-10 * np.abs(A).max()) == 3


def test_inverted_element_is_rejected():
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    with pytest.raises(ValueError):
        element_matrices(4, xyz, np.array([[0, 2, 1, 3]], dtype=np.int32))
    with pytest.raises(ValueError):
        element_matrices(4, xyz, np.array([[0, 1, 2, 2]], dtype=np.int32))


# --- fully integrated hexahedron (2 x 2 x 2 Gauss points) -------------------

def test_full_hex_unit_cube_is_the_textbook_matrix():
    """The trilinear unit cube's exact conduction matrix: 1/3 on the diagonal,
    0 between corners sharing an edge, -1/12 across a face diagonal and across
    the body diagonal."""
    from oracle.elements import hex8_full
    xe = (HEX8_NATURAL + 1.0) / 2.0
    A, _, V = hex8_full(xe)
    s = HEX8_NATURAL
    diff = (s[:, None, :] != s[None, :, :]).sum(axis=2)      # 0 same, 1 edge, 2 face diagonal, 3 body diagonal
    expect = np.select([diff == 0, diff == 1], [1.0 / 3.0, 0.0], -1.0 / 12.0)
    np.testing.assert_allclose(A, expect, rtol=0, atol=1e-15)
    assert V == pytest.approx(1.0, rel=1e-15)


def test_full_hex_frustum_volume_and_affine_energy_are_exact():
    """A square frustum (base 2 x 2, top 1 x 1, height 1, planar faces) has
    volume (4 + 1 + 2) / 3; the full rule integrates the trilinear element's
    det J exactly, so V_e and the energy |g|^2 V_e of an affine field are
    exact, while the one-point rule gives 8 det J(centre) = 9/4."""
    from oracle.elements import hex8_full
    xe = np.array([[-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0],
                   [-.5, -.5, 1], [.5, -.5, 1], [.5, .5, 1], [-.5, .5, 1]], dtype=float)
    A, det_min, V = hex8_full(xe)
    assert V == pytest.approx(7.0 / 3.0, rel=1e-14)
    assert hex8_reduced(xe)[2] == pytest.approx(9.0 / 4.0, rel=1e-14)
    rng = np.random.default_rng(3)
    for _ in range(5):
        g = rng.normal(size=3)
        T = xe @ g + rng.normal()
        assert T @ A @ T == pytest.approx(g @ g * 7.0 / 3.0, rel=1e-12)
    assert det_min > 0


def test_full_hex_has_no_hourglass_modes():
    """Only constants are in the null space: the four hourglass patterns that
    the one-point rule cannot see carry energy, on a cube and a distorted hex."""
    from oracle.elements import hex8_full
    s = HEX8_NATURAL
    hourglass = [s[:, 0] * s[:, 1], s[:, 1] * s[:, 2], s[:, 0] * s[:, 2], s[:, 0] * s[:, 1] * s[:, 2]]
    rng = np.random.default_rng(7)
    cube = (s + 1.0) / 2.0
    for xe in (cube, cube + 0.15 * rng.uniform(-1, 1, size=(8, 3))):
        A, _, _ = hex8_full(xe)
        w = np.linalg.eigvalsh(A)
        assert abs(w[0]) < 1e-14 * w[-1] and w[1] > 1e-3 * w[-1]
        for h in hourglass:
            assert h @ A @ h > 1e-3 * w[-1]
    for h in hourglass:                                         # the one-point rule does not see them
        assert abs(h @ hex8_reduced(cube)[0] @ h) < 1e-14


def test_full_hex_kirchhoff_bar_is_unchanged():
    """A field linear in x inside every element is affine, so both rules give
    it the same exact energy: the Dirichlet bar's steady state under the full
    rule is the same Kirchhoff-transform solution."""
    from oracle import Oracle, critical_dt
    from synth.meshes import box_face_nodes, hex_box
    from synth.problem import Material, Problem
    n, H = 8, 1e-3
    m = hex_box(n, 1, 1, H)
    mat = Material(T_ref=37.0, rho0=1060.0, drho=-1.4286, c0=3600.0, dc=7.14286, k0=0.53, dk=0.02)
    left, right = box_face_nodes(m, ("x0",)), box_face_nodes(m, ("x1",))
    p = Problem(m.elem_type, m.xyz, m.conn, mat, dirichlet_nodes=np.concatenate([left, right]),
                dirichlet_T=np.concatenate([np.full(4, 37.0), np.full(4, 65.0)]), T0=40.0, hex_rule="full")
    orc = Oracle(p)
    T = orc.run(0.9 * critical_dt(orc, 30.0, 70.0), 6000)
    u = lambda t: mat.k0 * (t - 37.0) + 0.5 * mat.dk * (t - 37.0) ** 2   # noqa: E731
    target = u(37.0) + (u(65.0) - u(37.0)) * m.grid_index[:, 0] / n
    expect = 37.0 + (-mat.k0 + np.sqrt(mat.k0 ** 2 + 2 * mat.dk * target)) / mat.dk
    np.testing.assert_allclose(T, expect, rtol=0, atol=1e-10)


# --- hourglass-stabilised one-point hexahedron ---------------------------------

def _distorted_hex(seed):
    from oracle.elements import HEX8_NATURAL
    rng = np.random.default_rng(seed)
    return 0.5e-3 * (HEX8_NATURAL + 1.0) + rng.uniform(-0.12e-3, 0.12e-3, (8, 3))


def test_hourglass_strength_zero_is_the_one_point_rule():
    from oracle.elements import hex8_hourglass, hex8_reduced
    xe = _distorted_hex(1)
    assert np.array_equal(hex8_hourglass(xe, 0.0)[0], hex8_reduced(xe)[0])


def test_hourglass_term_leaves_linear_fields_alone_on_distorted_hexes():
    """gamma_a is orthogonal to every linear field, so A T = A_1pt T for
    T = a + b . x on any element (the patch test the one-point rule passes)."""
    from oracle.elements import hex8_hourglass, hex8_reduced
    rng = np.random.default_rng(2)
    for seed in range(5):
        xe = _distorted_hex(seed)
        A, _, _ = hex8_hourglass(xe, 0.3)
        A1, _, _ = hex8_reduced(xe)
        for _ in range(3):
            T = rng.normal() + xe @ rng.normal(size=3) * 1e3
            np.testing.assert_allclose(A @ T, A1 @ T, rtol=0, atol=1e-13 * np.abs(A).max() * np.abs(T).max())
        np.testing.assert_allclose(A.sum(axis=1), 0.0, atol=1e-15 * np.abs(A).max())


def test_hourglass_energy_on_a_cube_is_three_eps_h():
    """Cube of edge h: A_1pt = (h/16) sum_d s_d s_d^T has trace 3h/2, so
    c = eps (3h/2) / 32; each hourglass pattern h_a has gamma_a = h_a and
    h_a . h_a = 8, giving the energy c * 64 = 3 eps h; different patterns do
    not couple, and the one-point part gives them nothing."""
    from oracle.elements import HEX8_HOURGLASS, HEX8_NATURAL, hex8_hourglass
    h, eps = 2e-3, 0.25
    xe = 0.5 * h * (HEX8_NATURAL + 1.0)
    A, _, _ = hex8_hourglass(xe, eps)
    E = HEX8_HOURGLASS @ A @ HEX8_HOURGLASS.T
    np.testing.assert_allclose(E, 3 * eps * h * np.eye(4), rtol=1e-13, atol=1e-18)


def test_hourglass_element_null_space_is_constants_only():
    from oracle.elements import hex8_hourglass, hex8_reduced
    for seed in range(4):
        xe = _distorted_hex(10 + seed)
        w = np.linalg.eigvalsh(hex8_hourglass(xe, 0.1)[0])
        w1 = np.linalg.eigvalsh(hex8_reduced(xe)[0])
        assert abs(w[0]) < 1e-12 * w[-1] and w[1] > 1e-6 * w[-1]    # one zero: the constant
        assert np.sum(np.abs(w1) < 1e-12 * w1[-1]) == 5                # the plain rule: constant + 4 hourglass


def test_element_matrices_do_not_depend_on_where_the_element_sits():
    """A_e depends on the corners only through their differences (Eq. 15-16),
    so computing it from coordinates relative to any anchor (as a tile's local
    coordinates are) gives the same matrix: a rigid translation by 6 cm
    changes no entry beyond the rounding of the translated coordinates."""
    from oracle.elements import HEX8_NATURAL, hex8_reduced, tet4_linear
    rng = np.random.default_rng(9)
    shift = np.array([0.061, -0.044, 0.037])
    for _ in range(5):
        xt = rng.uniform(0, 1e-3, (4, 3))
        xt[1:] += np.eye(3) * 1e-3                                  # well shaped, positive orientation
        A, _, _ = tet4_linear(xt)
        B, _, _ = tet4_linear(xt + shift)
        np.testing.assert_allclose(B, A, rtol=0, atol=1e-11 * np.abs(A).max())
        xh = 0.5e-3 * (HEX8_NATURAL + 1.0) + rng.uniform(-0.1e-3, 0.1e-3, (8, 3))
        A, _, _ = hex8_reduced(xh)
        B, _, _ = hex8_reduced(xh + shift)
        np.testing.assert_allclose(B, A, rtol=0, atol=1e-11 * np.abs(A).max())
