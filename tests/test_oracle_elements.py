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
