"""Element matrices A_e of Eq. 16 for the two element types of Section 2.3.3.

Oracle code (test infrastructure only).  Every function here is pinned by
tests/test_oracle_elements.py against closed forms: the unit right tetrahedron,
the unit cube, exact gradient energy for affine fields, and the hourglass
null-space of the one-point hexahedron; the fully integrated hexahedron
(2 x 2 x 2 Gauss points) against the textbook unit-cube matrix, exact
energies and volumes of distorted elements, and a null space of constants
only; the hourglass-stabilised one-point hexahedron against the plain rule
at zero strength, linear fields left with exactly the one-point energy on
distorted elements, the closed-form hourglass energy 3 eps h on a cube, and
a null space of constants only.
"""
from __future__ import annotations

import numpy as np

# Trilinear hex8 shape functions N_n = (1 + s_x xi)(1 + s_y eta)(1 + s_z zeta) / 8,
# corner n having natural coordinates s_n in {-1, +1}^3 (bottom face
# counter-clockwise, then top face).
HEX8_NATURAL = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                         [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.float64)


def hex8_dN_dxi_centre() -> np.ndarray:
    """dN_n/dxi_j at xi = eta = zeta = 0, as a (3, 8) array: s_n,j / 8."""
    return HEX8_NATURAL.T / 8.0


def hex8_reduced(xe: np.ndarray):
    """One-point (reduced integration) hexahedron, Eq. 14 and Eq. 16.

    xe: (..., 8, 3) corner coordinates.  J_ij = sum_n x_n,i dN_n/dxi_j is taken
    at the element centre, the single integration point; B = J^-T dN/dxi gives
    the temperature gradient matrix; A = 8 det(J) B^T B.  Returns (A, detJ,
    V_e) with V_e = 8 det J (the reference cube has volume 8)."""
    dN = hex8_dN_dxi_centre()                                  # (3, 8)
    J = np.einsum("...ni,jn->...ij", xe, dN)                   # (..., 3, 3)
    detJ = np.linalg.det(J)
    B = np.einsum("...ji,jn->...in", np.linalg.inv(J), dN)    # J^-T dN: (..., 3, 8)
    A = 8.0 * detJ[..., None, None] * np.einsum("...in,...im->...nm", B, B)
    return A, detJ, 8.0 * detJ


def hex8_full(xe: np.ndarray):
    """Fully integrated hexahedron: A = sum over the 2 x 2 x 2 Gauss points
    (xi, eta, zeta in {-1, +1} / sqrt 3, unit weights) of det J B^T B, with J
    and B = J^-T dN/dxi taken at each point -- the textbook rule, exact for
    the trilinear element's gradient energy, so no hourglass modes remain.
    Returns (A, min det J over the points, V_e = sum of det J)."""
    g = 1.0 / np.sqrt(3.0)
    A = 0.0
    V = 0.0
    dmin = None
    for p in HEX8_NATURAL * g:                                   # the 8 Gauss points
        f = 1.0 + HEX8_NATURAL * p                               # (8, 3): 1 + s_n,j p_j
        dN = np.empty((3, 8))
        dN[0] = HEX8_NATURAL[:, 0] * f[:, 1] * f[:, 2] / 8.0
        dN[1] = HEX8_NATURAL[:, 1] * f[:, 0] * f[:, 2] / 8.0
        dN[2] = HEX8_NATURAL[:, 2] * f[:, 0] * f[:, 1] / 8.0
        J = np.einsum("...ni,jn->...ij", xe, dN)
        detJ = np.linalg.det(J)
        B = np.einsum("...ji,jn->...in", np.linalg.inv(J), dN)
        A = A + detJ[..., None, None] * np.einsum("...in,...im->...nm", B, B)
        V = V + detJ
        dmin = detJ if dmin is None else np.minimum(dmin, detJ)
    return A, dmin, V


# The four hourglass patterns of the hexahedron: products of the corner signs
# (s_x s_y, s_y s_z, s_z s_x, s_x s_y s_z), orthogonal to the constant and to
# each s_d; the one-point rule gives them no energy.
HEX8_HOURGLASS = np.stack([HEX8_NATURAL[:, 0] * HEX8_NATURAL[:, 1], HEX8_NATURAL[:, 1] * HEX8_NATURAL[:, 2],
                           HEX8_NATURAL[:, 2] * HEX8_NATURAL[:, 0],
                           HEX8_NATURAL[:, 0] * HEX8_NATURAL[:, 1] * HEX8_NATURAL[:, 2]])   # (4, 8)


def hex8_hourglass(xe: np.ndarray, eps: float):
    """One-point hexahedron with hourglass stabilisation (the paper keeps
    Eq. 14 and defers hourglass control to another work).  The hourglass
    vectors are made blind to linear fields,
        gamma_a = h_a - sum_i (h_a . x_i) b_i,
    with x_i the corners' i-th coordinates and b_i the i-th row of the
    one-point B (Eq. 14), so that gamma_a . T = 0 for every T linear in x
    (b_i . x_j = delta_ij); then
        A = A_1pt + c sum_a gamma_a gamma_a^T,  c = eps trace(A_1pt) / 32,
    so that on a parallelepiped (gamma_a = h_a, |h_a|^2 = 8) the added
    matrix has eps times the trace of the one-point matrix.  Constant and
    linear fields keep exactly the one-point energy; the four hourglass modes
    get a positive one.  Returns (A, det J, V_e) like hex8_reduced."""
    A1, detJ, V = hex8_reduced(xe)
    dN = hex8_dN_dxi_centre()                                   # (3, 8)
    J = np.einsum("...ni,jn->...ij", xe, dN)
    B = np.einsum("...ji,jn->...in", np.linalg.inv(J), dN)     # (..., 3, 8): b_i rows
    hx = np.einsum("an,...ni->...ai", HEX8_HOURGLASS, xe)        # (..., 4, 3): h_a . x_i
    gamma = HEX8_HOURGLASS - np.einsum("...ai,...in->...an", hx, B)   # (..., 4, 8)
    c = eps * np.trace(A1, axis1=-2, axis2=-1) / 32.0
    A = A1 + c[..., None, None] * np.einsum("...an,...am->...nm", gamma, gamma)
    return A, detJ, V


def tet4_linear(xe: np.ndarray):
    """Linear tetrahedron, Eq. 15 and Eq. 16.

    xe: (..., 4, 3).  With the edge matrix E = [x1-x0, x2-x0, x3-x0] (as
    columns), the barycentric gradients of corners 1..3 are the rows of E^-1
    and the gradient of corner 0 is minus their sum.  V_tet = det(E) / 6 and
    A = V_tet B^T B.  Returns (A, det(E), V_tet)."""
    E = np.swapaxes(xe[..., 1:, :] - xe[..., :1, :], -1, -2)    # (..., 3, 3) columns = edges
    detE = np.linalg.det(E)
    G = np.linalg.inv(E)                                       # rows = grad lambda_1..3
    B = np.concatenate([-G.sum(axis=-2, keepdims=True), G], axis=-2)   # (..., 4, 3)
    V = detE / 6.0
    A = V[..., None, None] * np.einsum("...ni,...mi->...nm", B, B)
    return A, detE, V


def element_matrices(elem_type: int, xyz: np.ndarray, conn: np.ndarray, hex_rule: str = "one-point",
                     hourglass_eps: float = 0.0):
    """A_e, the orientation determinant and V_e for every element of a mesh
    (hex_rule: "one-point", Eq. 14; "full", 2 x 2 x 2 Gauss points; or
    "hourglass", the one-point rule with hourglass stabilisation hourglass_eps).

    Raises ValueError for an element with det <= 0 (inverted or degenerate),
    which the method cannot use (Algorithm 1, pre-computation)."""
    xe = xyz[conn]
    if elem_type == 8 and hex_rule == "full":
        A, det, V = hex8_full(xe)
    elif elem_type == 8 and hex_rule == "hourglass":
        A, det, V = hex8_hourglass(xe, hourglass_eps)
    elif elem_type == 8:
        A, det, V = hex8_reduced(xe)
    elif elem_type == 4:
        A, det, V = tet4_linear(xe)
    else:
        raise ValueError(f"unknown element type {elem_type}")
    bad = np.nonzero(~(det > 0))[0]
    if len(bad):
        raise ValueError(f"element {int(bad[0])} has non-positive Jacobian determinant")
    return A, det, V
