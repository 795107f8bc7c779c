"""Largest eigenvalue of Eq. 9's operator on a uniform hex8 box, by separation
of variables.

Oracle code (test infrastructure only).  On a box of n^3 cubes of edge h the
one-point hexahedron (Eq. 14) has A_e = (h/16) sum_d s_d s_d^T, and each
corner-sign vector s_d is a Kronecker product of a 1-D pattern (-1, +1) along
d and (1, 1) along the other two axes.  Assembled over the tensor grid:

    K0 = (k0 h / 16) (D (x) S (x) S + S (x) D (x) S + S (x) S (x) D),

with the 1-D assemblies D = sum (-1, 1)(-1, 1)^T and S = sum (1, 1)(1, 1)^T.
The lumped volumes (Section 2.3.4) are h^3 v (x) v (x) v with v = 1/2 at a
boundary node and 1 inside; perfusion is w_b c_b times them; a film on the
z = max face adds h_film h^2 v (x) v (x) e_top.  With Dirichlet nodes on the
four side faces and on z = 0, the free x and y nodes are the interior ones,
where D and S are the Toeplitz matrices tridiag(-1, 2, -1) and
tridiag(1, 2, 1): both are diagonalised by the sine vectors, with eigenvalues
2 -+ 2 cos(i pi / n).  Each pair of x and y modes leaves a symmetric
tridiagonal problem in z (the top node keeps half a row and half a volume),
so lambda_max of Eq. 9 is the largest of (n-1)^2 tridiagonal eigenvalues --
the same number that ``critical_dt`` finds with a dense or Lanczos solver on
the assembled matrices, reached here without assembling anything.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import eigh_tridiagonal

from .critical_dt import td_scale


def lambda_max_hex_box(n: int, h: float, k0: float, rho0c0: float, wbcb: float, h_film: float) -> float:
    """lambda_max of C0^-1/2 (K0 + diag(beta + hA)) C0^-1/2 on the free nodes of
    an n^3 hex box: Dirichlet on x = 0, x = L, y = 0, y = L and z = 0, film
    h_film on z = L (nodes 1 .. n in z are free)."""
    th = np.arange(1, n) * np.pi / n
    d = 2.0 - 2.0 * np.cos(th)            # D on the interior nodes
    s = 2.0 + 2.0 * np.cos(th)            # S on the interior nodes
    # z: nodes 1 .. n; D, S rows of the 1-D assembly (the top node has one element)
    dz_diag = np.full(n, 2.0); dz_diag[-1] = 1.0
    sz_diag = np.full(n, 2.0); sz_diag[-1] = 1.0
    dz_off = np.full(n - 1, -1.0)
    sz_off = np.full(n - 1, 1.0)
    vz = np.ones(n); vz[-1] = 0.5
    c = k0 * h / 16.0
    scale = 1.0 / np.sqrt(rho0c0 * h ** 3 * vz)   # C0^-1/2 on the z line (v = 1 in x and y)
    film = np.zeros(n); film[-1] = h_film * h * h
    best = -np.inf
    for i in range(n - 1):
        for j in range(n - 1):
            a = c * (d[i] * s[j] + s[i] * d[j])    # multiplies S in z
            b = c * s[i] * s[j]                    # multiplies D in z
            diag = a * sz_diag + b * dz_diag + wbcb * h ** 3 * vz + film
            off = a * sz_off + b * dz_off
            lam = eigh_tridiagonal(diag * scale * scale, off * scale[:-1] * scale[1:], eigvals_only=True,
                                   select="i", select_range=(n - 1, n - 1))[0]
            best = max(best, float(lam))
    return best


def critical_dt_hex_box(problem, n: int, h: float) -> float:
    """Eq. 9's dt_cr = 2 / (s lambda_max) for a problem built like
    synth.scenarios.cube_hex_td_convective(n, h) (one material, uniform
    perfusion, film on z = max, Dirichlet on the other five faces)."""
    m = problem.material
    pf = problem.perfusion
    lam = lambda_max_hex_box(n, h, m.k0, m.rho0 * m.c0, pf.w_b * pf.c_b, problem.conv_h)
    return 2.0 / (td_scale(m, problem.T_lo, problem.T_hi) * lam)
