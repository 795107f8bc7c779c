"""Critical time step of the explicit scheme, Eq. 9: dt_cr = 2 / |lambda_max|.

Oracle code (test infrastructure only).

lambda_max is the largest eigenvalue of the generalised problem
(K + K_b + H) x = lambda C x on the free (non-Dirichlet) nodes, with K
assembled at the reference conductivity k0, K_b = diag(beta) the lumped
perfusion, H = diag(hA) the lumped film condition and C = diag(V rho0 c0).
With temperature-dependent laws (Eq. 2) the paper does not say at which
temperature to take it; the reading used here bounds it over the declared
range [T_lo, T_hi]:

    lambda_TD <= s * lambda_0,  s = max(1, max_T k(T)/k0) * max(1, max_T rho0 c0 / (rho(T) c(T)))

which holds because k_e <= max k makes K(T) <= (max k / k0) K0 in the Loewner
order and C(T) >= min(rho c) / (rho0 c0) C0 elementwise.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .global_form import Oracle


def td_scale(material, T_lo: float, T_hi: float) -> float:
    """The factor s above.  For linear laws rho(T) c(T) is a quadratic in T,
    so its minimum over [T_lo, T_hi] is at an end point or at its vertex; for
    tabulated laws the same holds on every interval, and k is largest at an
    end point or a table point."""
    m = material
    if m.table is not None:
        return _td_scale_table(m, T_lo, T_hi)
    k_max = max(m.k0 + m.dk * (T_lo - m.T_ref), m.k0 + m.dk * (T_hi - m.T_ref))
    cands = [T_lo, T_hi]
    a = m.drho * m.dc                       # rho c = (rho0 + drho u)(c0 + dc u), u = T - T_ref
    if a != 0.0:
        u_v = -(m.rho0 * m.dc + m.c0 * m.drho) / (2.0 * a)
        if T_lo < m.T_ref + u_v < T_hi:
            cands.append(m.T_ref + u_v)
    rc_min = min((m.rho0 + m.drho * (T - m.T_ref)) * (m.c0 + m.dc * (T - m.T_ref)) for T in cands)
    if rc_min <= 0.0:
        raise ValueError("rho(T) c(T) is not positive on the declared range")
    return max(1.0, k_max / m.k0) * max(1.0, m.rho0 * m.c0 / rc_min)


def _td_scale_table(m, T_lo: float, T_hi: float) -> float:
    from .global_form import piecewise_linear
    Tj, rho, c, k = (np.asarray(a, dtype=np.float64) for a in m.table)
    pts = [T_lo, T_hi] + [t for t in Tj if T_lo < t < T_hi]
    k_max = float(np.max(piecewise_linear(Tj, k, np.array(pts))))
    cands = list(pts)
    n = len(Tj)
    for i in range(n - 1):                  # vertex of rho c on interval i (also the extended end ones)
        sr = (rho[i + 1] - rho[i]) / (Tj[i + 1] - Tj[i])
        sc = (c[i + 1] - c[i]) / (Tj[i + 1] - Tj[i])
        if sr * sc != 0.0:
            tv = Tj[i] - (rho[i] * sc + c[i] * sr) / (2.0 * sr * sc)
            lo = -np.inf if i == 0 else Tj[i]
            hi = np.inf if i == n - 2 else Tj[i + 1]
            if max(lo, T_lo) < tv < min(hi, T_hi):
                cands.append(tv)
    cands = np.array(cands)
    rc_min = float(np.min(piecewise_linear(Tj, rho, cands) * piecewise_linear(Tj, c, cands)))
    if rc_min <= 0.0 or np.min(piecewise_linear(Tj, k, np.array(pts))) <= 0.0:
        raise ValueError("rho(T) c(T) or k(T) is not positive on the declared range")
    return max(1.0, k_max / m.k0) * max(1.0, m.rho0 * m.c0 / rc_min)


def region_scale(materials, T_lo: float, T_hi: float) -> float:
    """The factor s for heterogeneous tissue (linear laws), against the
    reference state of the first region's material (k0, rho0 c0):
    s = max(1, max_r max_T k_r / k0) * max(1, rho0 c0 / min_r min_T rho_r c_r).
    It bounds the step as td_scale does: every k_e is at most max k, and
    C_i = sum_r W_ri rho_r c_r is at least min(rho c) V_i."""
    ref = materials[0]
    k_max = max(max(m.k0 + m.dk * (T_lo - m.T_ref), m.k0 + m.dk * (T_hi - m.T_ref)) for m in materials)
    rc_min = min(_rc_min(m, T_lo, T_hi) for m in materials)
    return max(1.0, k_max / ref.k0) * max(1.0, ref.rho0 * ref.c0 / rc_min)


def _rc_min(m, T_lo: float, T_hi: float) -> float:
    """min over [T_lo, T_hi] of rho(T) c(T) for linear laws (end points or the vertex)."""
    if m.table is not None:
        raise ValueError("heterogeneous tissue takes linear laws")
    cands = [T_lo, T_hi]
    a = m.drho * m.dc
    if a != 0.0:
        u_v = -(m.rho0 * m.dc + m.c0 * m.drho) / (2.0 * a)
        if T_lo < m.T_ref + u_v < T_hi:
            cands.append(m.T_ref + u_v)
    rc = min((m.rho0 + m.drho * (T - m.T_ref)) * (m.c0 + m.dc * (T - m.T_ref)) for T in cands)
    if rc <= 0.0:
        raise ValueError("rho(T) c(T) is not positive on the declared range")
    return rc


def reference_operator(orc: Oracle) -> sp.csr_matrix:
    """C0^-1/2 (K0 + K_b + H) C0^-1/2 restricted to free nodes (symmetric).
    Heterogeneous tissue: K0 and C0 at the first region's reference state
    everywhere and K_b at the largest w_b c_b of any region -- an operator that
    bounds every region's from above once scaled by region_scale."""
    m = orc.p.material
    beta = orc.beta
    if orc.regions is not None:
        m = orc.p.region_materials[0]
        beta = max(pf.w_b * pf.c_b for pf in orc.p.region_perfusion) * orc.V
    K0 = orc.assemble_K(np.full(len(orc.conn), m.k0))
    D = sp.diags(beta + orc.hA)
    C0 = orc.V * m.rho0 * m.c0
    f = np.nonzero(orc.free)[0]
    S = sp.diags(1.0 / np.sqrt(C0[f]))
    return (S @ (K0 + D)[f][:, f] @ S).tocsr()


def lambda_max_reference(orc: Oracle, dense_limit: int = 3000) -> float:
    M = reference_operator(orc)
    n = M.shape[0]
    if n == 0:
        return 0.0
    if n <= dense_limit:
        return float(np.linalg.eigvalsh(M.toarray())[-1])
    vals = spla.eigsh(M, k=1, which="LA", tol=1e-13, return_eigenvectors=False)
    return float(vals[0])


def critical_dt(problem_or_oracle, T_lo: float | None = None, T_hi: float | None = None) -> float:
    """dt_cr = 2 / (s * lambda_max(reference)) over [T_lo, T_hi] (default: the
    problem's declared range)."""
    orc = problem_or_oracle if isinstance(problem_or_oracle, Oracle) else Oracle(problem_or_oracle)
    p = orc.p
    T_lo = p.T_lo if T_lo is None else T_lo
    T_hi = p.T_hi if T_hi is None else T_hi
    if p.regions is None:
        s = td_scale(p.material, T_lo, T_hi)
    else:
        s = region_scale(p.region_materials, T_lo, T_hi)
    return 2.0 / (s * lambda_max_reference(orc))


def element_bound_dt(orc: Oracle) -> float:
    """A conservative step at reference properties from two upper bounds:
    lambda_max(K0, C0) <= max_e lambda_max(k0 A_e, diag(V_e rho0 c0 / nv))
    (the element eigenvalue bound, as C0 is the sum of the element shares),
    and, by Weyl's inequality, the diagonal terms add at most
    max_i (beta_i + hA_i) / C0_i."""
    m = orc.p.material
    nv = orc.conn.shape[1]
    ce = orc.V_e * m.rho0 * m.c0 / nv
    lam_e = np.linalg.eigvalsh(m.k0 * orc.A_e)[:, -1] / ce
    C0 = orc.V * m.rho0 * m.c0
    lam_n = np.max((orc.beta + orc.hA)[orc.free] / C0[orc.free]) if orc.free.any() else 0.0
    return 2.0 / (lam_e.max() + lam_n)
