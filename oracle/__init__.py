"""FP64 CPU oracle for the FED-FEM Pennes bio-heat step (Zhang & Chauhan,
arXiv:1909.05098).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it, and the oracle never calls the library: the two share no
kernels, headers, helpers or constants.  Both read the same seeded inputs from
``synth/``, which holds no arithmetic of the method.

The oracle takes the *global, assembled* route of the paper: it forms the
conduction matrix K(T) = sum_e k_e A_e explicitly (Eq. 7, 8, 11), with lumped
(diagonal) capacitance and perfusion (Section 2.3.4), and steps
T <- T + dt C^-1 (Q - K T) (Eq. 8 with the sign reading below).  The GPU path
instead takes the element-level route of Eq. 10-19 and never assembles K.

Readings of the paper it follows (each also listed in the design notes):

* conduction enters with a minus sign: the printed Eq. 7/8/10/18/19 show
  "+K T" / "+F", but Eq. 12 makes F_e = int k B^T B dV T positive
  semi-definite, so "+F" would be anti-diffusive; -F is the physical reading;
* (K T)_i is evaluated as sum_j K_ij (T_j - T_i), equal to (K T)_i because the
  rows of K sum to zero; a uniform field then yields exactly zero;
* perfusion is written beta_i (T_a - T_i) and convection hA_i (T_inf - T_i);
* k_e is the plain mean of the nodal k(T_n) (Eq. 13);
* C_i = V_i rho(T_i) c(T_i) with V_i the lumped volume (mass split equally
  over the element's nodes, Section 2.3.4);
* hex8 elements use one integration point at the element centre (Eq. 14),
  with no hourglass control, and V_e = 8 det J;
* Dirichlet nodes are held at their value from initialisation (Eq. 3) and win
  over any other boundary condition on the same node;
* sources are lumped with the same V_i: Q_i = V_i (Q_m + Q_r(x_i)) + q_i.
"""
from .elements import hex8_reduced, tet4_linear, element_matrices   # noqa: F401
from .global_form import Oracle, arrhenius_increment, cem43_increment, piecewise_linear   # noqa: F401
from .critical_dt import critical_dt, td_scale, element_bound_dt     # noqa: F401
from .metrics import eq20_error, table_stats                          # noqa: F401
from .sampled import sampled_run                                      # noqa: F401
