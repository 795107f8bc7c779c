// Element conduction loads of Eq. 17, F_e = k_e A_e T_e, in the factored form
// A_e = G^T M_e G that the pre-computation stores (Eq. 16).
//
//  * hex8, one point (Eq. 14): B = J^-T dN/dxi with dN_n/dxi = s_n / 8 at the
//    centre, s_n in {-1,+1}^3 the corner's natural coordinates, so
//    A = 8 det J (s/8)^T J^-1 J^-T (s/8) = s^T M s with M = (det J / 8) J^-1 J^-T;
//  * tet4 (Eq. 15): B = E^-T G, E = [x1-x0, x2-x0, x3-x0], G = [-1 I], so
//    A = G^T M G with M = V_tet E^-1 E^-T.
//
// M is symmetric: stored as m00 m11 m22 m01 m02 m12.  The loads act on the
// differences d_n = T_n - T_0 (A 1 = 0 makes this the same product and keeps a
// uniform field exactly load-free).  k_e is the mean of the nodal k(T_n)
// (Eq. 13).  Every kernel variant calls these functions, and the library is
// built without floating-point contraction, so all variants round alike.
#pragma once

#include <cuda_runtime.h>

namespace fedfem {

template <typename R>
struct Law {           // p(T) = p0 + dp (T - T_ref)
    R T_ref, p0, dp;
    __device__ __forceinline__ R operator()(R T) const { return p0 + dp * (T - T_ref); }
};

// hex8: t[8] nodal temperatures, m[6], k_e already formed -> F[8]
template <typename R>
__device__ __forceinline__ void hex8_loads(const R t[8], const R m[6], R ke, R F[8]) {
    R d1 = t[1] - t[0], d2 = t[2] - t[0], d3 = t[3] - t[0];
    R d4 = t[4] - t[0], d5 = t[5] - t[0], d6 = t[6] - t[0], d7 = t[7] - t[0];
    // g = s^T-weighted sums; corner signs (x,y,z):
    // 0(-,-,-) 1(+,-,-) 2(+,+,-) 3(-,+,-) 4(-,-,+) 5(+,-,+) 6(+,+,+) 7(-,+,+), d0 = 0
    R gx = ((d1 + d2) + (d5 + d6)) - ((d3 + d4) + d7);
    R gy = ((d2 + d3) + (d6 + d7)) - ((d1 + d4) + d5);
    R gz = ((d4 + d5) + (d6 + d7)) - ((d1 + d2) + d3);
    R qx = ke * ((m[0] * gx + m[3] * gy) + m[4] * gz);
    R qy = ke * ((m[3] * gx + m[1] * gy) + m[5] * gz);
    R qz = ke * ((m[4] * gx + m[5] * gy) + m[2] * gz);
    R a = qx + qy, b = qx - qy;
    F[0] = -a - qz;  F[1] = b - qz;  F[2] = a - qz;  F[3] = -b - qz;
    F[4] = -a + qz;  F[5] = b + qz;  F[6] = a + qz;  F[7] = -b + qz;
}

// tet4: t[4], m[6], k_e -> F[4]
template <typename R>
__device__ __forceinline__ void tet4_loads(const R t[4], const R m[6], R ke, R F[4]) {
    R g0 = t[1] - t[0], g1 = t[2] - t[0], g2 = t[3] - t[0];
    R q0 = ke * ((m[0] * g0 + m[3] * g1) + m[4] * g2);
    R q1 = ke * ((m[3] * g0 + m[1] * g1) + m[5] * g2);
    R q2 = ke * ((m[4] * g0 + m[5] * g1) + m[2] * g2);
    F[0] = -((q0 + q1) + q2);
    F[1] = q0; F[2] = q1; F[3] = q2;
}

// k_e of Eq. 13: mean over the element's nodes of k(T_n)
template <typename R, int NV>
__device__ __forceinline__ R element_k(const R t[NV], const Law<R>& k) {
    R s = k(t[0]);
#pragma unroll
    for (int n = 1; n < NV; ++n) s = s + k(t[n]);
    return s * (R(1) / R(NV));
}

}  // namespace fedfem
