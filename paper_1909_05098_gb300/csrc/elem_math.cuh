// Element conduction loads of Eq. 17, F_e = k_e A_e T_e, in the factored form
// A_e = G^T M_e G that the pre-computation stores (Eq. 16).
//
//  * hex8, one point (Eq. 14): B = J^-T dN/dxi with dN_n/dxi = s_n / 8 at the
//    centre, s_n in {-1,+1}^3 the corner's natural coordinates, so
//    A = 8 det J (s/8)^T J^-1 J^-T (s/8) = s^T M s with M = (det J / 8) J^-1 J^-T;
//  * tet4 (Eq. 15): B = E^-T G, E = [x1-x0, x2-x0, x3-x0], G = [-1 I], so
//    A = G^T M G with M = V_tet E^-1 E^-T.
//
// M is symmetric: stored as m00 m11 m22 m01 m02 m12.  G T is formed from
// differences of nodal temperatures only (G 1 = 0, so this is the same
// product; a uniform field gives exactly zero load).  For the hexahedron each
// gradient component is the sum of the four edge differences along that
// natural direction.  k_e is the mean of the nodal k(T_n) (Eq. 13).  Every
// kernel variant calls these functions; fused multiply-adds are written out
// explicitly and the library is built without automatic contraction, so all
// variants round alike.
#pragma once

#include <cuda_runtime.h>

namespace fedfem {

template <typename R>
__device__ __forceinline__ R fmadd(R a, R b, R c) { return fma(a, b, c); }

// Four independent problems (scenario lanes) that share a mesh: every
// operation acts on each lane exactly as the scalar code acts on one problem,
// so a lane's result is bit-identical to running that problem alone.
struct __align__(16) F4 {
    float x, y, z, w;
};
__device__ __forceinline__ F4 f4(float v) { return F4{v, v, v, v}; }
__device__ __forceinline__ F4 operator+(F4 a, F4 b) { return F4{a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w}; }
__device__ __forceinline__ F4 operator-(F4 a, F4 b) { return F4{a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w}; }
__device__ __forceinline__ F4 operator*(F4 a, F4 b) { return F4{a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w}; }
__device__ __forceinline__ F4 operator/(F4 a, F4 b) { return F4{a.x / b.x, a.y / b.y, a.z / b.z, a.w / b.w}; }

// the explicit increment's quotient r / C: FP64 state divides exactly (IEEE);
// FP32 state uses the fast quotient (a few ulp), far below the rounding of r
// itself and carried into the compensated sum like any other increment
__device__ __forceinline__ double increment_div(double a, double b) { return a / b; }
__device__ __forceinline__ float increment_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ F4 increment_div(F4 a, F4 b) {
    return F4{__fdividef(a.x, b.x), __fdividef(a.y, b.y), __fdividef(a.z, b.z), __fdividef(a.w, b.w)};
}
__device__ __forceinline__ F4 operator-(F4 a) { return F4{-a.x, -a.y, -a.z, -a.w}; }
__device__ __forceinline__ F4 operator+(F4 a, float b) { return a + f4(b); }
__device__ __forceinline__ F4 operator-(F4 a, float b) { return a - f4(b); }
__device__ __forceinline__ F4 operator-(float a, F4 b) { return f4(a) - b; }
__device__ __forceinline__ F4 operator*(float a, F4 b) { return f4(a) * b; }
__device__ __forceinline__ F4 fmadd(F4 a, F4 b, F4 c) {
    return F4{fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y), fmaf(a.z, b.z, c.z), fmaf(a.w, b.w, c.w)};
}
__device__ __forceinline__ F4 fmadd(float a, F4 b, F4 c) { return fmadd(f4(a), b, c); }
__device__ __forceinline__ F4 fmadd(float a, F4 b, float c) { return fmadd(f4(a), b, f4(c)); }
__device__ __forceinline__ F4 fmadd(F4 a, F4 b, float c) { return fmadd(a, b, f4(c)); }
__device__ __forceinline__ bool all_in(F4 v, float lo, float hi) {
    return (v.x >= lo && v.x <= hi) && (v.y >= lo && v.y <= hi) && (v.z >= lo && v.z <= hi) && (v.w >= lo && v.w <= hi);
}
__device__ __forceinline__ bool all_in(float v, float lo, float hi) { return v >= lo && v <= hi; }
__device__ __forceinline__ bool all_in(double v, double lo, double hi) { return v >= lo && v <= hi; }

template <typename R>
struct Law {           // p(T) = p0 + dp (T - T_ref)
    R T_ref, p0, dp;
    __device__ __forceinline__ R operator()(R T) const { return fmadd(dp, T - T_ref, p0); }
    template <typename L>
    __device__ __forceinline__ L at(L T) const { return fmadd(dp, T - T_ref, p0); }
};

// hex8: t[8] nodal temperatures, m[6], k_e already formed -> F[8]
// (R: element-matrix type; L: temperature type, R itself or F4 lanes)
template <typename R, typename L = R>
__device__ __forceinline__ void hex8_loads(const L t[8], const R m[6], L ke, L F[8]) {
    // corner signs (x,y,z): 0(-,-,-) 1(+,-,-) 2(+,+,-) 3(-,+,-) 4(-,-,+) 5(+,-,+) 6(+,+,+) 7(-,+,+);
    // g = sum_n s_n T_n, grouped as edge differences
    const L gx = ((t[1] - t[0]) + (t[2] - t[3])) + ((t[5] - t[4]) + (t[6] - t[7]));
    const L gy = ((t[3] - t[0]) + (t[2] - t[1])) + ((t[7] - t[4]) + (t[6] - t[5]));
    const L gz = ((t[4] - t[0]) + (t[5] - t[1])) + ((t[6] - t[2]) + (t[7] - t[3]));
    const L qx = ke * fmadd(m[0], gx, fmadd(m[3], gy, m[4] * gz));
    const L qy = ke * fmadd(m[3], gx, fmadd(m[1], gy, m[5] * gz));
    const L qz = ke * fmadd(m[4], gx, fmadd(m[5], gy, m[2] * gz));
    L a = qx + qy, b = qx - qy;
    F[0] = -a - qz;  F[1] = b - qz;  F[2] = a - qz;  F[3] = -b - qz;
    F[4] = -a + qz;  F[5] = b + qz;  F[6] = a + qz;  F[7] = -b + qz;
}

// tet4: t[4], m[6], k_e -> F[4]
template <typename R, typename L = R>
__device__ __forceinline__ void tet4_loads(const L t[4], const R m[6], L ke, L F[4]) {
    const L g0 = t[1] - t[0], g1 = t[2] - t[0], g2 = t[3] - t[0];
    const L q0 = ke * fmadd(m[0], g0, fmadd(m[3], g1, m[4] * g2));
    const L q1 = ke * fmadd(m[3], g0, fmadd(m[1], g1, m[5] * g2));
    const L q2 = ke * fmadd(m[4], g0, fmadd(m[5], g1, m[2] * g2));
    F[0] = -((q0 + q1) + q2);
    F[1] = q0; F[2] = q1; F[3] = q2;
}

// k_e of Eq. 13: mean over the element's nodes of k(T_n)  (K: a law with at())
template <typename R, int NV, typename L = R, typename K>
__device__ __forceinline__ L element_k(const L t[NV], const K& k) {
    L s = k.at(t[0]);
#pragma unroll
    for (int n = 1; n < NV; ++n) s = s + k.at(t[n]);
    return R(1) / R(NV) * s;
}

}  // namespace fedfem
