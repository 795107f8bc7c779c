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
// differences of nodal temperatures, or of equally grouped sums of them (G 1 =
// 0, so this is the same product; a uniform field gives exactly zero load).
// k_e is the mean of the nodal k(T_n) (Eq. 13).  Every kernel variant calls
// these functions; fused multiply-adds are written out explicitly and the
// library is built without automatic contraction, so all variants round
// alike.  FP32 work on pairs of values uses the packed f32x2 instructions,
// whose lanes round exactly as the scalar instructions do.
#pragma once

#include <cuda_runtime.h>

namespace fedfem {

template <typename R>
__device__ __forceinline__ R fmadd(R a, R b, R c) { return fma(a, b, c); }

// Packed FP32 pairs: one f32x2 instruction (Blackwell) computes both lanes,
// each rounded to nearest exactly as the scalar instruction rounds it, so a
// packed computation gives the same bits as the scalar one in the same order.
__device__ __forceinline__ unsigned long long pack2(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
    return unpack2(r);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
    return unpack2(r);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
    return unpack2(r);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {   // a * b + c, one rounding
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)), "l"(pack2(c)));
    return unpack2(r);
}

// Four independent problems (scenario lanes) that share a mesh: every
// operation acts on each lane exactly as the scalar code acts on one problem,
// so a lane's result is bit-identical to running that problem alone.  The
// lanes go through the packed instructions two at a time.
struct __align__(16) F4 {
    float x, y, z, w;
};
__device__ __forceinline__ F4 f4(float v) { return F4{v, v, v, v}; }
__device__ __forceinline__ F4 join(float2 a, float2 b) { return F4{a.x, a.y, b.x, b.y}; }
__device__ __forceinline__ float2 lo2(F4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(F4 a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ F4 operator+(F4 a, F4 b) { return join(add2(lo2(a), lo2(b)), add2(hi2(a), hi2(b))); }
__device__ __forceinline__ F4 operator-(F4 a, F4 b) { return join(sub2(lo2(a), lo2(b)), sub2(hi2(a), hi2(b))); }
__device__ __forceinline__ F4 operator*(F4 a, F4 b) { return join(mul2(lo2(a), lo2(b)), mul2(hi2(a), hi2(b))); }
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
    return join(fma2(lo2(a), lo2(b), lo2(c)), fma2(hi2(a), hi2(b), hi2(c)));
}
__device__ __forceinline__ F4 fmadd(float a, F4 b, F4 c) { return fmadd(f4(a), b, c); }
__device__ __forceinline__ F4 fmadd(float a, F4 b, float c) { return fmadd(f4(a), b, f4(c)); }
__device__ __forceinline__ F4 fmadd(F4 a, F4 b, float c) { return fmadd(a, b, f4(c)); }
// max(x, 0): the ramp of one kink of a piecewise-linear law
__device__ __forceinline__ float ramp(float x) { return fmaxf(x, 0.0f); }
__device__ __forceinline__ double ramp(double x) { return fmax(x, 0.0); }
__device__ __forceinline__ float2 ramp(float2 x) { return make_float2(fmaxf(x.x, 0.0f), fmaxf(x.y, 0.0f)); }
__device__ __forceinline__ F4 ramp(F4 x) { return F4{ramp(x.x), ramp(x.y), ramp(x.z), ramp(x.w)}; }
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

// hex8 gradient g = sum_n s_n T_n, corner signs (x,y,z): 0(-,-,-) 1(+,-,-)
// 2(+,+,-) 3(-,+,-) 4(-,-,+) 5(+,-,+) 6(+,+,+) 7(-,+,+).  With the x-pair sums
// a = (t0 + t3, t1 + t2) and b = (t4 + t7, t5 + t6):
//   gx = (a.y + b.y) - (a.x + b.x),
//   gy = ((t3 - t0) + (t7 - t4)) + ((t2 - t1) + (t6 - t5)),
//   gz = (b.x - a.x) + (b.y - a.y);
// every term is a difference of equally grouped sums, so a uniform field
// gives exactly zero.  FP32 computes the pairs with f32x2 instructions.
template <typename L>
__device__ __forceinline__ void hex8_gradient(const L t[8], L& gx, L& gy, L& gz) {
    const L ax = t[0] + t[3], ay = t[1] + t[2], bx = t[4] + t[7], by = t[5] + t[6];
    gx = (ay + by) - (ax + bx);
    gy = ((t[3] - t[0]) + (t[7] - t[4])) + ((t[2] - t[1]) + (t[6] - t[5]));
    gz = (bx - ax) + (by - ay);
}
template <>
__device__ __forceinline__ void hex8_gradient<float>(const float t[8], float& gx, float& gy, float& gz) {
    const float2 p01 = make_float2(t[0], t[1]), p32 = make_float2(t[3], t[2]);
    const float2 p45 = make_float2(t[4], t[5]), p76 = make_float2(t[7], t[6]);
    const float2 a = add2(p01, p32), b = add2(p45, p76);
    const float2 w = add2(a, b), v = sub2(b, a);
    const float2 u = add2(sub2(p32, p01), sub2(p76, p45));
    gx = w.y - w.x;
    gy = u.x + u.y;
    gz = v.x + v.y;
}

// hex8: t[8] nodal temperatures, m[6], k_e already formed -> F[8]
// (R: element-matrix type; L: temperature type, R itself or F4 lanes)
template <typename R, typename L = R>
__device__ __forceinline__ void hex8_loads(const L t[8], const R m[6], L ke, L F[8]) {
    L gx, gy, gz;
    hex8_gradient<L>(t, gx, gy, gz);
    const L qx = ke * fmadd(m[0], gx, fmadd(m[3], gy, m[4] * gz));
    const L qy = ke * fmadd(m[3], gx, fmadd(m[1], gy, m[5] * gz));
    const L qz = ke * fmadd(m[4], gx, fmadd(m[5], gy, m[2] * gz));
    L a = qx + qy, b = qx - qy;
    F[0] = -a - qz;  F[1] = b - qz;  F[2] = a - qz;  F[3] = -b - qz;
    F[4] = -a + qz;  F[5] = b + qz;  F[6] = a + qz;  F[7] = -b + qz;
}

// Hourglass-stabilised one-point hex8.  The four hourglass patterns are the
// sign products h_1 = s_x s_y, h_2 = s_y s_z, h_3 = s_z s_x, h_4 = s_x s_y s_z;
// their amplitudes, made blind to linear fields with the per-element
// weights w (gamma_a = h_a - sum_d w_ad s_d, row-major a x d), are
// q_a = h_a . T - sum_d w_ad g_d with g_d = s_d . T.  With the strength
// c = eps4 trace(M) (eps4 = eps / 4, so that on a parallelepiped the added
// matrix has eps times the trace of the one-point one):
//   F = k_e [ s^T (M g - c W^T q) + c H^T q ].
// Every h_a . T is a sum of four nodal differences (a uniform field gives
// exactly zero).
template <typename R, typename L = R>
__device__ __forceinline__ void hex8_hourglass_loads(const L t[8], const R m[6], const R w[12], R eps4, L ke,
                                                     L F[8]) {
    L g0, g1, g2;
    hex8_gradient<L>(t, g0, g1, g2);
    // corner signs (x,y,z): 0(-,-,-) 1(+,-,-) 2(+,+,-) 3(-,+,-) 4(-,-,+) 5(+,-,+) 6(+,+,+) 7(-,+,+)
    const L h0 = ((t[0] - t[1]) + (t[2] - t[3])) + ((t[4] - t[5]) + (t[6] - t[7]));   // s_x s_y
    const L h1 = ((t[0] - t[2]) + (t[1] - t[3])) + ((t[6] - t[4]) + (t[7] - t[5]));   // s_y s_z
    const L h2 = ((t[0] - t[1]) + (t[3] - t[2])) + ((t[5] - t[4]) + (t[6] - t[7]));   // s_z s_x
    const L h3 = ((t[1] - t[0]) + (t[3] - t[2])) + ((t[4] - t[5]) + (t[6] - t[7]));   // s_x s_y s_z
    const R c = eps4 * ((m[0] + m[1]) + m[2]);
    const L q0 = c * (h0 - fmadd(w[0], g0, fmadd(w[1], g1, w[2] * g2)));
    const L q1 = c * (h1 - fmadd(w[3], g0, fmadd(w[4], g1, w[5] * g2)));
    const L q2 = c * (h2 - fmadd(w[6], g0, fmadd(w[7], g1, w[8] * g2)));
    const L q3 = c * (h3 - fmadd(w[9], g0, fmadd(w[10], g1, w[11] * g2)));
    // gradient flux less the hourglass vectors' linear parts: M g - W^T (c q)
    const L rx = fmadd(w[0], q0, fmadd(w[3], q1, fmadd(w[6], q2, w[9] * q3)));
    const L ry = fmadd(w[1], q0, fmadd(w[4], q1, fmadd(w[7], q2, w[10] * q3)));
    const L rz = fmadd(w[2], q0, fmadd(w[5], q1, fmadd(w[8], q2, w[11] * q3)));
    const L qx = ke * (fmadd(m[0], g0, fmadd(m[3], g1, m[4] * g2)) - rx);
    const L qy = ke * (fmadd(m[3], g0, fmadd(m[1], g1, m[5] * g2)) - ry);
    const L qz = ke * (fmadd(m[4], g0, fmadd(m[5], g1, m[2] * g2)) - rz);
    const L p0 = ke * q0, p1 = ke * q1, p2 = ke * q2, p3 = ke * q3;
    const L a = qx + qy, b = qx - qy;
    // s^T (qx, qy, qz) + H^T (p0 .. p3), corner by corner
    F[0] = (-a - qz) + ((p0 + p1) + (p2 - p3));
    F[1] = (b - qz) + ((p3 - p0) + (p1 - p2));
    F[2] = (a - qz) + ((p0 - p1) - (p2 + p3));
    F[3] = (-b - qz) + ((p2 + p3) - (p0 + p1));
    F[4] = (-a + qz) + ((p0 + p3) - (p1 + p2));
    F[5] = (b + qz) + ((p2 - p0) - (p1 + p3));
    F[6] = (a + qz) + ((p0 + p1) + (p2 + p3));
    F[7] = (-b + qz) + ((p1 - p0) - (p2 + p3));
}

// tet4 factored matrix from corner coordinates (Eq. 15-16, recomputed in the
// time loop instead of read from memory): with the edges a = x1 - x0,
// b = x2 - x0, c = x3 - x0 (the columns of E), the rows of E^-1 are
// (b x c, c x a, a x b) / det E and det E = a . (b x c), so
//   M = V_tet E^-1 E^-T = (r_i . r_j) / (6 det E),  r = (b x c, c x a, a x b).
// x: the four corners (w unused), relative to any common anchor.
__device__ __forceinline__ void tet4_matrix(const float4 x[4], float m[6]) {
    const float ax = x[1].x - x[0].x, ay = x[1].y - x[0].y, az = x[1].z - x[0].z;
    const float bx = x[2].x - x[0].x, by = x[2].y - x[0].y, bz = x[2].z - x[0].z;
    const float cx = x[3].x - x[0].x, cy = x[3].y - x[0].y, cz = x[3].z - x[0].z;
    const float r0x = fmaf(by, cz, -bz * cy), r0y = fmaf(bz, cx, -bx * cz), r0z = fmaf(bx, cy, -by * cx);
    const float r1x = fmaf(cy, az, -cz * ay), r1y = fmaf(cz, ax, -cx * az), r1z = fmaf(cx, ay, -cy * ax);
    const float r2x = fmaf(ay, bz, -az * by), r2y = fmaf(az, bx, -ax * bz), r2z = fmaf(ax, by, -ay * bx);
    const float det = fmaf(ax, r0x, fmaf(ay, r0y, az * r0z));
    const float s = 1.0f / (6.0f * det);
    m[0] = s * fmaf(r0x, r0x, fmaf(r0y, r0y, r0z * r0z));
    m[1] = s * fmaf(r1x, r1x, fmaf(r1y, r1y, r1z * r1z));
    m[2] = s * fmaf(r2x, r2x, fmaf(r2y, r2y, r2z * r2z));
    m[3] = s * fmaf(r0x, r1x, fmaf(r0y, r1y, r0z * r1z));
    m[4] = s * fmaf(r0x, r2x, fmaf(r0y, r2y, r0z * r2z));
    m[5] = s * fmaf(r1x, r2x, fmaf(r1y, r2y, r1z * r2z));
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

// k_e of Eq. 13: mean over the element's nodes of k(T_n)  (K: a law with at()).
// The nodal values are summed as ((k0 + k3) + (k4 + k7)) + ((k1 + k2) + (k5 + k6))
// (hex8) or (k0 + k2) + (k1 + k3) (tet4), the pair order of the packed FP32 path.
template <int NV, typename L>
__device__ __forceinline__ L sum_nodal(const L k[NV]) {
    if constexpr (NV == 8) return ((k[0] + k[3]) + (k[4] + k[7])) + ((k[1] + k[2]) + (k[5] + k[6]));
    else return (k[0] + k[2]) + (k[1] + k[3]);
}
template <typename R, int NV, typename L = R, typename K>
__device__ __forceinline__ L element_k(const L t[NV], const K& k) {
    L kn[NV];
#pragma unroll
    for (int n = 0; n < NV; ++n) kn[n] = k.at(t[n]);
    return R(1) / R(NV) * sum_nodal<NV, L>(kn);
}
// a linear law on FP32 temperatures: k(T) of two nodes per instruction
template <typename R, int NV, typename L = R>
__device__ __forceinline__ float element_k(const float t[NV], const Law<float>& k) {
    const float2 tr = make_float2(k.T_ref, k.T_ref), dp = make_float2(k.dp, k.dp), p0 = make_float2(k.p0, k.p0);
    if constexpr (NV == 8) {
        const float2 k01 = fma2(dp, sub2(make_float2(t[0], t[1]), tr), p0);
        const float2 k32 = fma2(dp, sub2(make_float2(t[3], t[2]), tr), p0);
        const float2 k45 = fma2(dp, sub2(make_float2(t[4], t[5]), tr), p0);
        const float2 k76 = fma2(dp, sub2(make_float2(t[7], t[6]), tr), p0);
        const float2 s = add2(add2(k01, k32), add2(k45, k76));
        return 0.125f * (s.x + s.y);
    } else {
        const float2 k01 = fma2(dp, sub2(make_float2(t[0], t[1]), tr), p0);
        const float2 k23 = fma2(dp, sub2(make_float2(t[2], t[3]), tr), p0);
        const float2 s = add2(k01, k23);
        return 0.25f * (s.x + s.y);
    }
}

}  // namespace fedfem
