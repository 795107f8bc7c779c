// Pre-computation stage of Algorithm 1 in FP64 on the GPU:
//   * element geometry: J at the centre (hex8, Eq. 14) or the edge matrix
//     (tet4, Eq. 15), det > 0 check, M_e of the factored A_e (Eq. 16), V_e;
//   * lumped volumes V_i = sum_e V_e / nv (Section 2.3.4), gathered in the
//     fixed slot order; constant loads Q_i = V_i (Q_m + Q_r(x_i)) + q_i;
//     film terms h A_i with A_i = sum_faces area / nverts;
//   * lambda_max of C0^-1/2 (K0 + K_b + H) C0^-1/2 by Lanczos, for dt_cr of Eq. 9;
//   * initial field and read-back (input-order scatter on the device).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "elem_math.cuh"
#include "fedfem_internal.h"

namespace fedfem {
namespace {

constexpr int kThreads = 256;

inline int blocks_for(int64_t n, int t = kThreads) {
    int64_t b = (n + t - 1) / t;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 30));
}

__device__ __forceinline__ void load_conn(const int4* conn4, int64_t E, int64_t e, int nv, int c[8]) {
    int4 a = conn4[e];
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    if (nv == 8) {
        int4 b = conn4[E + e];
        c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
    }
}

__global__ void k_geometry(PreArgs a) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > a.E) return;
    if (e == a.E) { a.Vshare[e] = 0.0; return; }        // zero slot of the gather
    int c[8];
    load_conn(a.conn4, a.E, e, a.nv, c);
    double J[3][3];
    if (a.nv == 8) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) J[i][j] = 0.0;
        for (int n = 0; n < 8; ++n) {
            const double s0 = (n == 1 || n == 2 || n == 5 || n == 6) ? 0.125 : -0.125;
            const double s1 = (n == 2 || n == 3 || n == 6 || n == 7) ? 0.125 : -0.125;
            const double s2 = (n >= 4) ? 0.125 : -0.125;
            const double X[3] = {a.x[c[n]], a.y[c[n]], a.z[c[n]]};
            for (int i = 0; i < 3; ++i) {
                J[i][0] += X[i] * s0;
                J[i][1] += X[i] * s1;
                J[i][2] += X[i] * s2;
            }
        }
    } else {
        const double X0[3] = {a.x[c[0]], a.y[c[0]], a.z[c[0]]};
        for (int j = 0; j < 3; ++j) {
            const int n = c[j + 1];
            J[0][j] = a.x[n] - X0[0];
            J[1][j] = a.y[n] - X0[1];
            J[2][j] = a.z[n] - X0[2];
        }
    }
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (!(det > 0.0)) {
        atomicMin(a.bad_elem, (int)e);
        return;
    }
    // inverse = adjugate / det; adj[j][i] = cofactor[i][j]
    double inv[3][3];
    inv[0][0] = c00 / det; inv[1][0] = c01 / det; inv[2][0] = c02 / det;
    inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    // P = J^-1 J^-T
    double P[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            P[i][j] = inv[i][0] * inv[j][0] + inv[i][1] * inv[j][1] + inv[i][2] * inv[j][2];
    const double w = (a.nv == 8) ? det * 0.125 : det / 6.0;   // hex: det J / 8; tet: V_tet
    const double Ve = (a.nv == 8) ? 8.0 * det : det / 6.0;
    const int64_t E = a.E;
    if (a.nv == 8 && a.W64) {   // hourglass weights w_ad = (1/8) sum_i (h_a . x_i) (J^-1)_di
        double hx[4][3] = {};
        for (int n = 0; n < 8; ++n) {
            const double sx = (n == 1 || n == 2 || n == 5 || n == 6) ? 1.0 : -1.0;
            const double sy = (n == 2 || n == 3 || n == 6 || n == 7) ? 1.0 : -1.0;
            const double sz = (n >= 4) ? 1.0 : -1.0;
            const double h[4] = {sx * sy, sy * sz, sz * sx, sx * sy * sz};
            const double X[3] = {a.x[c[n]], a.y[c[n]], a.z[c[n]]};
            for (int q = 0; q < 4; ++q)
                for (int i = 0; i < 3; ++i) hx[q][i] += h[q] * X[i];
        }
        for (int q = 0; q < 4; ++q)
            for (int d = 0; d < 3; ++d)
                a.W64[(3 * q + d) * E + e] = 0.125 * (hx[q][0] * inv[d][0] + hx[q][1] * inv[d][1] + hx[q][2] * inv[d][2]);
    }
    a.M64[0 * E + e] = w * P[0][0];
    a.M64[1 * E + e] = w * P[1][1];
    a.M64[2 * E + e] = w * P[2][2];
    a.M64[3 * E + e] = w * P[0][1];
    a.M64[4 * E + e] = w * P[0][2];
    a.M64[5 * E + e] = w * P[1][2];
    a.Vshare[e] = Ve / a.nv;
}

// Fully integrated hex8: A_e = sum over the 2 x 2 x 2 Gauss points
// (natural coordinates +-1/sqrt 3, unit weights) of det J B^T B, B = J^-T
// dN/dxi at the point; V_e = sum of det J (exact for the trilinear element).
// Writes the 28 entries a < b (pair order a-major) and V_e / 8; an element
// with det J <= 0 at any point is reported like an inverted one.
__global__ void k_geometry_full(PreArgs a) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.E) return;
    int c[8];
    load_conn(a.conn4, a.E, e, 8, c);
    double X[8][3];
    for (int n = 0; n < 8; ++n) { X[n][0] = a.x[c[n]]; X[n][1] = a.y[c[n]]; X[n][2] = a.z[c[n]]; }
    double A[28];
    for (int q = 0; q < 28; ++q) A[q] = 0.0;
    double V = 0.0;
    bool bad = false;
    const double gp = 0.57735026918962576451;   // 1 / sqrt 3
    for (int g = 0; g < 8; ++g) {
        const double p0 = (g == 1 || g == 2 || g == 5 || g == 6) ? gp : -gp;
        const double p1 = (g == 2 || g == 3 || g == 6 || g == 7) ? gp : -gp;
        const double p2 = (g >= 4) ? gp : -gp;
        double dN[3][8];
        for (int n = 0; n < 8; ++n) {
            const double s0 = (n == 1 || n == 2 || n == 5 || n == 6) ? 1.0 : -1.0;
            const double s1 = (n == 2 || n == 3 || n == 6 || n == 7) ? 1.0 : -1.0;
            const double s2 = (n >= 4) ? 1.0 : -1.0;
            const double f0 = 1.0 + s0 * p0, f1 = 1.0 + s1 * p1, f2 = 1.0 + s2 * p2;
            dN[0][n] = 0.125 * s0 * f1 * f2;
            dN[1][n] = 0.125 * s1 * f0 * f2;
            dN[2][n] = 0.125 * s2 * f0 * f1;
        }
        double J[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double t = 0.0;
                for (int n = 0; n < 8; ++n) t += X[n][i] * dN[j][n];
                J[i][j] = t;
            }
        const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        if (!(det > 0.0)) { bad = true; break; }
        double inv[3][3];   // inverse = adjugate / det
        inv[0][0] = c00 / det; inv[1][0] = c01 / det; inv[2][0] = c02 / det;
        inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        double B[3][8];     // grad N_n = J^-T dN/dxi: B[i][n] = sum_j inv[j][i] dN[j][n]
        for (int i = 0; i < 3; ++i)
            for (int n = 0; n < 8; ++n) B[i][n] = inv[0][i] * dN[0][n] + inv[1][i] * dN[1][n] + inv[2][i] * dN[2][n];
        int q = 0;
        for (int m = 0; m < 8; ++m)
            for (int n = m + 1; n < 8; ++n, ++q) A[q] += det * (B[0][m] * B[0][n] + B[1][m] * B[1][n] + B[2][m] * B[2][n]);
        V += det;
    }
    if (bad) {
        atomicMin(a.bad_elem, (int)e);
        return;
    }
    for (int q = 0; q < 28; ++q) a.A28[q * a.E + e] = A[q];
    a.Vshare[e] = V / 8.0;
}

__global__ void k_faces(PreArgs a) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= a.n_faces) return;
    const int32_t* v = a.faces + f * a.face_nv;
    double p[4][3];
    for (int k = 0; k < a.face_nv; ++k) { p[k][0] = a.x[v[k]]; p[k][1] = a.y[v[k]]; p[k][2] = a.z[v[k]]; }
    double u[3], w[3];
    for (int d = 0; d < 3; ++d) {
        if (a.face_nv == 3) { u[d] = p[1][d] - p[0][d]; w[d] = p[2][d] - p[0][d]; }
        else { u[d] = p[2][d] - p[0][d]; w[d] = p[3][d] - p[1][d]; }   // the two diagonals
    }
    const double cx = u[1] * w[2] - u[2] * w[1];
    const double cy = u[2] * w[0] - u[0] * w[2];
    const double cz = u[0] * w[1] - u[1] * w[0];
    const double area = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
    a.face_share[f] = a.h_film * (area / a.face_nv);
}

__global__ void k_nodal(PreArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N_free) return;
    const int64_t s = i >> 5;
    const int lane = (int)(i & 31);
    const int32_t off = a.sell_off[s];
    const int w = (a.sell_off[s + 1] - off) >> 5;
    double V = 0.0;
    for (int k = 0; k < w; ++k) V += a.Vshare[a.sell_ids[off + 32 * k + lane] / a.nv];
    a.V[i] = V;
    const double X = a.x[i], Y = a.y[i], Z = a.z[i];
    for (int l = 0; l < a.n_lanes; ++l) {      // scenario lanes share V, differ in sources
        double q = 0.0;
        const int grp = a.node_group ? a.node_group[i] : -1;
        for (int j = 0; j < a.n_src; ++j) {
            const double* S = a.src + 7 * j;
            if (S[5] >= 0.0 && (int)S[5] != l) continue;
            if (S[6] >= 0.0 && (int)S[6] != grp) continue;
            const double r2 = (X - S[0]) * (X - S[0]) + (Y - S[1]) * (Y - S[1]) + (Z - S[2]) * (Z - S[2]);
            q += S[4] * exp(-r2 / (2.0 * S[3] * S[3]));
        }
        if (a.qr_node) q += a.qr_node[l * a.N_free + i];
        double Q = V * (a.Q_m + q);
        if (a.flux_node) Q += a.flux_node[i];
        a.Q[l * a.N_free + i] = Q;
    }
    if (i >= a.N_plain) {
        const int64_t c = i - a.N_plain;
        double hA = 0.0;
        for (int32_t p = a.conv_off[c]; p < a.conv_off[c + 1]; ++p) hA += a.face_share[a.conv_face[p]];
        a.hA[c] = hA;
    }
}

// Heterogeneous tissue: for every free node, the sums over its elements (the
// node's slot list) of the element share V_e / nv times its region's
// coefficients coef[5 r + q]: rho c = q0 + q1 u + q2 u^2, w_b c_b (q3) and
// Q_m (q4).  Cq receives the first four as planes of N_free; the metabolic
// sum is added to every lane's load.
__global__ void k_regions(PreArgs a, const unsigned char* emat, const double* coef, double* Cq) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N_free) return;
    const int64_t s = i >> 5;
    const int lane = (int)(i & 31);
    const int32_t off = a.sell_off[s];
    const int w = (a.sell_off[s + 1] - off) >> 5;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < w; ++k) {
        const int64_t e = a.sell_ids[off + 32 * k + lane] / a.nv;
        if (e >= a.E) continue;   // pad slot
        const double v = a.Vshare[e];
        const double* q = coef + 5 * (int)emat[e];
#pragma unroll
        for (int j = 0; j < 5; ++j) acc[j] += v * q[j];
    }
    for (int j = 0; j < 4; ++j) Cq[j * a.N_free + i] = acc[j];
    for (int l = 0; l < a.n_lanes; ++l) a.Q[l * a.N_free + i] += acc[4];
}

__global__ void k_to_f32(const double* src, float* dst, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}

__global__ void k_pack_lanes(const double* src, float* dst, int n_lanes, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int l = 0; l < n_lanes; ++l) dst[i * n_lanes + l] = (float)src[l * n + i];
}

// ---- Lanczos pieces (FP64) --------------------------------------------------

struct LzArgs {
    PreArgs p;
    double k0;
    double* u;        // N: C0^-1/2 v on free nodes, 0 on Dirichlet nodes
    double* slots;    // E*nv + 1
    const double* sinv;   // N_free: C0^-1/2
    const double* diag;   // N_free: beta + hA
    const double* v;
    double* w;
};

__global__ void k_lz_prep(double* sinv, double* diag, const double* V, const double* hA, int64_t N_free,
                          int64_t N_plain, double rho0c0, double wbcb, const double* beta) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N_free) return;
    sinv[i] = 1.0 / sqrt(V[i] * rho0c0);
    diag[i] = (beta ? beta[i] : wbcb * V[i]) + (i >= N_plain ? hA[i - N_plain] : 0.0);
}

__global__ void k_lz_scatter(LzArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.p.N_free) a.u[i] = a.sinv[i] * a.v[i];
}

__global__ void k_lz_elem(LzArgs a) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.p.E) return;
    const int64_t E = a.p.E;
    double m[6];
    for (int j = 0; j < 6; ++j) m[j] = a.p.M64[j * E + e];
    int c[8];
    load_conn(a.p.conn4, E, e, a.p.nv, c);
    if (a.p.nv == 8 && a.p.A28) {   // fully integrated: F_m = k0 sum_n A_mn (u_n - u_m)
        double t[8], F[8];
        for (int n = 0; n < 8; ++n) { t[n] = a.u[c[n]]; F[n] = 0.0; }
        int q = 0;
        for (int m2 = 0; m2 < 8; ++m2)
            for (int n = m2 + 1; n < 8; ++n, ++q) {
                const double w = a.p.A28[q * E + e] * (t[n] - t[m2]);
                F[m2] += w;
                F[n] -= w;
            }
        for (int n = 0; n < 8; ++n) a.slots[e * 8 + n] = a.k0 * F[n];
    } else if (a.p.nv == 8 && a.p.W64) {   // hourglass-stabilised one-point rule
        double t[8], F[8], w[12];
        for (int n = 0; n < 8; ++n) t[n] = a.u[c[n]];
        for (int q = 0; q < 12; ++q) w[q] = a.p.W64[q * E + e];
        hex8_hourglass_loads<double>(t, m, w, a.p.hg_eps4, a.k0, F);
        for (int n = 0; n < 8; ++n) a.slots[e * 8 + n] = F[n];
    } else if (a.p.nv == 8) {
        double t[8], F[8];
        for (int n = 0; n < 8; ++n) t[n] = a.u[c[n]];
        hex8_loads<double>(t, m, a.k0, F);
        for (int n = 0; n < 8; ++n) a.slots[e * 8 + n] = F[n];
    } else {
        double t[4], F[4];
        for (int n = 0; n < 4; ++n) t[n] = a.u[c[n]];
        tet4_loads<double>(t, m, a.k0, F);
        for (int n = 0; n < 4; ++n) a.slots[e * 4 + n] = F[n];
    }
}

__global__ void k_lz_node(LzArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.p.N_free) return;
    const int64_t s = i >> 5;
    const int lane = (int)(i & 31);
    const int32_t off = a.p.sell_off[s];
    const int w = (a.p.sell_off[s + 1] - off) >> 5;
    double F = 0.0;
    for (int k = 0; k < w; ++k) F += a.slots[a.p.sell_ids[off + 32 * k + lane]];
    a.w[i] = a.sinv[i] * (F + a.diag[i] * a.u[i]);
}

constexpr int kRedBlocks = 512;

__global__ void k_dot_partial(const double* x, const double* y, int64_t n, double* part) {
    __shared__ double sh[kThreads];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += x[i] * y[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_final(const double* part, int n, double* out) {
    __shared__ double sh[kThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// w <- w - alpha v - beta vprev
__global__ void k_lz_orth(double* w, const double* v, const double* vprev, double alpha, double beta, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = (w[i] - alpha * v[i]) - beta * vprev[i];
}

// vprev <- v; v <- w / beta
__global__ void k_lz_shift(double* vprev, double* v, const double* w, double inv_beta, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { vprev[i] = v[i]; v[i] = w[i] * inv_beta; }
}

// deterministic start vector: splitmix64 of the index, mapped to (-1, 1)
__global__ void k_lz_start(double* v, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = (unsigned long long)i + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    v[i] = ((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0 + 1e-3;
}

// Largest eigenvalue of the symmetric tridiagonal (a, b) by Sturm-count bisection.
double tridiag_max(const std::vector<double>& a, const std::vector<double>& b) {
    const int m = (int)a.size();
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < m; ++i) {
        double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    auto n_below = [&](double x) {
        int cnt = 0;
        double d = a[0] - x;
        if (d < 0) ++cnt;
        for (int i = 1; i < m; ++i) {
            const double dd = (d == 0.0) ? 1e-300 : d;
            d = (a[i] - x) - b[i - 1] * b[i - 1] / dd;
            if (d < 0) ++cnt;
        }
        return cnt;
    };
    for (int it = 0; it < 200 && hi - lo > 1e-16 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (n_below(mid) == m) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

cudaError_t launch_geometry(const PreArgs& a, cudaStream_t s) {
    k_geometry<<<blocks_for(a.E + 1), kThreads, 0, s>>>(a);
    if (a.n_faces > 0) k_faces<<<blocks_for(a.n_faces), kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_geometry_full(const PreArgs& a, cudaStream_t s) {
    if (a.E > 0) k_geometry_full<<<blocks_for(a.E), kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_nodal(const PreArgs& a, cudaStream_t s) {
    if (a.N_free > 0) k_nodal<<<blocks_for(a.N_free), kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_regions(const PreArgs& a, const unsigned char* emat, const double* coef, double* Cq,
                           cudaStream_t s) {
    if (a.N_free > 0) k_regions<<<blocks_for(a.N_free), kThreads, 0, s>>>(a, emat, coef, Cq);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* src, float* dst, int64_t n, cudaStream_t s) {
    if (n > 0) k_to_f32<<<blocks_for(n), kThreads, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_pack_lanes(const double* src, float* dst, int n_lanes, int64_t n, cudaStream_t s) {
    if (n > 0) k_pack_lanes<<<blocks_for(n), kThreads, 0, s>>>(src, dst, n_lanes, n);
    return cudaGetLastError();
}

std::string lanczos_lambda_max(const PreArgs& p, double k0, double rho0c0, double wbcb, const double* beta, int max_iter,
                               double rel_tol, LanczosResult& out, cudaStream_t s) {
    const int64_t n = p.N_free;
    out = LanczosResult();
    if (n == 0) return "";
    double *u = nullptr, *slots = nullptr, *sinv = nullptr, *diag = nullptr, *v = nullptr, *vp = nullptr,
           *w = nullptr, *part = nullptr, *res = nullptr;
    auto cleanup = [&]() {
        cudaFree(u); cudaFree(slots); cudaFree(sinv); cudaFree(diag); cudaFree(v); cudaFree(vp);
        cudaFree(w); cudaFree(part); cudaFree(res);
    };
#define LZ_CHECK(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) { cleanup(); return std::string("lanczos: ") + cudaGetErrorString(_e); } } while (0)
    LZ_CHECK(cudaMalloc(&u, sizeof(double) * p.N));
    LZ_CHECK(cudaMalloc(&slots, sizeof(double) * (p.E * p.nv + 1)));
    LZ_CHECK(cudaMalloc(&sinv, sizeof(double) * n));
    LZ_CHECK(cudaMalloc(&diag, sizeof(double) * n));
    LZ_CHECK(cudaMalloc(&v, sizeof(double) * n));
    LZ_CHECK(cudaMalloc(&vp, sizeof(double) * n));
    LZ_CHECK(cudaMalloc(&w, sizeof(double) * n));
    LZ_CHECK(cudaMalloc(&part, sizeof(double) * kRedBlocks));
    LZ_CHECK(cudaMalloc(&res, sizeof(double)));
    LZ_CHECK(cudaMemsetAsync(u, 0, sizeof(double) * p.N, s));
    LZ_CHECK(cudaMemsetAsync(slots, 0, sizeof(double) * (p.E * p.nv + 1), s));
    LZ_CHECK(cudaMemsetAsync(vp, 0, sizeof(double) * n, s));
    k_lz_prep<<<blocks_for(n), kThreads, 0, s>>>(sinv, diag, p.V, p.hA, n, p.N_plain, rho0c0, wbcb, beta);
    k_lz_start<<<blocks_for(n), kThreads, 0, s>>>(v, n);
    LZ_CHECK(cudaGetLastError());
    const int rb = (int)std::min<int64_t>(kRedBlocks, (n + kThreads - 1) / kThreads);
    auto dot = [&](const double* x, const double* y, double& r) -> cudaError_t {
        k_dot_partial<<<rb, kThreads, 0, s>>>(x, y, n, part);
        k_sum_final<<<1, kThreads, 0, s>>>(part, rb, res);
        cudaError_t e = cudaMemcpyAsync(&r, res, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return e;
        return cudaStreamSynchronize(s);
    };
    double nrm2 = 0;
    LZ_CHECK(dot(v, v, nrm2));
    k_lz_shift<<<blocks_for(n), kThreads, 0, s>>>(vp, v, v, 1.0 / std::sqrt(nrm2), n);
    LZ_CHECK(cudaMemsetAsync(vp, 0, sizeof(double) * n, s));
    LzArgs la{p, k0, u, slots, sinv, diag, v, w};
    std::vector<double> al, be;
    double beta_prev = 0.0, theta_prev = 0.0;
    int stable = 0;
    for (int j = 0; j < max_iter && j < n; ++j) {
        k_lz_scatter<<<blocks_for(n), kThreads, 0, s>>>(la);
        k_lz_elem<<<blocks_for(p.E), kThreads, 0, s>>>(la);
        k_lz_node<<<blocks_for(n), kThreads, 0, s>>>(la);
        LZ_CHECK(cudaGetLastError());
        double alpha = 0;
        LZ_CHECK(dot(w, v, alpha));
        k_lz_orth<<<blocks_for(n), kThreads, 0, s>>>(w, v, vp, alpha, beta_prev, n);
        double bb = 0;
        LZ_CHECK(dot(w, w, bb));
        const double beta = std::sqrt(std::max(bb, 0.0));
        al.push_back(alpha);
        const double theta = tridiag_max(al, be);
        out.iterations = j + 1;
        out.lambda = theta;
        if (j > 0 && std::fabs(theta - theta_prev) <= rel_tol * std::fabs(theta)) ++stable; else stable = 0;
        theta_prev = theta;
        if (stable >= 5) break;
        if (!(beta > 1e-13 * std::fabs(theta))) break;   // invariant subspace found: exact
        be.push_back(beta);
        k_lz_shift<<<blocks_for(n), kThreads, 0, s>>>(vp, v, w, 1.0 / beta, n);
        LZ_CHECK(cudaGetLastError());
        beta_prev = beta;
    }
#undef LZ_CHECK
    cleanup();
    return "";
}

// ---- initial state and read-back ---------------------------------------------

namespace {
__global__ void k_init64(int64_t N, int64_t N_free, const int32_t* node_of, const double* T_in,
                         const double* T_dir, double* T) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) T[i] = (i >= N_free) ? T_dir[i - N_free] : T_in[node_of[i]];
}
// FP32 state interleaved by lane: T[i * n_lanes + lane]
__global__ void k_init32(int n_lanes, int64_t N, int64_t N_free, const int32_t* node_of, const double* T_in,
                         const double* T_dir, float* T, float* Tlo, bool kahan) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int l = 0; l < n_lanes; ++l) {
        const double v = (i >= N_free) ? T_dir[i - N_free] : T_in[l * N + node_of[i]];
        const float hi = (float)v;
        T[i * n_lanes + l] = hi;
        Tlo[i * n_lanes + l] = kahan ? (float)(v - (double)hi) : 0.0f;
    }
}
__global__ void k_read64(int64_t N, const int32_t* node_of, const double* T, double* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[node_of[i]] = T[i];
}
__global__ void k_read32(int n_lanes, int lane, int64_t N, const int32_t* node_of, const float* T, const float* Tlo,
                         double* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[node_of[i]] = (double)T[i * n_lanes + lane] + (double)Tlo[i * n_lanes + lane];
}
}  // namespace

cudaError_t launch_init_state(int precision, int n_lanes, int64_t N, int64_t N_free, const int32_t* node_of,
                              const double* T_in, const double* T_dir, void* T, float* Tlo, cudaStream_t s) {
    if (precision == FEDFEM_FP64)
        k_init64<<<blocks_for(N), kThreads, 0, s>>>(N, N_free, node_of, T_in, T_dir, (double*)T);
    else
        k_init32<<<blocks_for(N), kThreads, 0, s>>>(n_lanes, N, N_free, node_of, T_in, T_dir, (float*)T, Tlo,
                                                    precision == FEDFEM_FP32_KAHAN);
    return cudaGetLastError();
}

cudaError_t launch_read_state(int precision, int n_lanes, int lane, int64_t N, const int32_t* node_of,
                              const void* T, const float* Tlo, double* out, cudaStream_t s) {
    if (precision == FEDFEM_FP64)
        k_read64<<<blocks_for(N), kThreads, 0, s>>>(N, node_of, (const double*)T, out);
    else
        k_read32<<<blocks_for(N), kThreads, 0, s>>>(n_lanes, lane, N, node_of, (const float*)T, Tlo, out);
    return cudaGetLastError();
}

}  // namespace fedfem

// ---- FP64 pipe throughput (measurement helper) ----------------------------
// Eight independent chains of fused multiply-adds per thread, so that every
// FP64 unit has work each cycle; the sum goes to a sink so that nothing is
// optimised away.  FLOPs = 2 * 8 * iterations * threads.
namespace fedfem {
namespace {
__global__ void k_fp64_fma_loop(long long iterations, double* sink) {
    const double b = 0.9999999999, c = 1e-9;
    double x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = 1.0 + 1e-3 * (q + (double)threadIdx.x * 1e-6);
    for (long long k = 0; k < iterations; ++k) {
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = fma(x[q], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += x[q];
    if (s == 12345.678) sink[blockIdx.x] = s;   // never true; keeps the chains live
}
}  // namespace
}  // namespace fedfem

extern "C" int fedfem_fp64_fma_loop(long long iterations, int blocks, int threads, double* sink_dev, void* stream) {
    if (iterations < 1 || blocks < 1 || threads < 32 || threads > 1024 || !sink_dev) return FEDFEM_E_ARG;
    fedfem::k_fp64_fma_loop<<<blocks, threads, 0, (cudaStream_t)stream>>>(iterations, sink_dev);
    return cudaGetLastError() == cudaSuccess ? FEDFEM_OK : FEDFEM_E_CUDA;
}
