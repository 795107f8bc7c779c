// fedfem_step_static: explicit steps for callers that cannot allocate device
// memory -- for example code that runs inside another framework's memory pool,
// a real-time loop where allocation is forbidden after start-up, or a plug-in
// that must not call cudaMalloc/cudaFree.  The caller passes every input and
// output as its own device buffers; all temporary storage (the per-element
// loads, the element matrices, the lumped volumes and loads) lives in ONE
// file-scope device array of fixed size, so the call allocates nothing.
//
// Limits: at most kStaticMaxElems elements and kStaticMaxNodes nodes.  The array
// (about 18.3 MB) is held by every GPU that loads this library until the
// process exits.  All calls share it: two calls whose work overlaps on the GPU
// (different streams, or different host threads) race and corrupt each other.
//
// Every index the caller passes is checked on the device before it is used
// (k_static_check); a bad index, a node that no element uses (and that is not
// held) or an element with det J <= 0 raises the flag word, after which every
// later kernel of the call returns at once, so the caller's temperatures are
// left as they were.
#include <algorithm>
#include <climits>

#include "elem_math.cuh"
#include "fedfem_internal.h"

namespace fedfem {
namespace {

constexpr int64_t kStaticMaxElems = 131072;
constexpr int64_t kStaticMaxNodes = 160000;
// [element loads: 8 per element][M: 6 per element][V_e / nv: 1 per element]
// [V_i][Q_i][flag words]
constexpr int64_t kOffSlots = 0;
constexpr int64_t kOffM = kOffSlots + 8 * kStaticMaxElems;
constexpr int64_t kOffVshare = kOffM + 6 * kStaticMaxElems;
constexpr int64_t kOffV = kOffVshare + kStaticMaxElems;
constexpr int64_t kOffQ = kOffV + kStaticMaxNodes;
constexpr int64_t kOffFlag = kOffQ + kStaticMaxNodes;
constexpr int64_t kStaticWords = kOffFlag + 8;

static __device__ __align__(256) double g_static_scratch[kStaticWords];

struct StaticArgs {
    int nv;
    int64_t N, E;
    const double* xyz;
    const int32_t* conn;
    const int32_t* row_ptr;
    const int32_t* slot;
    const double* q_r;
    const unsigned char* held;
    double* T;
    double* s;     // the static scratch
    Law<double> k;
    Law<double> rho, c;
    double wbcb, T_a, Q_m, dt;
};

// a mesh defect found earlier in this call: leave everything untouched
__device__ __forceinline__ bool static_failed(const StaticArgs& a) { return a.s[kOffFlag] != 0.0; }

// Index checks of the caller's mesh and gather, before anything reads through
// them: every corner names a node in [0, N); row_ptr starts at 0, never
// decreases and ends at E * nv; each row lists slots in [0, E * nv) in
// increasing order whose corner is that row's node (so every (element,
// corner) appears exactly once); a node with an empty row must be held.
// Each access is bounded on its own, so a malformed array is read in range.
__global__ void k_static_check(StaticArgs a) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nslot = a.E * a.nv;
    bool bad = false;
    if (t < nslot) {
        const int32_t g = a.conn[t];
        bad = g < 0 || g >= a.N;
    }
    if (t < a.N) {
        const int64_t r0 = a.row_ptr[t], r1 = a.row_ptr[t + 1];
        if ((t == 0 && r0 != 0) || (t == a.N - 1 && r1 != nslot) || r0 < 0 || r1 < r0 || r1 > nslot) {
            bad = true;
        } else {
            if (r1 == r0 && !(a.held && a.held[t])) bad = true;   // no element: zero capacity
            int64_t prev = -1;
            for (int64_t p = r0; p < r1 && !bad; ++p) {
                const int64_t q = a.slot[p];
                if (q <= prev || q >= nslot || a.conn[q] != (int32_t)t) bad = true;
                prev = q;
            }
        }
    }
    if (bad) a.s[kOffFlag] = 1.0;
}

__global__ void k_static_geom(StaticArgs a) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.E || static_failed(a)) return;
    const int32_t* cn = a.conn + e * a.nv;
    double J[3][3];
    if (a.nv == 8) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) J[i][j] = 0.0;
        for (int n = 0; n < 8; ++n) {
            const double s0 = (n == 1 || n == 2 || n == 5 || n == 6) ? 0.125 : -0.125;
            const double s1 = (n == 2 || n == 3 || n == 6 || n == 7) ? 0.125 : -0.125;
            const double s2 = (n >= 4) ? 0.125 : -0.125;
            for (int i = 0; i < 3; ++i) {
                const double X = a.xyz[3 * (int64_t)cn[n] + i];
                J[i][0] += X * s0;
                J[i][1] += X * s1;
                J[i][2] += X * s2;
            }
        }
    } else {
        for (int j = 0; j < 3; ++j)
            for (int i = 0; i < 3; ++i) J[i][j] = a.xyz[3 * (int64_t)cn[j + 1] + i] - a.xyz[3 * (int64_t)cn[0] + i];
    }
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (!(det > 0.0)) {
        a.s[kOffFlag] = 1.0;   // inverted or degenerate element
        return;
    }
    double inv[3][3];
    inv[0][0] = c00 / det; inv[1][0] = c01 / det; inv[2][0] = c02 / det;
    inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    double P[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            P[i][j] = inv[i][0] * inv[j][0] + inv[i][1] * inv[j][1] + inv[i][2] * inv[j][2];
    const double w = (a.nv == 8) ? det * 0.125 : det / 6.0;
    const double Ve = (a.nv == 8) ? 8.0 * det : det / 6.0;
    double* M = a.s + kOffM;
    M[0 * kStaticMaxElems + e] = w * P[0][0];
    M[1 * kStaticMaxElems + e] = w * P[1][1];
    M[2 * kStaticMaxElems + e] = w * P[2][2];
    M[3 * kStaticMaxElems + e] = w * P[0][1];
    M[4 * kStaticMaxElems + e] = w * P[0][2];
    M[5 * kStaticMaxElems + e] = w * P[1][2];
    a.s[kOffVshare + e] = Ve / a.nv;
}

__global__ void k_static_nodal(StaticArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N || static_failed(a)) return;
    double V = 0.0;
    for (int32_t p = a.row_ptr[i]; p < a.row_ptr[i + 1]; ++p) V += a.s[kOffVshare + a.slot[p] / a.nv];
    a.s[kOffV + i] = V;
    a.s[kOffQ + i] = V * (a.Q_m + (a.q_r ? a.q_r[i] : 0.0));
}

__global__ void k_static_elem(StaticArgs a) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.E || static_failed(a)) return;
    const int32_t* cn = a.conn + e * a.nv;
    double m[6];
    for (int j = 0; j < 6; ++j) m[j] = a.s[kOffM + j * kStaticMaxElems + e];
    double* out = a.s + kOffSlots + e * a.nv;
    if (a.nv == 8) {
        double t[8], F[8];
        for (int n = 0; n < 8; ++n) t[n] = a.T[cn[n]];
        hex8_loads<double>(t, m, element_k<double, 8>(t, a.k), F);
        for (int n = 0; n < 8; ++n) out[n] = F[n];
    } else {
        double t[4], F[4];
        for (int n = 0; n < 4; ++n) t[n] = a.T[cn[n]];
        tet4_loads<double>(t, m, element_k<double, 4>(t, a.k), F);
        for (int n = 0; n < 4; ++n) out[n] = F[n];
    }
}

__global__ void k_static_node(StaticArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N || (a.held && a.held[i]) || static_failed(a)) return;
    double F = 0.0;
    for (int32_t p = a.row_ptr[i]; p < a.row_ptr[i + 1]; ++p) F = F + a.s[kOffSlots + a.slot[p]];
    const double T = a.T[i];
    const double V = a.s[kOffV + i];
    const double C = (V * a.rho(T)) * a.c(T);
    const double r = fmadd(a.wbcb * V, a.T_a - T, a.s[kOffQ + i]) - F;
    a.T[i] = T + (a.dt * r) / C;
}

// Device address of the scratch array on the current device.  Looked up on
// every call: the lookup is cheap next to the launches, and an address kept
// from an earlier call would be stale once the device's context is recreated
// (after cudaDeviceReset, the module is loaded again elsewhere).
cudaError_t static_scratch(double** out) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

inline int grid_for(int64_t n) { return (int)((n + 255) / 256); }

}  // namespace
}  // namespace fedfem

using namespace fedfem;

extern "C" int fedfem_step_static(int elem_type, int64_t n_nodes, int64_t n_elems, const double* xyz_dev,
                                  const int32_t* conn_dev, const int32_t* row_ptr_dev, const int32_t* slot_dev,
                                  const fedfem_material* mat, const fedfem_perfusion* perf, const double* q_r_dev,
                                  const unsigned char* held_dev, double dt, int64_t n_steps, double* T_dev,
                                  void* cuda_stream) {
    if (elem_type != FEDFEM_HEX8 && elem_type != FEDFEM_TET4) return FEDFEM_E_ARG;
    if (n_nodes <= 0 || n_elems <= 0 || n_steps < 0 || !(dt > 0)) return FEDFEM_E_ARG;
    if (n_nodes > kStaticMaxNodes || n_elems > kStaticMaxElems) return FEDFEM_E_ARG;   // beyond the fixed scratch
    if (!xyz_dev || !conn_dev || !row_ptr_dev || !slot_dev || !mat || !perf || !T_dev) return FEDFEM_E_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double* s = nullptr;
    if (static_scratch(&s) != cudaSuccess) return FEDFEM_E_CUDA;
    StaticArgs a{};
    a.nv = elem_type; a.N = n_nodes; a.E = n_elems;
    a.xyz = xyz_dev; a.conn = conn_dev; a.row_ptr = row_ptr_dev; a.slot = slot_dev;
    a.q_r = q_r_dev; a.held = held_dev; a.T = T_dev; a.s = s;
    a.k = Law<double>{mat->T_ref, mat->k0, mat->dk};
    a.rho = Law<double>{mat->T_ref, mat->rho0, mat->drho};
    a.c = Law<double>{mat->T_ref, mat->c0, mat->dc};
    a.wbcb = perf->w_b * perf->c_b; a.T_a = perf->T_a; a.Q_m = perf->Q_m; a.dt = dt;
    // the flag word keeps the previous call's value: clear it first
    if (cudaMemsetAsync(s + kOffFlag, 0, sizeof(double), st) != cudaSuccess) return FEDFEM_E_CUDA;
    k_static_check<<<grid_for(std::max(n_nodes, n_elems * elem_type)), 256, 0, st>>>(a);
    k_static_geom<<<grid_for(n_elems), 256, 0, st>>>(a);
    k_static_nodal<<<grid_for(n_nodes), 256, 0, st>>>(a);
    for (int64_t k = 0; k < n_steps; ++k) {
        k_static_elem<<<grid_for(n_elems), 256, 0, st>>>(a);
        k_static_node<<<grid_for(n_nodes), 256, 0, st>>>(a);
    }
    if (cudaGetLastError() != cudaSuccess) return FEDFEM_E_CUDA;
    double flag = 0.0;
    if (cudaMemcpyAsync(&flag, s + kOffFlag, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return FEDFEM_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FEDFEM_E_CUDA;
    return flag != 0.0 ? FEDFEM_E_MESH : FEDFEM_OK;
}
