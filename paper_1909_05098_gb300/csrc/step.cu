// The time loop of Algorithm 1: an element phase (Eq. 17 with
// k_e of Eq. 13) writing each element's nodal loads into its own slots, then
// a node phase that gathers every free node's slots in a fixed order (the sum
// of Eq. 11, no atomics), forms the lumped capacitance C_i(T) and applies the
// explicit update of Eq. 19 with the conduction load entering as -F (physical
// diffusion), the perfusion as beta_i (T_a - T_i) and the film condition as
// hA_i (T_inf - T_i).  Dirichlet nodes (Eq. 3) are never written.
//
// FP32 state is an unevaluated pair (hi, lo): the increment is added by
// compensated summation (Fast2Sum on |hi| >= |increment + lo|), element
// gradients and properties use hi.  Kernel families:
//   * two-phase: one element launch and one node launch per step;
//   * persistent: one cooperative launch runs n steps; the two phases are
//     separated by a grid barrier whose spin is bounded (clock64 limit), after
//     which the kernel records a timeout and returns.
#include <algorithm>
#include <climits>

#include <cooperative_groups.h>

#include "elem_math.cuh"
#include "fedfem_internal.h"

namespace fedfem {
namespace {

template <typename R>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

template <typename R>
struct Vec;
template <>
struct Vec<float> {
    static __device__ __forceinline__ void store4(float* p, const float* v) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct Vec<double> {
    static __device__ __forceinline__ void store4(double* p, const double* v) {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
};

// Property P (0 rho, 1 c, 2 k) of a piecewise-linear table at T, from its
// first interval and the slope change at each interior point (the same
// function as the value and slope of the interval that holds T; the end
// intervals extend beyond the table).  Every term reads launch arguments;
// the point count is the same for every thread, so its test is uniform.
template <int P, typename R, typename L, typename X>
__device__ __forceinline__ X tab_law(const StepArgs<R, L>& a, X T) {
    X v = fmadd(a.tab_s0[P], T - a.tab_T[0], a.tab_p0[P]);
#pragma unroll
    for (int q = 1; q < kMaxTable - 1; ++q)
        if (q < a.n_tab - 1) v = fmadd(a.tab_d[P][q], ramp(T - a.tab_T[q]), v);
    return v;
}

// k(T) from the property table
template <typename R, typename L>
struct TabKLaw {
    const StepArgs<R, L>& a;
    template <typename X>
    __device__ __forceinline__ X at(X T) const { return tab_law<2>(a, T); }
};

// Eq. 13's k_e under a table law: k at every corner as tab_law<2> computes
// it (the same operations in the same order, so the same bits), with one
// uniform test per interior point for the whole element; FP32 corners go in
// pairs through the packed instructions, paired as in sum_nodal.
template <typename R, int NV, typename L, typename R2, typename L2>
__device__ __forceinline__ L element_k(const L t[NV], const TabKLaw<R2, L2>& kl) {
    const StepArgs<R2, L2>& a = kl.a;
    if constexpr (std::is_same<L, float>::value) {
        constexpr int NP = NV / 2;
        float2 tp[NP];
        if constexpr (NV == 8) {
            tp[0] = make_float2(t[0], t[1]); tp[1] = make_float2(t[3], t[2]);
            tp[2] = make_float2(t[4], t[5]); tp[3] = make_float2(t[7], t[6]);
        } else {
            tp[0] = make_float2(t[0], t[1]); tp[1] = make_float2(t[2], t[3]);
        }
        const float2 T0 = make_float2(a.tab_T[0], a.tab_T[0]);
        const float2 s0 = make_float2(a.tab_s0[2], a.tab_s0[2]), p0 = make_float2(a.tab_p0[2], a.tab_p0[2]);
        float2 kp[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) kp[i] = fma2(s0, sub2(tp[i], T0), p0);
#pragma unroll
        for (int q = 1; q < kMaxTable - 1; ++q)
            if (q < a.n_tab - 1) {
                const float2 Tq = make_float2(a.tab_T[q], a.tab_T[q]), dq = make_float2(a.tab_d[2][q], a.tab_d[2][q]);
#pragma unroll
                for (int i = 0; i < NP; ++i) kp[i] = fma2(dq, ramp(sub2(tp[i], Tq)), kp[i]);
            }
        if constexpr (NV == 8) {
            const float2 s = add2(add2(kp[0], kp[1]), add2(kp[2], kp[3]));
            return 0.125f * (s.x + s.y);
        } else {
            const float2 s = add2(kp[0], kp[1]);
            return 0.25f * (s.x + s.y);
        }
    } else {
        L kn[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) kn[n] = fmadd(a.tab_s0[2], t[n] - a.tab_T[0], a.tab_p0[2]);
#pragma unroll
        for (int q = 1; q < kMaxTable - 1; ++q)
            if (q < a.n_tab - 1) {
#pragma unroll
                for (int n = 0; n < NV; ++n) kn[n] = fmadd(a.tab_d[2][q], ramp(t[n] - a.tab_T[q]), kn[n]);
            }
        return R(1) / R(NV) * sum_nodal<NV, L>(kn);
    }
}

// The element k laws of a context, as functions of the element index j: the
// material's law (Plain), each element's region law (Region), or the table
// (Table).  Kernels built with the extensions pick one per launch or tile
// (uniform), so no element pays a branch between them.
template <typename R, typename L>
struct PlainK {
    const StepArgs<R, L>& a;
    __device__ __forceinline__ Law<R> operator()(int64_t) const { return Law<R>{a.T_ref, a.k0, a.dk}; }
};
template <typename R, typename L>
struct RegionK {
    const StepArgs<R, L>& a;
    const unsigned char* em;
    __device__ __forceinline__ Law<R> operator()(int64_t j) const {
        const R* q = a.mat_k + 3 * (int)em[j];
        return Law<R>{__ldg(q), __ldg(q + 1), __ldg(q + 2)};
    }
};
template <typename R, typename L>
struct TableK {
    const StepArgs<R, L>& a;
    __device__ __forceinline__ TabKLaw<R, L> operator()(int64_t) const { return TabKLaw<R, L>{a}; }
};

// f(k) with the context's element k laws (em: region ids of the elements, or null)
template <int MODE, typename R, typename L, typename Fn>
__device__ __forceinline__ void with_k_laws(const StepArgs<R, L>& a, const unsigned char* em, Fn&& f) {
    if constexpr ((MODE & 2) != 0) {
        if (a.n_tab > 0) f(TableK<R, L>{a});
        else if (em) f(RegionK<R, L>{a, em});
        else f(PlainK<R, L>{a});
    } else {
        f(PlainK<R, L>{a});
    }
}

// Fully integrated hex8: F_m = k_e sum_n A_mn (T_n - T_m) over the 28 pairs
// (the zero row sums give the diagonal; a uniform field gives exactly 0)
template <typename R>
__device__ __forceinline__ void hex8_full_loads(const StepArgs<R>& a, int64_t e, const R t[8], R ke, R F[8]) {
    const int64_t E = a.E;
#pragma unroll
    for (int n = 0; n < 8; ++n) F[n] = R(0);
    int q = 0;
#pragma unroll
    for (int m = 0; m < 8; ++m)
#pragma unroll
        for (int n = m + 1; n < 8; ++n, ++q) {
            const R w = a.A28[q * E + e] * (t[n] - t[m]);
            F[m] = F[m] + w;
            F[n] = F[n] - w;
        }
#pragma unroll
    for (int n = 0; n < 8; ++n) F[n] = ke * F[n];
}

template <typename R, int NV, int MODE>
__device__ __forceinline__ void element_phase(const StepArgs<R>& a, int64_t e) {
    const int64_t E = a.E;
    int c[8];
    const int4 c0 = a.conn4[e];
    c[0] = c0.x; c[1] = c0.y; c[2] = c0.z; c[3] = c0.w;
    if (NV == 8) {
        const int4 c1 = a.conn4[E + e];
        c[4] = c1.x; c[5] = c1.y; c[6] = c1.z; c[7] = c1.w;
    }
    R m[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) m[j] = a.M[j * E + e];
    R t[NV];
#pragma unroll
    for (int n = 0; n < NV; ++n) t[n] = a.T[c[n]];
    R ke;
    with_k_laws<MODE>(a, a.emat, [&](const auto& kl) { ke = element_k<R, NV>(t, kl(e)); });
    R F[NV];
    bool full = false, hg = false;
    if constexpr ((MODE & 2) != 0 && NV == 8) {
        full = a.A28 != nullptr;
        hg = a.W12 != nullptr;
    }
    if constexpr (NV == 8) {
        if (full) {
            hex8_full_loads<R>(a, e, t, ke, F);
        } else if (hg) {
            R w[12];
#pragma unroll
            for (int q = 0; q < 12; ++q) w[q] = a.W12[q * E + e];
            hex8_hourglass_loads<R>(t, m, w, a.hg_eps4, ke, F);
        } else {
            hex8_loads<R>(t, m, ke, F);
        }
    } else {
        tet4_loads<R>(t, m, ke, F);
    }
    R* out = a.slots + e * NV;
    Vec<R>::store4(out, F);
    if (NV == 8) Vec<R>::store4(out + 4, F + 4);
}

__device__ __forceinline__ void flag_range(DevStatus* st, int64_t i, long long step) {
    atomicOr(&st->flags, STATUS_RANGE);
    atomicMin(&st->fail_step, step);
    atomicMin(&st->fail_node, (long long)i);
}

// Eq. 19 for free node i: T is its current (hi) value, F the summed element
// loads; writes the new value to Tout[i] (and the compensation in place).
// The node's constant data (and its compensation) as loaded values.
template <typename R, typename L>
struct NodeVals {
    R V, hA;
    L Q, lo;
};

template <typename L>
__device__ __forceinline__ L lzero() { return L{}; }

template <typename R, typename L, int MODE>
__device__ __forceinline__ NodeVals<R, L> node_load(const StepArgs<R, L>& a, int64_t i) {
    NodeVals<R, L> v;
    v.V = a.V[i];
    v.Q = a.Q[i];
    v.hA = i >= a.N_plain ? a.hA[i - a.N_plain] : R(0);
    v.lo = (MODE & 1) ? a.Tlo[i] : lzero<L>();
    return v;
}

// f(t) of the source schedule for the step with index `step`
template <typename R, typename L>
__device__ __forceinline__ R schedule_factor(const StepArgs<R, L>& a, long long step) {
    const double t = a.t0 + (double)(step - a.step0) * a.dtd;
    int k = 0;
    while (k + 1 < a.n_seg && t >= a.seg_end[k]) ++k;
    return a.seg_f[k];
}

// Dose rate at the step's start temperature T: CEM43 (model 0), R^(43 - T)
// with R = 1/2 at or above 43 degC and 1/4 below, in equivalent minutes per
// minute; or the Arrhenius damage rate (model 1), A exp(-Ea / (R_gas T_K)) =
// exp(lnA - EaR / (T + 273.15)), per second.  The power is taken in the
// state's precision (FP32 state: exp2f, whose relative error is far below
// that of the FP32 temperature it is taken of).
__device__ __forceinline__ double dose_rate(int model, double lnA, double EaR, double T) {
    if (model == 1) return exp(lnA - EaR / (T + 273.15));
    return exp2(T >= 43.0 ? T - 43.0 : 2.0 * (T - 43.0));
}
// FP32 state, both models as one power of 2 without a branch:
// 2^(c43 s (T - 43) + a2 - g2 / T_K), s = 1 at or above 43 degC and 2 below;
// CEM43: c43 = 1, a2 = g2 = 0 (exactly the CEM43 exponent); Arrhenius:
// c43 = 0, a2 = log2 A, g2 = (Ea / R) / ln 2
__device__ __forceinline__ float dose_rate(float c43, float a2, float g2, float T) {
    const float e = c43 * (T >= 43.0f ? T - 43.0f : 2.0f * (T - 43.0f));
    return exp2f((e + a2) - g2 * __frcp_rn(T + 273.15f));
}
// The FP32 dose (hi, lo) plus an increment: y = inc + lo, then hi + y as an
// exact sum of two FP32 values (Knuth's TwoSum, valid whatever their sizes:
// the increment of a heating node can exceed the dose so far), so the pair
// carries the running dose to about 2^-48 relative with FP32 instructions only.
__device__ __forceinline__ float2 dose_sum(float2 d, float inc) {
    const float y = inc + d.y;
    const float s = d.x + y;
    const float yy = s - d.x;
    return make_float2(s, (d.x - (s - yy)) + (y - yy));
}
template <typename L>
__device__ __forceinline__ void dose_add(const StepArgs<double, L>& a, int64_t i, double T) {
    a.dose[i] += a.dose_dt * dose_rate(a.dose_model, a.dose_lnA, a.dose_EaR, T);
}
template <typename L>
__device__ __forceinline__ void dose_add(const StepArgs<float, L>& a, int64_t i, float T) {
    float2* d = reinterpret_cast<float2*>(a.dose) + i;
    *d = dose_sum(*d, a.dose_dt32 * dose_rate(a.dose_c43, a.dose_a2, a.dose_g2, T));
}
// four scenario lanes: the node's four (hi, lo) pairs are contiguous, each
// lane summed exactly as one lane alone
template <typename L>
__device__ __forceinline__ void dose_add(const StepArgs<float, L>& a, int64_t i, F4 T) {
    float4* d = reinterpret_cast<float4*>(a.dose) + 2 * i;
    const float4 p = d[0], q = d[1];
    const float2 d0 = dose_sum(make_float2(p.x, p.y), a.dose_dt32 * dose_rate(a.dose_c43, a.dose_a2, a.dose_g2, T.x));
    const float2 d1 = dose_sum(make_float2(p.z, p.w), a.dose_dt32 * dose_rate(a.dose_c43, a.dose_a2, a.dose_g2, T.y));
    const float2 d2 = dose_sum(make_float2(q.x, q.y), a.dose_dt32 * dose_rate(a.dose_c43, a.dose_a2, a.dose_g2, T.z));
    const float2 d3 = dose_sum(make_float2(q.z, q.w), a.dose_dt32 * dose_rate(a.dose_c43, a.dose_a2, a.dose_g2, T.w));
    d[0] = make_float4(d0.x, d0.y, d1.x, d1.y);
    d[1] = make_float4(d2.x, d2.y, d3.x, d3.y);
}

template <typename R, typename L, int MODE>
__device__ __forceinline__ void node_update_v(const StepArgs<R, L>& a, int64_t i, L T, L F,
                                              const NodeVals<R, L>& v, L* Tout, long long step) {
    const L u = T - a.T_ref;
    L rho = fmadd(a.drho, u, a.rho0);
    L c = fmadd(a.dc, u, a.c0);
    L C = (v.V * rho) * c;
    R beta = a.wbcb * v.V;
    L q = v.Q;
    if constexpr ((MODE & 2) != 0) {   // kernels built with the extensions
        if (a.n_tab > 0) {
            rho = tab_law<0>(a, T);
            c = tab_law<1>(a, T);
            C = (v.V * rho) * c;
        } else if (a.Cq) {             // regions: C and beta summed from the element shares
            const int64_t nf = a.N_free;
            C = fmadd(fmadd(a.Cq[2 * nf + i], u, a.Cq[nf + i]), u, a.Cq[i]);
            beta = a.Cq[3 * nf + i];
        }
        if (a.Qs) q = fmadd(schedule_factor(a, step), a.Qs[i], q);
        if (a.dose) dose_add(a, i, T);   // at the step's start temperature
    }
    L r = fmadd(beta, a.T_a - T, q) - F;
    if (i >= a.N_plain) r = fmadd(v.hA, a.T_inf - T, r);
    const L dT = increment_div(a.dt * r, C);
    L Tn;
    if (MODE & 1) {
        const L y = dT + v.lo;
        Tn = T + y;
        a.Tlo[i] = y - (Tn - T);
    } else {
        Tn = T + dT;
    }
    Tout[i] = Tn;
    if (!all_in(Tn, a.T_lo, a.T_hi)) flag_range(a.status, i, step);
}

template <typename R, typename L, int MODE>
__device__ __forceinline__ void node_update(const StepArgs<R, L>& a, int64_t i, L T, L F, L* Tout, long long step) {
    node_update_v<R, L, MODE>(a, i, T, F, node_load<R, L, MODE>(a, i), Tout, step);
}

// gather of node i's element loads from the global slots, in its fixed order
template <typename R, int MODE>
__device__ __forceinline__ void node_phase(const StepArgs<R>& a, int64_t i, long long step) {
    const int64_t s = i >> 5;
    const int lane = (int)(i & 31);
    const int32_t off = a.sell_off[s];
    const int w = (a.sell_off[s + 1] - off) >> 5;
    R F = R(0);
    for (int k = 0; k < w; ++k) F = F + a.slots[a.sell_ids[off + 32 * k + lane]];
    node_update<R, R, MODE>(a, i, a.T[i], F, a.T, step);
}

template <typename R, int NV, int MODE>
__global__ void __launch_bounds__(256) k_elem(StepArgs<R> a) {
    if (*(volatile int*)&a.status->flags) return;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < a.E) element_phase<R, NV, MODE>(a, e);
}

template <typename R, int MODE>
__global__ void __launch_bounds__(256) k_node(StepArgs<R> a, long long step) {
    if (*(volatile int*)&a.status->flags) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.N_free) node_phase<R, MODE>(a, i, step);
}

// ---- bounded grid barrier --------------------------------------------------

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// All blocks arrive once per call; target grows by gridDim.x per call.  A
// block waits at most spin_limit clock64 ticks, then records a timeout.
// Returns false when the loop must stop (timeout, or a flag raised before the
// barrier, which every block then sees alike).
__device__ __forceinline__ bool grid_barrier(DevStatus* st, unsigned long long& target, long long spin_limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        int ok = 1;
        if ((int)blockIdx.x != st->skip_barrier_block) red_release_add(&st->barrier, 1ULL);
        const long long t0 = clock64();
        while (ld_acquire(&st->barrier) < target) {
            if (ld_relaxed(&st->flags) & STATUS_TIMEOUT) { ok = 0; break; }
            if (clock64() - t0 > spin_limit) { atomicOr(&st->flags, STATUS_TIMEOUT); ok = 0; break; }
        }
        if (ok && ld_relaxed(&st->flags)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename R, int NV, int MODE>
__device__ __forceinline__ void persistent_steps(const StepArgs<R>& a, long long n_steps, long long spin_limit) {
    unsigned long long target = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    long long done = 0;
    if (!grid_barrier(a.status, target, spin_limit)) return;   // flags from an earlier call stop here
    for (long long s = 0; s < n_steps; ++s) {
        for (int64_t e = tid; e < a.E; e += stride) element_phase<R, NV, MODE>(a, e);
        if (!grid_barrier(a.status, target, spin_limit)) break;
        for (int64_t i = tid; i < a.N_free; i += stride) node_phase<R, MODE>(a, i, a.step0 + s);
        const bool ok = grid_barrier(a.status, target, spin_limit);
        done = s + 1;
        if (!ok) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.status->steps_done = a.step0 + done;
}
template <typename R, int NV, int MODE>
__global__ void __launch_bounds__(256) k_persistent(StepArgs<R> a, long long n_steps, long long spin_limit) {
    persistent_steps<R, NV, MODE>(a, n_steps, spin_limit);
}
// The extension build asks for at least 4 (FP32) or 3 (FP64) blocks per SM:
// without the bound the compiler keeps its per-element plane offsets live
// across the whole step loop (172 registers, one block per SM).
template <typename R, int NV, int MODE>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 3)
    k_persistent_ext(StepArgs<R> a, long long n_steps, long long spin_limit) {
    persistent_steps<R, NV, MODE>(a, n_steps, spin_limit);
}

// ---- tiled persistent kernels ------------------------------------------------
// Tile t owns free nodes [t*B, t*B + own).  Its constant data (element
// matrices, 16-bit local connectivity with each owned corner's rank in its
// node's sum, halo ids) is one packed block.  Per tile: the owned and halo
// temperatures sit in shared memory; every element touching an owned node
// computes its loads (Eq. 17) and writes each owned corner's load into row
// `rank` of that node's column of a load table; each owned node then sums its
// column in rank order (= input element order, the order of every other
// kernel), zeroing it for the next tile, and applies Eq. 19.  T is double-
// buffered (tiles read their neighbours' nodes as halo), so one grid barrier
// per step.
//
// Staged variant: a bulk (TMA) copy brings each block into one of two shared-
// memory stages, two tiles ahead; the next tile's temperatures are fetched
// with asynchronous copies while the current tile's node phase runs.

constexpr int kTiledThreads = 512;        // default block of the staged kernel (256 and 1024 also built)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// L2 policy for data read once per step and streamed: evicted before the
// node arrays, which every step reads again
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for a stage: false after spin_limit clock64 ticks
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long spin_limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > spin_limit) return false;
    return true;
}

// asynchronous global -> shared copy of one temperature (4, 8 or 16 bytes)
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
    if (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// the parts of a packed tile block
template <typename R>
struct TileView {
    int ne, ne_pad, nh, deg;
    // (every pointer is derived from the block, never null, so that shared-memory
    // blocks keep shared-space loads; hg and mf say which parts exist)
    bool hg, mf;
    const R* M;                 // ne_pad x 6: an element's six values together (absent in matrix-free blocks)
    const R* W;                 // hg blocks: ne_pad x 12 hourglass weights
    const float4* X;            // mf blocks: local node coordinates by local id
    const uint16_t* lc;         // nv entries per element
    const int32_t* halo;        // nh global node ids
};
// hg: blocks carry hourglass weights; mf_B > 0: matrix-free blocks of tiles of
// mf_B owned nodes (coordinates instead of element matrices)
template <typename R, int NV>
__device__ __forceinline__ TileView<R> tile_view(const unsigned char* blk, int hg = 0, int mf_B = 0) {
    const int4 hdr = *reinterpret_cast<const int4*>(blk);
    TileView<R> v;
    v.ne = hdr.x; v.ne_pad = hdr.y; v.nh = hdr.z; v.deg = hdr.w;
    v.hg = hg != 0 && mf_B == 0;
    v.mf = mf_B > 0;
    v.M = reinterpret_cast<const R*>(blk + 16);
    v.W = v.M + 6 * (size_t)v.ne_pad;
    v.X = reinterpret_cast<const float4*>(blk + 16);
    const size_t geo = v.mf ? 16 * (size_t)(mf_B + v.nh) : (v.hg ? 18 : 6) * (size_t)v.ne_pad * sizeof(R);
    v.lc = reinterpret_cast<const uint16_t*>(blk + 16 + geo);
    v.halo = reinterpret_cast<const int32_t*>(v.lc + NV * v.ne_pad);
    return v;
}

// the block variants a kernel build can meet: only the builds with the
// extensions (MODE bit 1) read hourglass weights or coordinates, so the plain
// builds see constants and keep their code
template <int MODE, typename R>
__device__ __forceinline__ int view_hg(const TileArgs<R>& ta) { return (MODE & 2) != 0 ? ta.hourglass : 0; }
template <int MODE, typename R>
__device__ __forceinline__ int view_mf(const TileArgs<R>& ta) { return (MODE & 2) != 0 && ta.mf ? ta.B : 0; }

// element loads inside a tile: the plain factored rule, or (kernels built with
// the extensions, blocks carrying weights) the hourglass-stabilised one
template <bool EXT, typename R, typename L, int NV>
__device__ __forceinline__ void tile_loads(const TileView<R>& v, int j, const L tt[NV], const R m[6], L ke, R eps4,
                                           L F[NV]) {
    if constexpr (NV == 8) {
        if constexpr (EXT) {
            if (v.hg) {
                R w[12];
#pragma unroll
                for (int q = 0; q < 12; q += 2) {
                    const typename Vec2<R>::type p = reinterpret_cast<const typename Vec2<R>::type*>(v.W + 12 * j)[q / 2];
                    w[q] = p.x;
                    w[q + 1] = p.y;
                }
                hex8_hourglass_loads<R, L>(tt, m, w, eps4, ke, F);
                return;
            }
        }
        hex8_loads<R, L>(tt, m, ke, F);
    } else {
        tet4_loads<R, L>(tt, m, ke, F);
    }
}

template <int NV>
struct LConn;
// (reload: a fresh load, so the entries need not stay in registers across the
// element math; the block may sit in shared or global memory)
template <>
struct LConn<8> {
    static __device__ __forceinline__ void split(uint4 v, int c[8]) {
        c[0] = v.x & 0xffff; c[1] = v.x >> 16; c[2] = v.y & 0xffff; c[3] = v.y >> 16;
        c[4] = v.z & 0xffff; c[5] = v.z >> 16; c[6] = v.w & 0xffff; c[7] = v.w >> 16;
    }
    static __device__ __forceinline__ void load(const uint16_t* p, int j, int c[8]) {
        split(reinterpret_cast<const uint4*>(p)[j], c);
    }
    template <bool SHARED>
    static __device__ __forceinline__ void reload(const uint16_t* p, int j, int c[8]) {
        uint4 v;
        if (SHARED)
            asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                         : "r"(smem_u32(reinterpret_cast<const uint4*>(p) + j)));
        else
            asm volatile("ld.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                         : "l"(reinterpret_cast<const uint4*>(p) + j));
        split(v, c);
    }
};
template <>
struct LConn<4> {
    static __device__ __forceinline__ void split(uint2 v, int c[4]) {
        c[0] = v.x & 0xffff; c[1] = v.x >> 16; c[2] = v.y & 0xffff; c[3] = v.y >> 16;
    }
    static __device__ __forceinline__ void load(const uint16_t* p, int j, int c[4]) {
        split(reinterpret_cast<const uint2*>(p)[j], c);
    }
    template <bool SHARED>
    static __device__ __forceinline__ void reload(const uint16_t* p, int j, int c[4]) {
        uint2 v;
        if (SHARED)
            asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];"
                         : "=r"(v.x), "=r"(v.y)
                         : "r"(smem_u32(reinterpret_cast<const uint2*>(p) + j)));
        else
            asm volatile("ld.global.v2.u32 {%0, %1}, [%2];"
                         : "=r"(v.x), "=r"(v.y)
                         : "l"(reinterpret_cast<const uint2*>(p) + j));
        split(v, c);
    }
};

// owned and halo temperatures of a tile into Ts (asynchronous copies when ASYNC;
// the caller commits, waits and synchronises)
template <typename L, bool ASYNC>
__device__ __forceinline__ void tile_fetch(const int32_t* halo, int nh, int64_t base, int own, const L* Tin, L* Ts) {
    for (int l = threadIdx.x; l < own; l += blockDim.x) {
        if (ASYNC) cp_async<sizeof(L)>(Ts + l, Tin + base + l);
        else Ts[l] = Tin[base + l];
    }
    for (int h = threadIdx.x; h < nh; h += blockDim.x) {
        if (ASYNC) cp_async<sizeof(L)>(Ts + own + h, Tin + halo[h]);
        else Ts[own + h] = Tin[halo[h]];
    }
}

// region ids of tile t's elements (null without regions)
template <int MODE, typename R, typename L>
__device__ __forceinline__ const unsigned char* tile_regions(const StepArgs<R, L>& a, int64_t t) {
    if constexpr ((MODE & 2) != 0) return a.emat_tile ? a.emat_tile + a.emat_off[t] : nullptr;
    else return nullptr;
}

// element phase of one tile: loads of every tile element; each owned corner's
// load goes to Fn[rank * B + local id], B the load table's row stride (the
// tile size plus one: odd, so that the rank rows of one node fall in
// different shared-memory banks)
template <typename R, typename L, int NV, bool SHARED, bool EXT, typename KL>
__device__ __forceinline__ void tile_elements_k(const KL& kl, const TileView<R>& v, int own, int B, int rank_shift,
                                                const L* Ts, L* Fn, R eps4) {
    const int id_mask = (1 << rank_shift) - 1;
    for (int j = threadIdx.x; j < v.ne; j += blockDim.x) {
        int c[NV];
        LConn<NV>::load(v.lc, j, c);
        L tt[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) tt[n] = Ts[c[n] & id_mask];
        R m[6];
        bool mf = false;
        if constexpr (EXT && NV == 4 && sizeof(R) == sizeof(float)) {   // matrix-free: M from the corners
            if (v.mf) {
                float4 xs[4];
#pragma unroll
                for (int n = 0; n < 4; ++n) xs[n] = v.X[c[n] & id_mask];
                tet4_matrix(xs, reinterpret_cast<float*>(m));
                mf = true;
            }
        }
        if (!mf) {
#pragma unroll
            for (int q = 0; q < 6; q += 2) {   // three 2-wide loads (8- or 16-byte aligned)
                const typename Vec2<R>::type p = reinterpret_cast<const typename Vec2<R>::type*>(v.M + 6 * j)[q / 2];
                m[q] = p.x;
                m[q + 1] = p.y;
            }
        }
        const L ke = element_k<R, NV, L>(tt, kl(j));
        L F[NV];
        tile_loads<EXT, R, L, NV>(v, j, tt, m, ke, eps4, F);
        LConn<NV>::template reload<SHARED>(v.lc, j, c);
#pragma unroll
        for (int n = 0; n < NV; ++n) {
            const int id = c[n] & id_mask;
            if (id < own) Fn[(c[n] >> rank_shift) * B + id] = F[n];
        }
    }
}

template <typename R, typename L, int NV, int MODE, bool SHARED>
__device__ __forceinline__ void tile_elements(const StepArgs<R, L>& a, const unsigned char* em, const TileView<R>& v,
                                              int own, int B, int rank_shift, const L* Ts, L* Fn) {
    with_k_laws<MODE>(a, em, [&](const auto& kl) {
        tile_elements_k<R, L, NV, SHARED, (MODE & 2) != 0>(kl, v, own, B, rank_shift, Ts, Fn, a.hg_eps4);
    });
}

// node phase: sum each owned node's column (rank order), clear it, Eq. 19.
// The first owned node of each thread (l0 = threadIdx.x) comes with its
// temperature T0 and constant data v0 already loaded; further nodes (tiles
// larger than the block) read theirs from Tin.
template <typename R, typename L, int MODE>
__device__ __forceinline__ void tile_nodes(const StepArgs<R, L>& a, int64_t base, int own, int deg, int B, L* Fn,
                                           L T0, const NodeVals<R, L>& v0, const L* Tin, L* Tout, long long step) {
    for (int l = threadIdx.x; l < own; l += blockDim.x) {
        L F = lzero<L>();
        L* col = Fn + l;
        int r = 0;
        for (; r + 8 <= deg; r += 8) {   // hex interiors: one unrolled pass of 8 rows
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                F = F + col[u * B];
                col[u * B] = lzero<L>();
            }
            col += 8 * B;
        }
        for (; r < deg; ++r, col += B) {
            F = F + *col;
            *col = lzero<L>();
        }
        if (l == (int)threadIdx.x) node_update_v<R, L, MODE>(a, base + l, T0, F, v0, Tout, step);
        else node_update<R, L, MODE>(a, base + l, Tin[base + l], F, Tout, step);
    }
}

template <typename R, typename L, int MODE>
__device__ __forceinline__ void first_node(const StepArgs<R, L>& a, int64_t base, int own, const L* Ts, L& T0,
                                           NodeVals<R, L>& v0) {
    if ((int)threadIdx.x < own) {
        v0 = node_load<R, L, MODE>(a, base + threadIdx.x);
        T0 = Ts[threadIdx.x];
    }
}

template <typename L>
__device__ __forceinline__ void zero_table(L* Fn, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) Fn[i] = lzero<L>();
}

// Direct variant: the same per-tile blocks read straight from global memory
// (coalesced within a tile), shared memory only for T and the load table, so
// more blocks fit on an SM.
// resident blocks per SM the direct tiled kernel is compiled for: one FP32
// lane fits 5 blocks of 256 threads without spills, FP64 or four-lane state
// needs about twice the registers
template <typename L>
struct DirectOccupancy {
    static constexpr int min_blocks = sizeof(L) >= 8 ? 3 : 5;
};

template <typename R, typename L, int NV, int MODE>
__global__ void __launch_bounds__(256, DirectOccupancy<L>::min_blocks) k_tiled_direct(StepArgs<R, L> a, TileArgs<R> ta, long long n_steps,
                                                      long long spin_limit) {
    extern __shared__ __align__(128) unsigned char smem[];
    L* Ts = reinterpret_cast<L*>(smem);
    L* Fn = reinterpret_cast<L*>(smem + ((size_t)ta.max_local * sizeof(L) + 15) / 16 * 16);
    zero_table(Fn, ta.max_deg * (ta.B + 1));
    unsigned long long target = 0;
    long long done = 0;
    if (!grid_barrier(a.status, target, spin_limit)) return;   // also orders the zeroing before first use
    for (long long s = 0; s < n_steps; ++s) {
        const L* Tin = (s & 1) ? a.T2 : a.T;
        L* Tout = (s & 1) ? a.T : a.T2;
        for (int64_t t = blockIdx.x; t < ta.n_tiles; t += gridDim.x) {
            const TileView<R> v = tile_view<R, NV>(ta.blocks + ta.block_off[t], view_hg<MODE>(ta), view_mf<MODE>(ta));
            const int64_t base = t * ta.B;
            const int own = (int)min((int64_t)ta.B, a.N_free - base);
            tile_fetch<L, false>(v.halo, v.nh, base, own, Tin, Ts);
            __syncthreads();
            L T0 = lzero<L>();
            NodeVals<R, L> v0{};
            first_node<R, L, MODE>(a, base, own, Ts, T0, v0);
            tile_elements<R, L, NV, MODE, false>(a, tile_regions<MODE>(a, t), v, own, ta.B + 1, ta.rank_shift, Ts, Fn);
            __syncthreads();   // loads complete; Ts is free for the next tile
            tile_nodes<R, L, MODE>(a, base, own, v.deg, ta.B + 1, Fn, T0, v0, Tin, Tout, a.step0 + s);
            __syncthreads();   // table cleared before the next tile writes it
        }
        const bool ok = grid_barrier(a.status, target, spin_limit);
        done = s + 1;
        if (!ok) break;
    }
    if (done & 1) {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N_free; i += stride) a.T[i] = a.T2[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.status->steps_done = a.step0 + done;
}

// resident blocks per SM the staged kernel is compiled for (TPB threads per
// block): 64 registers per thread for one FP32 lane, 128 for FP64 or
// four-lane state
template <typename L, int TPB>
struct StagedOccupancy {
    static constexpr int min_blocks = (sizeof(L) == 4 ? 1024 : 512) / TPB > 0 ? (sizeof(L) == 4 ? 1024 : 512) / TPB : 1;
};

template <typename R, typename L, int NV, int MODE, int TPB>
__global__ void __launch_bounds__(TPB, StagedOccupancy<L, TPB>::min_blocks)
    k_tiled(StepArgs<R, L> a, TileArgs<R> ta, long long n_steps, long long spin_limit) {
    // shared memory: 2 mbarriers | 2 block stages | temperatures | load table
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    const size_t stage_bytes = (size_t)ta.max_block;
    unsigned char* const stage0 = smem + 128;
    unsigned char* const stage1 = smem + 128 + stage_bytes;
    L* const Ts = reinterpret_cast<L*>(smem + 128 + 2 * stage_bytes);
    L* const Fn = reinterpret_cast<L*>(smem + 128 + 2 * stage_bytes + ((size_t)ta.max_local * sizeof(L) + 15) / 16 * 16);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    zero_table(Fn, ta.max_deg * (ta.B + 1));
    __syncthreads();
    unsigned long long target = 0;
    long long done = 0;
    if (!grid_barrier(a.status, target, spin_limit)) return;
    const int64_t first = blockIdx.x;
    const int n_my = first < ta.n_tiles ? (int)((ta.n_tiles - 1 - first) / gridDim.x + 1) : 0;
    // Tiles in launch order: kk = s * n_my + p is tile first + p * gridDim.x of step s (p, the
    // position in the step, is carried along with kk: no 64-bit division in the loop).  With at
    // most two tiles per block both stay in their stages for the whole launch; otherwise tile kk
    // uses stage kk & 1 and its copy is issued two tiles ahead.
    const bool resident = n_my <= 2;
    const long long total = (long long)n_steps * n_my;
    const uint64_t policy = policy_evict_first();
    uint32_t ph0 = 0u, ph1 = 0u;      // per stage: parity of the next completion
    bool pend0 = false, pend1 = false;   // per stage: copy issued and not yet waited for
    auto tile_at = [&](int p) { return first + (int64_t)p * gridDim.x; };
    auto buf_of = [&](long long kk, int p) { return resident ? p : (int)(kk & 1); };
    // tile kk (position p)'s block into its stage (thread 0 copies; every thread records it)
    auto issue = [&](long long kk, int p) {
        const int buf = buf_of(kk, p);
        if (threadIdx.x == 0) {
            const int64_t t = tile_at(p);
            const int64_t o0 = ta.block_off[t], o1 = ta.block_off[t + 1];
            fence_proxy_async();
            mbar_expect_tx(&bar[buf], (uint32_t)(o1 - o0));
            bulk_g2s(buf ? stage1 : stage0, ta.blocks + o0, (uint32_t)(o1 - o0), &bar[buf], policy);
        }
        if (buf) pend1 = true; else pend0 = true;
    };
    // wait for stage buf's outstanding copy: one thread polls, the block
    // synchronises on it; false (in every thread alike) when the wait gave up
    // (a copy whose wait gave up stays pending, so that the drain at exit waits for it again)
    auto land = [&](int buf) -> bool {
        bool ok = true;
        const bool pend = buf ? pend1 : pend0;
        if (pend && threadIdx.x == 0) ok = mbar_wait(&bar[buf], buf ? ph1 : ph0, spin_limit);
        const bool failed = __syncthreads_or(!ok) != 0;
        if (pend && !failed) {
            if (buf) { ph1 ^= 1u; pend1 = false; }
            else { ph0 ^= 1u; pend0 = false; }
        }
        return !failed;
    };
    auto fail_timeout = [&]() {
        if (threadIdx.x == 0) atomicOr(&a.status->flags, STATUS_TIMEOUT);
    };
    auto view_of = [&](long long kk, int p) { return tile_view<R, NV>(buf_of(kk, p) ? stage1 : stage0, view_hg<MODE>(ta), view_mf<MODE>(ta)); };
    // temperatures of tile kk (its stage has landed) into Ts, asynchronously
    auto fetch = [&](long long kk, int p, const L* Tin) {
        const TileView<R> v = view_of(kk, p);
        const int64_t base = tile_at(p) * ta.B;
        tile_fetch<L, true>(v.halo, v.nh, base, (int)min((int64_t)ta.B, a.N_free - base), Tin, Ts);
        cp_async_commit();
    };
    bool stop = false;
    if (total > 0) {
        for (int p = 0; p < 2 && p < n_my; ++p) issue(p, p);
        if (!land(0)) { fail_timeout(); stop = true; }
        else fetch(0, 0, a.T);
    }
    long long kk = 0;
    for (long long s = 0; s < n_steps && !stop; ++s) {
        const L* Tin = (s & 1) ? a.T2 : a.T;
        L* Tout = (s & 1) ? a.T : a.T2;
        for (int i = 0; i < n_my; ++i, ++kk) {
            cp_async_wait_all();
            __syncthreads();   // Ts of this tile complete; the table is clear
            const TileView<R> v = view_of(kk, i);
            const int64_t t = tile_at(i);
            const int64_t base = t * ta.B;
            const int own = (int)min((int64_t)ta.B, a.N_free - base);
            const int deg = v.deg;
            L T0 = lzero<L>();
            NodeVals<R, L> v0{};
            first_node<R, L, MODE>(a, base, own, Ts, T0, v0);
            tile_elements<R, L, NV, MODE, true>(a, tile_regions<MODE>(a, t), v, own, ta.B + 1, ta.rank_shift, Ts, Fn);
            __syncthreads();   // loads complete; this stage and Ts are free
            if (i + 1 < n_my) {   // the next tile of this step: its stage, then its temperatures
                if (!land(buf_of(kk + 1, i + 1))) { fail_timeout(); stop = true; break; }
                fetch(kk + 1, i + 1, Tin);
            }
            if (!resident && kk + 2 < total) issue(kk + 2, i + 2 < n_my ? i + 2 : i + 2 - n_my);
            tile_nodes<R, L, MODE>(a, base, own, deg, ta.B + 1, Fn, T0, v0, Tin, Tout, a.step0 + s);
        }
        if (stop) break;
        cp_async_wait_all();
        const bool ok = grid_barrier(a.status, target, spin_limit);
        done = s + 1;
        if (!ok) break;
        if (s + 1 < n_steps && n_my > 0) {   // the first tile of the next step reads this step's result
            if (!land(buf_of(kk, 0))) { fail_timeout(); break; }
            fetch(kk, 0, Tout);
        }
    }
    cp_async_wait_all();
    // copies nobody consumed (early stop): let them land before the block exits
    if (threadIdx.x == 0) {
        if (pend0) mbar_wait(&bar[0], ph0, spin_limit);
        if (pend1) mbar_wait(&bar[1], ph1, spin_limit);
    }
    if (done & 1) {   // the newest values are in T2: copy them back so that T is current
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N_free; i += stride) a.T[i] = a.T2[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.status->steps_done = a.step0 + done;
}

// ---- replicated-row tiles ------------------------------------------------------
// The staged kernel's data flow with a layout that needs no arithmetic on a
// corner's code.  Two shared arrays share one shape, row stride S (>= the
// tile's owned nodes):
//   Tr: rows 0 .. D-1 each hold the owned nodes' temperatures (row r, entry
//       l: owned node l), then the halo temperatures from entry D*S;
//   Fr: row r, entry l holds owned node l's rank-r element load; from entry
//       D*S a dump area that halo corners write and nobody reads.
// D is the largest rank count of any tile.  Each corner's 16-bit code is the
// byte offset of entry r*S + l (owned corner of rank r) or D*S + h (halo node
// h), so one offset gives both a corner's temperature (Tr) and its load slot
// (Fr): every corner writes its load unconditionally, and owned node l sums
// column l of Fr in rank order (= input element order, as in every other
// kernel) and clears it.  The owned temperatures are fetched into row 0 and
// copied into rows 1 .. deg-1 by the thread that fetched them.

// a corner's byte offset, extracted from the packed codes of an element
template <int NV>
struct RepCodes;
template <>
struct RepCodes<8> {
    static __device__ __forceinline__ void load(const uint16_t* p, int j, uint32_t o[8]) {
        const uint4 v = reinterpret_cast<const uint4*>(p)[j];
        o[0] = v.x & 0xffffu; o[1] = v.x >> 16; o[2] = v.y & 0xffffu; o[3] = v.y >> 16;
        o[4] = v.z & 0xffffu; o[5] = v.z >> 16; o[6] = v.w & 0xffffu; o[7] = v.w >> 16;
    }
};
template <>
struct RepCodes<4> {
    static __device__ __forceinline__ void load(const uint16_t* p, int j, uint32_t o[4]) {
        const uint2 v = reinterpret_cast<const uint2*>(p)[j];
        o[0] = v.x & 0xffffu; o[1] = v.x >> 16; o[2] = v.y & 0xffffu; o[3] = v.y >> 16;
    }
};

// element phase of one replicated-row tile
template <typename R, typename L, int NV, int TPB, bool EXT, typename KL>
__device__ __forceinline__ void rep_elements_k(const KL& kl, const TileView<R>& v, const unsigned char* Tr,
                                               unsigned char* Fr, R eps4) {
    for (int j = threadIdx.x; j < v.ne; j += TPB) {
        uint32_t o[NV];
        RepCodes<NV>::load(v.lc, j, o);
        L tt[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) tt[n] = *reinterpret_cast<const L*>(Tr + o[n]);
        R m[6];
#pragma unroll
        for (int q = 0; q < 6; q += 2) {
            const typename Vec2<R>::type p = reinterpret_cast<const typename Vec2<R>::type*>(v.M + 6 * j)[q / 2];
            m[q] = p.x;
            m[q + 1] = p.y;
        }
        const L ke = element_k<R, NV, L>(tt, kl(j));
        L F[NV];
        tile_loads<EXT, R, L, NV>(v, j, tt, m, ke, eps4, F);
#pragma unroll
        for (int n = 0; n < NV; ++n) *reinterpret_cast<L*>(Fr + o[n]) = F[n];
    }
}

// largest rank count the replicated-row kernels are built for (the host
// refuses meshes with more elements at one node)
template <int NV>
struct RepRows {
    static constexpr int value = NV == 8 ? 8 : 32;
};

template <typename R, typename L, int NV, int MODE, int TPB>
__global__ void __launch_bounds__(TPB, StagedOccupancy<L, TPB>::min_blocks)
    k_tiled_rep(StepArgs<R, L> a, TileArgs<R> ta, long long n_steps, long long spin_limit) {
    constexpr int S = TPB;                      // row stride: one owned node per thread
    constexpr int DMAX = RepRows<NV>::value;
    // shared memory: 2 mbarriers | Tr | Fr | 2 block stages
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    const size_t rep_bytes = ((size_t)(ta.rep_rows * S + ta.max_halo) * sizeof(L) + 15) / 16 * 16;
    unsigned char* const Tr = smem + 128;
    unsigned char* const Fr = smem + 128 + rep_bytes;
    const size_t stage_bytes = (size_t)ta.max_block;
    unsigned char* const stage0 = smem + 128 + 2 * rep_bytes;
    unsigned char* const stage1 = stage0 + stage_bytes;
    L* const T0row = reinterpret_cast<L*>(Tr);
    L* const Thalo = reinterpret_cast<L*>(Tr) + ta.rep_rows * S;
    L* const Fcol = reinterpret_cast<L*>(Fr);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    for (int i = threadIdx.x; i < ta.rep_rows * S; i += TPB) Fcol[i] = lzero<L>();
    __syncthreads();
    unsigned long long target = 0;
    long long done = 0;
    if (!grid_barrier(a.status, target, spin_limit)) return;
    const int64_t first = blockIdx.x;
    const int n_my = first < ta.n_tiles ? (int)((ta.n_tiles - 1 - first) / gridDim.x + 1) : 0;
    const bool resident = n_my <= 2;
    const long long total = (long long)n_steps * n_my;
    const uint64_t policy = policy_evict_first();
    uint32_t ph0 = 0u, ph1 = 0u;
    bool pend0 = false, pend1 = false;
    auto tile_at = [&](int p) { return first + (int64_t)p * gridDim.x; };
    auto buf_of = [&](long long kk, int p) { return resident ? p : (int)(kk & 1); };
    auto issue = [&](long long kk, int p) {
        const int buf = buf_of(kk, p);
        if (threadIdx.x == 0) {
            const int64_t t = tile_at(p);
            const int64_t o0 = ta.block_off[t], o1 = ta.block_off[t + 1];
            fence_proxy_async();
            mbar_expect_tx(&bar[buf], (uint32_t)(o1 - o0));
            bulk_g2s(buf ? stage1 : stage0, ta.blocks + o0, (uint32_t)(o1 - o0), &bar[buf], policy);
        }
        if (buf) pend1 = true; else pend0 = true;
    };
    // every thread waits for stage buf's copy itself (no block barrier); false when its bounded
    // wait gave up: the copy then stays pending (the drain at exit waits for it again), the
    // thread skips what would read the stage, and the block agrees to stop at its next barrier
    auto land = [&](int buf) -> bool {
        if (!(buf ? pend1 : pend0)) return true;
        if (!mbar_wait(&bar[buf], buf ? ph1 : ph0, spin_limit)) return false;
        if (buf) { ph1 ^= 1u; pend1 = false; }
        else { ph0 ^= 1u; pend0 = false; }
        return true;
    };
    auto fail_timeout = [&]() {
        if (threadIdx.x == 0) atomicOr(&a.status->flags, STATUS_TIMEOUT);
    };
    auto view_of = [&](long long kk, int p) {   // (no matrix-free blocks: the host refuses them here)
        return tile_view<R, NV>(buf_of(kk, p) ? stage1 : stage0, view_hg<MODE>(ta), 0);
    };
    // owned temperatures into row 0 (thread l fetches owned node l), halo ones after the rows
    auto fetch = [&](long long kk, int p, const L* Tin) {
        const TileView<R> v = view_of(kk, p);
        const int64_t base = tile_at(p) * ta.B;
        const int own = (int)min((int64_t)ta.B, a.N_free - base);
        if ((int)threadIdx.x < own) cp_async<sizeof(L)>(T0row + threadIdx.x, Tin + base + threadIdx.x);
        for (int h = threadIdx.x; h < v.nh; h += TPB) cp_async<sizeof(L)>(Thalo + h, Tin + v.halo[h]);
        cp_async_commit();
    };
    bool stop = false, failed = false;
    if (total > 0) {
        for (int p = 0; p < 2 && p < n_my; ++p) issue(p, p);
        if (land(0)) fetch(0, 0, a.T);
        else failed = true;
    }
    long long kk = 0;
    for (long long s = 0; s < n_steps && !stop; ++s) {
        const L* Tin = (s & 1) ? a.T2 : a.T;
        L* Tout = (s & 1) ? a.T : a.T2;
        for (int i = 0; i < n_my; ++i, ++kk) {
            const TileView<R> v = view_of(kk, i);
            const int64_t t = tile_at(i);
            const int64_t base = t * ta.B;
            const int own = (int)min((int64_t)ta.B, a.N_free - base);
            const int deg = v.deg;
            const int l = threadIdx.x;
            L T0 = lzero<L>();
            NodeVals<R, L> v0{};
            cp_async_wait_all();
            if (l < own) {   // this thread's own fetch has landed: copy it into the other rows
                T0 = T0row[l];
#pragma unroll
                for (int r = 1; r < DMAX; ++r)
                    if (r < deg) T0row[r * S + l] = T0;
                v0 = node_load<R, L, MODE>(a, base + l);
            }
            if (__syncthreads_or(failed)) { fail_timeout(); stop = true; break; }   // Tr complete; Fr clear
            with_k_laws<MODE>(a, tile_regions<MODE>(a, t), [&](const auto& kl) {
                rep_elements_k<R, L, NV, TPB, (MODE & 2) != 0>(kl, v, Tr, Fr, a.hg_eps4);
            });
            __syncthreads();   // loads complete; this stage and Tr are free
            if (i + 1 < n_my) {   // the next tile of this step: its stage, then its temperatures
                if (land(buf_of(kk + 1, i + 1))) fetch(kk + 1, i + 1, Tin);
                else failed = true;
            }
            if (!resident && kk + 2 < total) issue(kk + 2, i + 2 < n_my ? i + 2 : i + 2 - n_my);
            if (l < own) {   // node phase: column l in rank order, cleared for the next tile
                L F = lzero<L>();
#pragma unroll
                for (int r = 0; r < DMAX; ++r)
                    if (r < deg) {
                        F = F + Fcol[r * S + l];
                        Fcol[r * S + l] = lzero<L>();
                    }
                node_update_v<R, L, MODE>(a, base + l, T0, F, v0, Tout, a.step0 + s);
            }
        }
        if (stop) break;
        cp_async_wait_all();
        const bool ok = grid_barrier(a.status, target, spin_limit);
        done = s + 1;
        if (!ok) break;
        if (s + 1 < n_steps && n_my > 0) {   // the first tile of the next step reads this step's result
            if (land(buf_of(kk, 0))) fetch(kk, 0, Tout);
            else failed = true;
        }
    }
    cp_async_wait_all();
    if (failed && !stop) fail_timeout();   // a wait after the last tile gave up
    // copies nobody consumed (early stop): let them land before the block exits
    if (threadIdx.x == 0) {
        if (pend0) mbar_wait(&bar[0], ph0, spin_limit);
        if (pend1) mbar_wait(&bar[1], ph1, spin_limit);
    }
    if (done & 1) {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N_free; i += stride) a.T[i] = a.T2[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.status->steps_done = a.step0 + done;
}

// MODE bit 0: Kahan-compensated state; bit 1: built with the time-varying
// source, thermal-dose, tabulated-law and region paths (launched only when a
// context enables one)
template <typename R, typename L, int NV, int MODE>
auto tiled_kernel(const TileArgs<R>& ta) {
    if constexpr (sizeof(L) == sizeof(R)) {   // one lane: the replicated rows would not fit four
        if (ta.rep)
            return ta.threads == 128   ? k_tiled_rep<R, L, NV, MODE, 128>
                   : ta.threads == 256 ? k_tiled_rep<R, L, NV, MODE, 256>
                                       : k_tiled_rep<R, L, NV, MODE, kTiledThreads>;
    }
    return !ta.staged           ? k_tiled_direct<R, L, NV, MODE>
           : ta.threads == 256  ? k_tiled<R, L, NV, MODE, 256>
           : ta.threads == 1024 ? k_tiled<R, L, NV, MODE, 1024>
                                : k_tiled<R, L, NV, MODE, kTiledThreads>;
}

template <typename R, typename L, int NV, bool KAHAN>
cudaError_t launch_tiled_impl(const StepArgs<R, L>& a, const TileArgs<R>& ta, int64_t n_steps, LaunchCfg& cfg,
                              cudaStream_t s) {
    constexpr int M = KAHAN ? 1 : 0;
    auto kern = (a.Qs || a.dose || a.n_tab > 0 || a.emat || ta.hourglass || ta.mf) ? tiled_kernel<R, L, NV, M | 2>(ta)
                                                                                   : tiled_kernel<R, L, NV, M>(ta);
    const int b = ta.staged ? ta.threads : 256;
    cudaError_t err = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)ta.smem_bytes);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, b, ta.smem_bytes);
    if (err != cudaSuccess) return err;
    if (cfg.blocks_per_sm > 0) per_sm = std::min(per_sm, cfg.blocks_per_sm);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * cfg.sm_count, ta.n_tiles));
    cfg.grid_used = grid;
    StepArgs<R, L> args = a;
    TileArgs<R> targs = ta;
    long long n = n_steps, lim = cfg.spin_limit;
    void* params[] = {&args, &targs, &n, &lim};
    err = cudaMemsetAsync(&a.status->barrier, 0, sizeof(unsigned long long), s);
    if (err != cudaSuccess) return err;
    return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(b), params, ta.smem_bytes, s);
}

inline int blocks_for(int64_t n, int t) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, INT_MAX));
}

template <typename R, int NV, bool KAHAN>
cudaError_t launch_impl(const StepArgs<R>& a, int64_t n_steps, LaunchCfg& cfg, cudaStream_t s) {
    constexpr int M = KAHAN ? 1 : 0;
    const bool ext = a.Qs || a.dose || a.n_tab > 0 || a.emat || a.A28 || a.W12;
    if (cfg.kernel == FEDFEM_KERNEL_TWO_PHASE) {
        const int b = cfg.block > 0 ? std::min(cfg.block, 256) : 256;
        auto node = ext ? k_node<R, M | 2> : k_node<R, M>;
        auto elem = ext ? k_elem<R, NV, 2> : k_elem<R, NV, 0>;
        for (int64_t k = 0; k < n_steps; ++k) {
            elem<<<blocks_for(a.E, b), b, 0, s>>>(a);
            node<<<blocks_for(a.N_free, b), b, 0, s>>>(a, a.step0 + k);
        }
        return cudaGetLastError();
    }
    // persistent: one cooperative launch, grid = resident blocks
    auto kern = ext ? k_persistent_ext<R, NV, M | 2> : k_persistent<R, NV, M>;
    const int b = 256;
    int per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, b, 0);
    if (err != cudaSuccess) return err;
    if (cfg.blocks_per_sm > 0) per_sm = std::min(per_sm, cfg.blocks_per_sm);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t work = std::max(a.E, a.N_free);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * cfg.sm_count, blocks_for(work, b)));
    cfg.grid_used = grid;
    StepArgs<R> args = a;
    long long n = n_steps, lim = cfg.spin_limit;
    void* params[] = {&args, &n, &lim};
    err = cudaMemsetAsync(&a.status->barrier, 0, sizeof(unsigned long long), s);
    if (err != cudaSuccess) return err;
    return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(b), params, 0, s);
}

}  // namespace

cudaError_t launch_tiled_f64(const StepArgs<double>& a, const TileArgs<double>& t, int64_t n_steps, LaunchCfg& cfg,
                             cudaStream_t s) {
    return t.nv == 8 ? launch_tiled_impl<double, double, 8, false>(a, t, n_steps, cfg, s)
                     : launch_tiled_impl<double, double, 4, false>(a, t, n_steps, cfg, s);
}

cudaError_t launch_tiled_f32(const StepArgs<float>& a, const TileArgs<float>& t, bool kahan, int64_t n_steps,
                             LaunchCfg& cfg, cudaStream_t s) {
    if (t.nv == 8)
        return kahan ? launch_tiled_impl<float, float, 8, true>(a, t, n_steps, cfg, s)
                     : launch_tiled_impl<float, float, 8, false>(a, t, n_steps, cfg, s);
    return kahan ? launch_tiled_impl<float, float, 4, true>(a, t, n_steps, cfg, s)
                 : launch_tiled_impl<float, float, 4, false>(a, t, n_steps, cfg, s);
}

cudaError_t launch_tiled_f32x4(const StepArgs<float, F4>& a, const TileArgs<float>& t, bool kahan, int64_t n_steps,
                               LaunchCfg& cfg, cudaStream_t s) {
    if (t.nv == 8)
        return kahan ? launch_tiled_impl<float, F4, 8, true>(a, t, n_steps, cfg, s)
                     : launch_tiled_impl<float, F4, 8, false>(a, t, n_steps, cfg, s);
    return kahan ? launch_tiled_impl<float, F4, 4, true>(a, t, n_steps, cfg, s)
                 : launch_tiled_impl<float, F4, 4, false>(a, t, n_steps, cfg, s);
}

// staged: 0 direct, 1 staged, 2 staged with replicated rows
template <typename R, typename L, int NV, bool KAHAN>
const void* pick_tiled_k(int staged, int threads) {
    TileArgs<R> ta{};
    ta.staged = staged != 0;
    ta.rep = staged == 2;
    ta.threads = threads;
    return (const void*)tiled_kernel<R, L, NV, KAHAN ? 1 : 0>(ta);
}

template <typename R, typename L>
const void* pick_tiled(int staged, int threads, int nv, bool kahan) {
    if (nv == 8) return kahan ? pick_tiled_k<R, L, 8, true>(staged, threads) : pick_tiled_k<R, L, 8, false>(staged, threads);
    return kahan ? pick_tiled_k<R, L, 4, true>(staged, threads) : pick_tiled_k<R, L, 4, false>(staged, threads);
}

int tiled_blocks_per_sm(int precision, int nv, int staged, int threads, int lanes, size_t smem) {
    const int block = staged ? threads : 256;
    const bool kahan = precision == FEDFEM_FP32_KAHAN;
    const void* k = precision == FEDFEM_FP64 ? pick_tiled<double, double>(staged, threads, nv, false)
                    : lanes == 4            ? pick_tiled<float, F4>(staged, threads, nv, kahan)
                                            : pick_tiled<float, float>(staged, threads, nv, kahan);
    // a size the kernel cannot take is an answer (0 blocks), not an error: clear it
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm;
}

int tiled_threads() { return kTiledThreads; }

cudaError_t launch_steps_f64(const StepArgs<double>& a, int nv, int64_t n_steps, LaunchCfg& cfg, cudaStream_t s) {
    return nv == 8 ? launch_impl<double, 8, false>(a, n_steps, cfg, s) : launch_impl<double, 4, false>(a, n_steps, cfg, s);
}

cudaError_t launch_steps_f32(const StepArgs<float>& a, int nv, bool kahan, int64_t n_steps, LaunchCfg& cfg,
                             cudaStream_t s) {
    if (nv == 8) return kahan ? launch_impl<float, 8, true>(a, n_steps, cfg, s) : launch_impl<float, 8, false>(a, n_steps, cfg, s);
    return kahan ? launch_impl<float, 4, true>(a, n_steps, cfg, s) : launch_impl<float, 4, false>(a, n_steps, cfg, s);
}

}  // namespace fedfem
