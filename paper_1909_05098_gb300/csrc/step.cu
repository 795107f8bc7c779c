// The time loop of Algorithm 1 (lines 8-15): an element phase (Eq. 17 with
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

template <typename R, int NV>
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
    const Law<R> k{a.T_ref, a.k0, a.dk};
    const R ke = element_k<R, NV>(t, k);
    R F[NV];
    if (NV == 8) hex8_loads<R>(t, m, ke, F);
    else tet4_loads<R>(t, m, ke, F);
    R* out = a.slots + e * NV;
    Vec<R>::store4(out, F);
    if (NV == 8) Vec<R>::store4(out + 4, F + 4);
}

__device__ __forceinline__ void flag_range(DevStatus* st, int64_t i, long long step) {
    atomicOr(&st->flags, STATUS_RANGE);
    atomicMin(&st->fail_step, step);
    atomicMin(&st->fail_node, (long long)i);
}

// returns false when the node left [T_lo, T_hi] (or became NaN)
template <typename R, bool KAHAN>
__device__ __forceinline__ void node_phase(const StepArgs<R>& a, int64_t i, long long step) {
    const int64_t s = i >> 5;
    const int lane = (int)(i & 31);
    const int32_t off = a.sell_off[s];
    const int w = (a.sell_off[s + 1] - off) >> 5;
    R F = R(0);
    for (int k = 0; k < w; ++k) F = F + a.slots[a.sell_ids[off + 32 * k + lane]];
    const R T = a.T[i];
    const R u = T - a.T_ref;
    const R rho = a.rho0 + a.drho * u;
    const R c = a.c0 + a.dc * u;
    const R V = a.V[i];
    const R C = (V * rho) * c;
    R r = (a.Q[i] + (a.wbcb * V) * (a.T_a - T)) - F;
    if (i >= a.N_plain) r = r + a.hA[i - a.N_plain] * (a.T_inf - T);
    const R dT = (a.dt * r) / C;
    R Tn;
    if (KAHAN) {
        const R lo = a.Tlo[i];
        const R y = dT + lo;
        Tn = T + y;
        a.Tlo[i] = y - (Tn - T);
    } else {
        Tn = T + dT;
    }
    a.T[i] = Tn;
    if (!(Tn >= a.T_lo && Tn <= a.T_hi)) flag_range(a.status, i, step);
}

template <typename R, int NV>
__global__ void __launch_bounds__(256) k_elem(StepArgs<R> a) {
    if (*(volatile int*)&a.status->flags) return;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < a.E) element_phase<R, NV>(a, e);
}

template <typename R, bool KAHAN>
__global__ void __launch_bounds__(256) k_node(StepArgs<R> a, long long step) {
    if (*(volatile int*)&a.status->flags) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.N_free) node_phase<R, KAHAN>(a, i, step);
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

template <typename R, int NV, bool KAHAN>
__global__ void __launch_bounds__(256) k_persistent(StepArgs<R> a, long long n_steps, long long spin_limit) {
    unsigned long long target = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    long long done = 0;
    if (!grid_barrier(a.status, target, spin_limit)) return;   // flags from an earlier call stop here
    for (long long s = 0; s < n_steps; ++s) {
        for (int64_t e = tid; e < a.E; e += stride) element_phase<R, NV>(a, e);
        if (!grid_barrier(a.status, target, spin_limit)) break;
        for (int64_t i = tid; i < a.N_free; i += stride) node_phase<R, KAHAN>(a, i, a.step0 + s);
        const bool ok = grid_barrier(a.status, target, spin_limit);
        done = s + 1;
        if (!ok) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.status->steps_done = a.step0 + done;
}

inline int blocks_for(int64_t n, int t) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, INT_MAX));
}

template <typename R, int NV, bool KAHAN>
cudaError_t launch_impl(const StepArgs<R>& a, int64_t n_steps, LaunchCfg& cfg, cudaStream_t s) {
    if (cfg.kernel == FEDFEM_KERNEL_TWO_PHASE) {
        const int b = cfg.block > 0 ? std::min(cfg.block, 256) : 256;
        for (int64_t k = 0; k < n_steps; ++k) {
            k_elem<R, NV><<<blocks_for(a.E, b), b, 0, s>>>(a);
            k_node<R, KAHAN><<<blocks_for(a.N_free, b), b, 0, s>>>(a, a.step0 + k);
        }
        return cudaGetLastError();
    }
    // persistent: one cooperative launch, grid = resident blocks
    auto kern = k_persistent<R, NV, KAHAN>;
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

cudaError_t launch_steps_f64(const StepArgs<double>& a, int nv, int64_t n_steps, LaunchCfg& cfg, cudaStream_t s) {
    return nv == 8 ? launch_impl<double, 8, false>(a, n_steps, cfg, s) : launch_impl<double, 4, false>(a, n_steps, cfg, s);
}

cudaError_t launch_steps_f32(const StepArgs<float>& a, int nv, bool kahan, int64_t n_steps, LaunchCfg& cfg,
                             cudaStream_t s) {
    if (nv == 8) return kahan ? launch_impl<float, 8, true>(a, n_steps, cfg, s) : launch_impl<float, 8, false>(a, n_steps, cfg, s);
    return kahan ? launch_impl<float, 4, true>(a, n_steps, cfg, s) : launch_impl<float, 4, false>(a, n_steps, cfg, s);
}

}  // namespace fedfem
