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

template <typename R, typename L, bool KAHAN>
__device__ __forceinline__ NodeVals<R, L> node_load(const StepArgs<R, L>& a, int64_t i) {
    NodeVals<R, L> v;
    v.V = a.V[i];
    v.Q = a.Q[i];
    v.hA = i >= a.N_plain ? a.hA[i - a.N_plain] : R(0);
    v.lo = KAHAN ? a.Tlo[i] : lzero<L>();
    return v;
}

template <typename R, typename L, bool KAHAN>
__device__ __forceinline__ void node_update_v(const StepArgs<R, L>& a, int64_t i, L T, L F,
                                              const NodeVals<R, L>& v, L* Tout, long long step) {
    const L u = T - a.T_ref;
    const L rho = fmadd(a.drho, u, a.rho0);
    const L c = fmadd(a.dc, u, a.c0);
    const L C = (v.V * rho) * c;
    L r = fmadd(a.wbcb * v.V, a.T_a - T, v.Q) - F;
    if (i >= a.N_plain) r = fmadd(v.hA, a.T_inf - T, r);
    const L dT = (a.dt * r) / C;
    L Tn;
    if (KAHAN) {
        const L y = dT + v.lo;
        Tn = T + y;
        a.Tlo[i] = y - (Tn - T);
    } else {
        Tn = T + dT;
    }
    Tout[i] = Tn;
    if (!all_in(Tn, a.T_lo, a.T_hi)) flag_range(a.status, i, step);
}

template <typename R, typename L, bool KAHAN>
__device__ __forceinline__ void node_update(const StepArgs<R, L>& a, int64_t i, L T, L F, L* Tout, long long step) {
    node_update_v<R, L, KAHAN>(a, i, T, F, node_load<R, L, KAHAN>(a, i), Tout, step);
}

// gather of node i's element loads from the global slots, in its fixed order
template <typename R, bool KAHAN>
__device__ __forceinline__ void node_phase(const StepArgs<R>& a, int64_t i, long long step) {
    const int64_t s = i >> 5;
    const int lane = (int)(i & 31);
    const int32_t off = a.sell_off[s];
    const int w = (a.sell_off[s + 1] - off) >> 5;
    R F = R(0);
    for (int k = 0; k < w; ++k) F = F + a.slots[a.sell_ids[off + 32 * k + lane]];
    node_update<R, R, KAHAN>(a, i, a.T[i], F, a.T, step);
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

// ---- tiled persistent kernel ------------------------------------------------
// Tile t owns free nodes [t*B, t*B + own).  Its constant data (element
// matrices, 16-bit local connectivity, 16-bit gather lists, halo ids, slice
// offsets) is one packed block that a bulk (TMA) copy brings into a shared-
// memory stage; two stages alternate, so the next tile's block (and, across
// the grid barrier, the next step's first block) is in flight while the
// current tile computes.  Per tile: stage owned + halo temperatures, compute
// the loads of every element touching an owned node into shared memory, sum
// each owned node's loads in its fixed order, update.  T is double-buffered
// (tiles read their neighbours' nodes as halo), so one grid barrier per step.

constexpr int kTiledThreads = 512;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
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

template <int NV>
struct LConn;
template <>
struct LConn<8> {
    static __device__ __forceinline__ void load(const uint16_t* p, int j, int c[8]) {
        const uint4 v = reinterpret_cast<const uint4*>(p)[j];
        c[0] = v.x & 0xffff; c[1] = v.x >> 16; c[2] = v.y & 0xffff; c[3] = v.y >> 16;
        c[4] = v.z & 0xffff; c[5] = v.z >> 16; c[6] = v.w & 0xffff; c[7] = v.w >> 16;
    }
};
template <>
struct LConn<4> {
    static __device__ __forceinline__ void load(const uint16_t* p, int j, int c[4]) {
        const uint2 v = reinterpret_cast<const uint2*>(p)[j];
        c[0] = v.x & 0xffff; c[1] = v.x >> 16; c[2] = v.y & 0xffff; c[3] = v.y >> 16;
    }
};

template <typename R, typename L, int NV, bool KAHAN>
__device__ __forceinline__ void tile_compute(const StepArgs<R, L>& a, const TileArgs<R>& ta, int64_t t,
                                             const unsigned char* blk, const L* Tin, L* Tout, long long step, L* Ts,
                                             L* Fs) {
    const int4 hdr = *reinterpret_cast<const int4*>(blk);
    const int ne = hdr.x, ne_pad = hdr.y, nh = hdr.z, G = hdr.w;
    const R* M = reinterpret_cast<const R*>(blk + 16);
    const uint16_t* lc = reinterpret_cast<const uint16_t*>(blk + 16 + 6 * (size_t)ne_pad * sizeof(R));
    const uint16_t* gat = lc + NV * ne_pad;
    const int32_t* halo = reinterpret_cast<const int32_t*>(gat + G);
    const int32_t* so = halo + ((nh + 3) & ~3);
    const int64_t base = t * ta.B;
    const int own = (int)min((int64_t)ta.B, a.N_free - base);
    // this thread's first owned node: its data and temperature are fetched now,
    // so the loads overlap the staging and element phases
    const int l0 = threadIdx.x;
    const bool has0 = l0 < own;
    NodeVals<R, L> v0{};
    L T0 = lzero<L>();
    if (has0) {
        v0 = node_load<R, L, KAHAN>(a, base + l0);
        T0 = Tin[base + l0];
        Ts[l0] = T0;
    }
    for (int l = l0 + blockDim.x; l < own; l += blockDim.x) Ts[l] = Tin[base + l];
    for (int h = threadIdx.x; h < nh; h += blockDim.x) Ts[own + h] = Tin[halo[h]];
    __syncthreads();
    const Law<R> k{a.T_ref, a.k0, a.dk};
    for (int j = threadIdx.x; j < ne; j += blockDim.x) {
        int c[NV];
        LConn<NV>::load(lc, j, c);
        L tt[NV];
#pragma unroll
        for (int n = 0; n < NV; ++n) tt[n] = Ts[c[n]];
        R m[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) m[q] = M[q * ne_pad + j];
        const L ke = element_k<R, NV, L>(tt, k);
        L F[NV];
        if (NV == 8) hex8_loads<R, L>(tt, m, ke, F);
        else tet4_loads<R, L>(tt, m, ke, F);
#pragma unroll
        for (int n = 0; n < NV; ++n) Fs[n * ne_pad + j] = F[n];
    }
    __syncthreads();
    // Ts is not read below this point (own temperatures come from registers or
    // are re-read from Tin), so the next tile may overwrite it without a barrier
    for (int l = l0; l < own; l += blockDim.x) {
        const int sl = l >> 5, lane = l & 31;
        const int32_t off = so[sl];
        const int w = (so[sl + 1] - off) >> 5;
        const uint16_t* g = gat + off + lane;
        L F = lzero<L>();
        for (int q = 0; q < w; ++q) F = F + Fs[g[32 * q]];
        if (l == l0) node_update_v<R, L, KAHAN>(a, base + l, T0, F, v0, Tout, step);
        else node_update<R, L, KAHAN>(a, base + l, Tin[base + l], F, Tout, step);
    }
}

// Direct variant: the same per-tile blocks read straight from global memory
// (coalesced within a tile), shared memory only for T and the element loads,
// so more blocks fit on an SM.
// resident blocks per SM the direct tiled kernel is compiled for: one FP32
// lane fits 6 blocks of 256 threads, FP64 or four-lane state needs about twice
// the registers
template <typename L>
struct DirectOccupancy {
    static constexpr int min_blocks = sizeof(L) >= 8 ? 3 : 6;
};

template <typename R, typename L, int NV, bool KAHAN>
__global__ void __launch_bounds__(256, DirectOccupancy<L>::min_blocks) k_tiled_direct(StepArgs<R, L> a, TileArgs<R> ta, long long n_steps,
                                                      long long spin_limit) {
    extern __shared__ __align__(128) unsigned char smem[];
    L* Ts = reinterpret_cast<L*>(smem);
    L* Fs = Ts + ta.max_local;
    if (threadIdx.x == 0) Fs[ta.fs_words - 1] = lzero<L>();   // the zero cell every gather pad points at
    unsigned long long target = 0;
    long long done = 0;
    if (!grid_barrier(a.status, target, spin_limit)) return;
    for (long long s = 0; s < n_steps; ++s) {
        const L* Tin = (s & 1) ? a.T2 : a.T;
        L* Tout = (s & 1) ? a.T : a.T2;
        for (int64_t t = blockIdx.x; t < ta.n_tiles; t += gridDim.x)
            tile_compute<R, L, NV, KAHAN>(a, ta, t, ta.blocks + ta.block_off[t], Tin, Tout, a.step0 + s, Ts, Fs);
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

template <typename R, typename L, int NV, bool KAHAN>
__global__ void __launch_bounds__(kTiledThreads) k_tiled(StepArgs<R, L> a, TileArgs<R> ta, long long n_steps,
                                                         long long spin_limit) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    unsigned char* const stage0 = smem + 128;
    unsigned char* const stage1 = smem + 128 + ta.max_block;
    L* Ts = reinterpret_cast<L*>(smem + 128 + 2 * (size_t)ta.max_block);
    L* Fs = Ts + ta.max_local;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        Fs[ta.fs_words - 1] = lzero<L>();   // the zero cell every gather pad points at
    }
    __syncthreads();
    unsigned long long target = 0;
    long long done = 0;
    if (!grid_barrier(a.status, target, spin_limit)) return;
    const int64_t first = blockIdx.x;
    const int64_t n_my = first < ta.n_tiles ? (ta.n_tiles - 1 - first) / gridDim.x + 1 : 0;
    const bool single = n_my == 1;   // one tile per block: its block stays resident across steps
    uint32_t ph0 = 0u, ph1 = 0u;
    bool pending = false;
    int pbuf = 0;
    auto issue = [&](int64_t t, int buf) {
        const int64_t o = ta.block_off[t];
        const uint32_t bytes = (uint32_t)(ta.block_off[t + 1] - o);
        mbar_expect_tx(&bar[buf], bytes);
        bulk_g2s(buf ? stage1 : stage0, ta.blocks + o, bytes, &bar[buf]);
    };
    if (n_my > 0) {
        if (threadIdx.x == 0) issue(first, 0);
        pending = true;
        pbuf = 0;
    }
    long long kk = 0;
    bool stop = false;
    for (long long s = 0; s < n_steps && !stop; ++s) {
        const L* Tin = (s & 1) ? a.T2 : a.T;
        L* Tout = (s & 1) ? a.T : a.T2;
        for (int64_t i = 0; i < n_my; ++i, ++kk) {
            const int64_t t = first + i * gridDim.x;
            const int buf = single ? 0 : (int)(kk & 1);
            if (pending && pbuf == buf) {
                const uint32_t ph = buf ? ph1 : ph0;
                if (!mbar_wait(&bar[buf], ph, spin_limit)) {
                    if (threadIdx.x == 0) atomicOr(&a.status->flags, STATUS_TIMEOUT);
                    mbar_wait(&bar[buf], ph, spin_limit);   // the copy is from global memory: let it land
                    return;
                }
                if (buf) ph1 ^= 1u; else ph0 ^= 1u;
                pending = false;
            }
            __syncthreads();   // every thread is done with the other stage
            if (!single && (i + 1 < n_my || s + 1 < n_steps)) {
                const int64_t tn = (i + 1 < n_my) ? t + gridDim.x : first;
                if (threadIdx.x == 0) {
                    fence_proxy_async();
                    issue(tn, buf ^ 1);
                }
                pending = true;
                pbuf = buf ^ 1;
            }
            tile_compute<R, L, NV, KAHAN>(a, ta, t, buf ? stage1 : stage0, Tin, Tout, a.step0 + s, Ts, Fs);
        }
        const bool ok = grid_barrier(a.status, target, spin_limit);
        done = s + 1;
        if (!ok) stop = true;
    }
    if (pending) mbar_wait(&bar[pbuf], pbuf ? ph1 : ph0, spin_limit);   // a prefetch nobody consumed
    if (done & 1) {   // the newest values are in T2: copy them back so that T is current
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N_free; i += stride) a.T[i] = a.T2[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.status->steps_done = a.step0 + done;
}

template <typename R, typename L, int NV, bool KAHAN>
cudaError_t launch_tiled_impl(const StepArgs<R, L>& a, const TileArgs<R>& ta, int64_t n_steps, LaunchCfg& cfg,
                              cudaStream_t s) {
    auto kern = ta.staged ? k_tiled<R, L, NV, KAHAN> : k_tiled_direct<R, L, NV, KAHAN>;
    const int b = ta.staged ? kTiledThreads : 256;
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

template <typename R, typename L>
const void* pick_tiled(int staged, int nv, bool kahan) {
    if (staged) {
        if (nv == 8) return kahan ? (const void*)k_tiled<R, L, 8, true> : (const void*)k_tiled<R, L, 8, false>;
        return kahan ? (const void*)k_tiled<R, L, 4, true> : (const void*)k_tiled<R, L, 4, false>;
    }
    if (nv == 8) return kahan ? (const void*)k_tiled_direct<R, L, 8, true> : (const void*)k_tiled_direct<R, L, 8, false>;
    return kahan ? (const void*)k_tiled_direct<R, L, 4, true> : (const void*)k_tiled_direct<R, L, 4, false>;
}

int tiled_blocks_per_sm(int precision, int nv, int staged, int lanes, size_t smem) {
    const int block = staged ? kTiledThreads : 256;
    const bool kahan = precision == FEDFEM_FP32_KAHAN;
    const void* k = precision == FEDFEM_FP64 ? pick_tiled<double, double>(staged, nv, false)
                    : lanes == 4            ? pick_tiled<float, F4>(staged, nv, kahan)
                                            : pick_tiled<float, float>(staged, nv, kahan);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem) != cudaSuccess) return 0;
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
