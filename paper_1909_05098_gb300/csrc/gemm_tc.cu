// BF16 GEMM on the 5th-generation tensor cores (tcgen05, accumulators in TMEM)
// for the message-passing surrogate:  C = A B^T (+ bias, optional SiLU),
//   A: M x K bf16, row-major (K contiguous), leading dimension lda;
//   B: N x K bf16, row-major, leading dimension ldb;  N <= 256, N % 16 == 0;
//   K % 64 == 0 (callers pad); rows of A beyond M read as zero.
// One CTA computes a 128 x N tile.  K is consumed in blocks of 64 staged in
// shared memory in the no-swizzle "core matrix" layout (8 rows x 16 bytes per
// core matrix); one elected thread issues the MMAs (M=128, N, K=16 each) and
// commits them to an mbarrier; the four warps then read the accumulator rows
// back from TMEM (one row per thread) for the epilogue.
// Split-K: blockIdx.y takes K range [y*k_chunk, (y+1)*k_chunk) and writes an
// FP32 partial tile; gemm_reduce sums the partials in a fixed order.
// Every wait is bounded; on a timeout the kernel records an error flag, frees
// its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fedfem_internal.h"
#include "tcgen05.cuh"

namespace fedfem {
namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kThreads = 128;

using namespace tc;

// stage rows [r0, r0 + rows) x columns [k0, k0 + 64) of a row-major bf16
// matrix into the core-matrix layout: core (i, j) at ((i * 8) + j) * 128 bytes
__device__ __forceinline__ void stage(unsigned char* sm, const __nv_bfloat16* G, int64_t ld, int rows, int valid,
                                      int64_t r0, int k0) {
    for (int c = threadIdx.x; c < rows * 8; c += blockDim.x) {
        const int r = c >> 3, j = c & 7;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (r < valid) v = *reinterpret_cast<const uint4*>(G + (r0 + r) * ld + k0 + 8 * j);
        *reinterpret_cast<uint4*>(sm + (((r >> 3) * 8 + j) << 7) + ((r & 7) << 4)) = v;
    }
}

__global__ void __launch_bounds__(kThreads) k_gemm_tc(GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                       // 128 x 64 bf16 = 16 KB
    unsigned char* sB = smem + kBM * kBK * 2;       // N x 64 bf16
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncols = g.N <= 32 ? 32 : g.N <= 64 ? 64 : g.N <= 128 ? 128 : 256;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) mbar_init(&bar);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const int64_t m0 = (int64_t)blockIdx.x * kBM;
    const int valid_m = (int)min((int64_t)kBM, (int64_t)g.M - m0);
    const int kbeg = blockIdx.y * g.k_chunk;
    const int kend = min(g.K, kbeg + g.k_chunk);
    const uint32_t idesc = instr_desc(kBM, g.N);
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = kbeg; k0 < kend && ok; k0 += kBK) {
        stage(sA, (const __nv_bfloat16*)g.A, g.lda, kBM, valid_m, m0, k0);
        stage(sB, (const __nv_bfloat16*)g.B, g.ldb, g.N, g.N, 0, k0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor-core reads
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int s = 0; s < kBK / 16; ++s) {
                const uint64_t ad = smem_desc(s_u32(sA) + s * 256, 128, 1024);
                const uint64_t bd = smem_desc(s_u32(sB) + s * 256, 128, 1024);
                mma_bf16(tmem, ad, bd, idesc, (k0 > kbeg || s > 0) ? 1u : 0u);
            }
            mma_commit(&bar);
        }
        // the MMAs must finish reading shared memory before the next block is staged;
        // the decision to stop is made by the whole block at once
        const int timed_out = __syncthreads_or(!mbar_wait(&bar, phase, 2000000000LL));
        if (timed_out) {
            if (threadIdx.x == 0) atomicOr(g.status, 1);
            mbar_wait(&bar, phase, 2000000000LL);   // let MMAs in flight finish before TMEM is freed
            ok = false;
        }
        phase ^= 1u;
        __syncthreads();
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // epilogue: this thread owns row 32*warp + lane of the tile
        const int r = 32 * warp + lane;
        const int64_t row = m0 + r;
        for (int c0 = 0; c0 < g.N; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            if (r < valid_m) {
                if (g.partial) {
                    float* P = g.partial + ((int64_t)blockIdx.y * g.M + row) * g.N + c0;
#pragma unroll
                    for (int i = 0; i < 32; ++i) P[i] = v[i];
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        float z = v[i] + (g.bias ? g.bias[c0 + i] : 0.0f);
                        if (g.Z) g.Z[row * g.ldz + c0 + i] = z;
                        const float y = g.act ? silu(z) : z;
                        if (g.Cf) g.Cf[row * g.ldc + c0 + i] = y;
                        if (g.Cb) ((__nv_bfloat16*)g.Cb)[row * g.ldc + c0 + i] = __float2bfloat16_rn(y);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// C = sum over splits (fixed order) + bias, optional SiLU
__global__ void k_gemm_reduce(GemmArgs g, int splits) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)g.M * g.N) return;
    const int64_t row = i / g.N;
    const int col = (int)(i % g.N);
    float z = 0.0f;
    for (int s = 0; s < splits; ++s) z += g.partial[(int64_t)s * g.M * g.N + i];
    if (g.bias) z += g.bias[col];
    if (g.Z) g.Z[row * g.ldz + col] = z;
    const float y = g.act ? silu(z) : z;
    if (g.Cf) g.Cf[row * g.ldc + col] = y;
    if (g.Cb) ((__nv_bfloat16*)g.Cb)[row * g.ldc + col] = __float2bfloat16_rn(y);
}

}  // namespace

size_t gemm_partial_floats(int M, int N, int K, int k_chunk) {
    const int splits = (K + k_chunk - 1) / k_chunk;
    return splits > 1 ? (size_t)splits * M * N : 0;
}

cudaError_t launch_gemm_tc(GemmArgs g, cudaStream_t s) {
    if (g.N <= 0 || g.N > 256 || g.N % 16 || g.K <= 0 || g.K % kBK || g.M <= 0) return cudaErrorInvalidValue;
    if (g.lda % 8 || g.ldb % 8) return cudaErrorInvalidValue;
    if (g.k_chunk <= 0 || g.k_chunk > g.K) g.k_chunk = g.K;
    g.k_chunk = (g.k_chunk + kBK - 1) / kBK * kBK;
    const int splits = (g.K + g.k_chunk - 1) / g.k_chunk;
    const size_t smem = (size_t)(kBM + g.N) * kBK * 2;
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    GemmArgs ga = g;
    if (splits > 1 && !g.partial) return cudaErrorInvalidValue;
    if (splits == 1) ga.partial = nullptr;
    dim3 grid((unsigned)((g.M + kBM - 1) / kBM), (unsigned)splits);
    k_gemm_tc<<<grid, kThreads, smem, s>>>(ga);
    e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    const int64_t n = (int64_t)g.M * g.N;
    k_gemm_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, splits);
    return cudaGetLastError();
}

}  // namespace fedfem

// C ABI entry point (tests and the surrogate's host code)
extern "C" int fedfem_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K,
                                int k_chunk, const float* bias, int act, float* Z, int64_t ldz, float* Cf,
                                void* Cb, int64_t ldc, float* partial, int* status, void* stream) {
    fedfem::GemmArgs g{};
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb;
    g.M = M; g.N = N; g.K = K; g.k_chunk = k_chunk; g.bias = bias; g.act = act;
    g.Z = Z; g.ldz = ldz; g.Cf = Cf; g.Cb = Cb; g.ldc = ldc; g.partial = partial; g.status = status;
    if (!status) return FEDFEM_E_ARG;
    cudaError_t e = fedfem::launch_gemm_tc(g, (cudaStream_t)stream);
    return e == cudaSuccess ? FEDFEM_OK : (e == cudaErrorInvalidValue ? FEDFEM_E_ARG : FEDFEM_E_CUDA);
}
