// Message-passing surrogate: forward, backward and Adam on the GPU.
//
// The paper points to neural networks for stable dynamics as future work
// (Section 4); this surrogate advances the FED-FEM field many explicit steps
// at once and is checked against (and replaced by) the plain explicit path.
// Network (hidden H = 64, L layers, encode-process-decode):
//   h = SiLU(W_ne x + b_ne),  e = SiLU(W_ee f + b_ee)
//   per layer: msg = SiLU(W_e [e; h_src; h_dst] + b_e); e += msg;
//              a_i = sum of msg into i;  h += SiLU(W_n [h; a] + b_n)
//   y = w_d . h + b_d
// GEMMs run on the tensor cores (gemm_tc.cu) with BF16 operands and FP32
// accumulation; the residual states h, e and all reductions are FP32.  Every
// sum has a fixed order (CSR gathers, two-pass column sums), so a training
// step is deterministic.  Parameter layout (flat, row-major):
//   W_ne[H][5] b_ne[H] W_ee[H][4] b_ee[H] {W_e[H][3H] b_e[H] W_n[H][2H] b_n[H]} x L  w_d[H] b_d[1]
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fedfem_internal.h"
#include "tcgen05.cuh"

using bf16 = __nv_bfloat16;

namespace fedfem {
namespace {

constexpr int H = 64;
constexpr int NIN = 5, EIN = 4;
constexpr int kT = 256;

inline unsigned grid(int64_t n, int t = kT) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ float sig(float z) { return 1.0f / (1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_f(float z) { return z * sig(z); }
__device__ __forceinline__ float dsilu_f(float z) {
    const float s = sig(z);
    return s * (1.0f + z * (1.0f - s));
}

__global__ void k_encode(int64_t R, int nin, const float* x, const float* W, const float* b, float* z, float* h) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * H) return;
    const int64_t r = i / H;
    const int k = (int)(i % H);
    float acc = b[k];
    for (int j = 0; j < nin; ++j) acc += W[k * nin + j] * x[r * nin + j];
    z[i] = acc;
    h[i] = silu_f(acc);
}

__global__ void k_bcast_edges(int64_t B, int64_t E, const float* e0, float* e) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B * E * H) e[i] = e0[i % (E * H)];
}

// Xe[b*E + m] = bf16([e; h_src; h_dst])
__global__ void k_build_xe(int64_t B, int64_t E, int64_t N, const int32_t* src, const int32_t* dst, const float* e,
                           const float* h, bf16* Xe) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * E * 3 * H) return;
    const int64_t row = i / (3 * H);
    const int c = (int)(i % (3 * H));
    const int64_t b = row / E, m = row % E;
    float v;
    if (c < H) v = e[row * H + c];
    else if (c < 2 * H) v = h[(b * N + src[m]) * H + (c - H)];
    else v = h[(b * N + dst[m]) * H + (c - 2 * H)];
    Xe[i] = __float2bfloat16_rn(v);
}

__global__ void k_add(int64_t n, float* y, const float* x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}

// a[b*N + i] = sum of msg over edges into i (edges sorted by destination)
__global__ void k_aggregate(int64_t B, int64_t E, int64_t N, const int32_t* in_ptr, const float* msg, float* a) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * N * H) return;
    const int64_t row = t / H;
    const int k = (int)(t % H);
    const int64_t b = row / N, i = row % N;
    float s = 0.0f;
    for (int32_t m = in_ptr[i]; m < in_ptr[i + 1]; ++m) s += msg[(b * E + m) * H + k];
    a[t] = s;
}

// Xn = bf16([h; a])
__global__ void k_build_xn(int64_t R, const float* h, const float* a, bf16* Xn) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * 2 * H) return;
    const int64_t r = i / (2 * H);
    const int c = (int)(i % (2 * H));
    Xn[i] = __float2bfloat16_rn(c < H ? h[r * H + c] : a[r * H + c - H]);
}

__global__ void k_decode(int64_t R, const float* h, const float* w, const float* b, float* y) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    float s = b[0];
    for (int k = 0; k < H; ++k) s += w[k] * h[r * H + k];
    y[r] = s;
}

// residual r = (y - t) * mask, dy = 2 r / count, per-block partial sums of r^2
__global__ void k_loss(int64_t B, int64_t N, const float* y, const float* t, const float* mask, float inv_count,
                       float* dy, float* part) {
    __shared__ float sh[kT];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float r2 = 0.0f;
    if (i < B * N) {
        const float r = (y[i] - t[i]) * mask[i % N];
        dy[i] = 2.0f * r * inv_count;
        r2 = r * r;
    }
    sh[threadIdx.x] = r2;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_dec_bwd(int64_t R, const float* dy, const float* w, float* dh) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < R * H) dh[i] = dy[i / H] * w[i % H];
}

// out[k*J + j] = sum_r A[r*lda + k] * (X ? X[r*ldx + j] : 1), two passes, fixed order
constexpr int kChunk = 256;
__global__ void k_colsum_part(int64_t R, int K, int J, const float* A, int lda, const float* X, int ldx,
                              float* part) {
    const int o = blockIdx.y * blockDim.x + threadIdx.x;
    if (o >= K * J) return;
    const int k = o / J, j = o % J;
    const int64_t r0 = (int64_t)blockIdx.x * kChunk, r1 = min(R, r0 + kChunk);
    float s = 0.0f;
    for (int64_t r = r0; r < r1; ++r) s += A[r * lda + k] * (X ? X[r * ldx + j] : 1.0f);
    part[(int64_t)blockIdx.x * K * J + o] = s;
}
__global__ void k_colsum_final(int chunks, int KJ, const float* part, float* out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= KJ) return;
    float s = 0.0f;
    for (int c = 0; c < chunks; ++c) s += part[(int64_t)c * KJ + o];
    out[o] = s;
}

// dz = d * SiLU'(z): fp32 and bf16 copies
__global__ void k_dsilu(int64_t n, const float* d, const float* z, float* dz, bf16* dzb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = d[i] * dsilu_f(z[i]);
    dz[i] = v;
    dzb[i] = __float2bfloat16_rn(v);
}

// out[c*ldo + r] = in[r*ldi + c] for r < R (rows R..Rp zero), c < C; 32x32 tiles
__global__ void k_transpose(int64_t R, int64_t Rp, int C, const bf16* in, int64_t ldi, bf16* out, int64_t ldo) {
    __shared__ bf16 tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t r = r0 + y;
        const int c = c0 + threadIdx.x;
        bf16 v = __float2bfloat16_rn(0.0f);
        if (r < R && c < C) v = in[r * ldi + c];
        tile[y][threadIdx.x] = v;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y;
        const int64_t r = r0 + threadIdx.x;
        if (c < C && r < Rp) out[(int64_t)c * ldo + r] = tile[threadIdx.x][y];
    }
}

// dh += dXn[:, :H]
__global__ void k_node_bwd(int64_t R, const float* dXn, float* dh) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < R * H) dh[i] += dXn[(i / H) * 2 * H + i % H];
}

// dmsg = de + da[dst];  dz = dmsg * SiLU'(z_e)
__global__ void k_dmsg(int64_t B, int64_t E, int64_t N, const int32_t* dst, const float* de, const float* dXn,
                       const float* ze, float* dz, bf16* dzb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * E * H) return;
    const int64_t row = i / H;
    const int k = (int)(i % H);
    const int64_t b = row / E, m = row % E;
    const float d = de[i] + dXn[(b * N + dst[m]) * 2 * H + H + k];
    const float v = d * dsilu_f(ze[i]);
    dz[i] = v;
    dzb[i] = __float2bfloat16_rn(v);
}

// de += dXe[:, :H]
__global__ void k_edge_bwd(int64_t R, const float* dXe, float* de) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < R * H) de[i] += dXe[(i / H) * 3 * H + i % H];
}

// dh[i] += sum over edges out of i of dXe[:, H:2H] + over edges into i of dXe[:, 2H:3H]
__global__ void k_node_scatter(int64_t B, int64_t E, int64_t N, const int32_t* out_ptr, const int32_t* out_edge,
                               const int32_t* in_ptr, const float* dXe, float* dh) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * N * H) return;
    const int64_t row = t / H;
    const int k = (int)(t % H);
    const int64_t b = row / N, i = row % N;
    float s = 0.0f;
    for (int32_t p = out_ptr[i]; p < out_ptr[i + 1]; ++p) s += dXe[(b * E + out_edge[p]) * 3 * H + H + k];
    for (int32_t m = in_ptr[i]; m < in_ptr[i + 1]; ++m) s += dXe[(b * E + m) * 3 * H + 2 * H + k];
    dh[t] += s;
}

// dz_ee[m] = (sum_b de[b, m]) * SiLU'(z_ee[m])
__global__ void k_edge_enc_bwd(int64_t B, int64_t E, const float* de, const float* zee, float* dz) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= E * H) return;
    float s = 0.0f;
    for (int64_t b = 0; b < B; ++b) s += de[b * E * H + i];
    dz[i] = s * dsilu_f(zee[i]);
}

__global__ void k_dsilu_f32(int64_t n, const float* d, const float* z, float* dz) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dz[i] = d[i] * dsilu_f(z[i]);
}

__global__ void k_adam(int64_t n, float* P, const float* G, float* m, float* v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// W (rows x cols fp32) -> Wb (bf16 same layout) and WbT (cols x rows)
__global__ void k_weights_bf16(int rows, int cols, const float* W, bf16* Wb, bf16* WbT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const int r = i / cols, c = i % cols;
    const bf16 v = __float2bfloat16_rn(W[i]);
    Wb[i] = v;
    WbT[c * rows + r] = v;
}

__global__ void k_edge_features(int64_t E, const int32_t* src, const int32_t* dst, const double* xyz, double inv_h,
                                float* f) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= E) return;
    double d[3], n2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        d[c] = (xyz[3 * (int64_t)dst[m] + c] - xyz[3 * (int64_t)src[m] + c]) * inv_h;
        n2 += d[c] * d[c];
    }
    for (int c = 0; c < 3; ++c) f[m * 4 + c] = (float)d[c];
    f[m * 4 + 3] = (float)sqrt(n2);
}

// node inputs [(T - 37)/10, q/1e7, k(T)/k0, c(T)/c0, Dirichlet]
__global__ void k_features(int64_t B, int64_t N, const float* T, const float* q, const unsigned char* D,
                           fedfem_material m, float* x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * N) return;
    const float t = T[i];
    x[i * 5 + 0] = (t - 37.0f) * 0.1f;
    x[i * 5 + 1] = q[i] * 1e-7f;
    x[i * 5 + 2] = (float)((m.k0 + m.dk * ((double)t - m.T_ref)) / m.k0);
    x[i * 5 + 3] = (float)((m.c0 + m.dc * ((double)t - m.T_ref)) / m.c0);
    x[i * 5 + 4] = D ? (float)D[i % N] : 0.0f;
}

// ---- fused inference ---------------------------------------------------------
// One layer of the network in two tensor-core kernels, without the training
// caches: the edge kernel gathers [e; h_src; h_dst] for 128 edges straight into
// shared memory (BF16, core-matrix layout), multiplies by W_e^T (tcgen05, FP32
// accumulators in TMEM), and in its epilogue forms msg = SiLU(acc + b_e),
// e += msg and the sum of msg over each destination node's in-edges (edge tiles
// hold whole in-edge lists, summed in edge order); the node kernel gathers
// [h; a], multiplies by W_n^T and adds SiLU(acc + b_n) to h in place (on the
// last layer also the decoder).  Rounding points, the MMA sequence and every
// summation order are those of the unfused forward, so both give the same
// numbers.

constexpr int kRows = 128;                      // rows (edges or nodes) per tile
constexpr int kPad = 68;                        // floats per padded FP32 row in shared memory
constexpr uint32_t kKBlock = kRows * 64 * 2;    // bytes of one 128 x 64 BF16 K-block
constexpr uint32_t kWBlock = 64 * 64 * 2;       // bytes of one 64 x 64 BF16 weight K-block

struct EdgeTile {
    int32_t m0, count, n0, n1;   // edges [m0, m0 + count) are the in-edges of nodes [n0, n1)
};

__device__ __forceinline__ uint4 pack8(float4 a, float4 b) {
    uint4 r;
    __nv_bfloat162 p;
    p = __floats2bfloat162_rn(a.x, a.y); r.x = *reinterpret_cast<uint32_t*>(&p);
    p = __floats2bfloat162_rn(a.z, a.w); r.y = *reinterpret_cast<uint32_t*>(&p);
    p = __floats2bfloat162_rn(b.x, b.y); r.z = *reinterpret_cast<uint32_t*>(&p);
    p = __floats2bfloat162_rn(b.z, b.w); r.w = *reinterpret_cast<uint32_t*>(&p);
    return r;
}

// W (64 x K, row-major BF16) into K/64 core-matrix blocks of 64 x 64
__device__ __forceinline__ void stage_weights(unsigned char* sB, const bf16* W, int K) {
    const int chunks = K / 8;
    for (int c = threadIdx.x; c < 64 * chunks; c += blockDim.x) {
        const int r = c / chunks, kc = c % chunks;
        const uint4 v = *reinterpret_cast<const uint4*>(W + (int64_t)r * K + 8 * kc);
        *reinterpret_cast<uint4*>(sB + (kc >> 3) * kWBlock + tc::core_offset(r, 8 * (kc & 7))) = v;
    }
}

// SEG 64-wide FP32 row segments of tile row r into K-blocks 0..SEG-1 (BF16):
// all of the lane's loads are issued before any conversion, so a warp keeps
// 4 x SEG loads in flight instead of a chain of dependent ones
template <int SEG>
__device__ __forceinline__ void stage_rows(unsigned char* sA, int r, const float* const (&row)[SEG], bool valid) {
    const int lane = threadIdx.x & 31;
    float4 v[SEG][2][2];
#pragma unroll
    for (int sg = 0; sg < SEG; ++sg)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int j = (lane >> 3) + 4 * q;
            if (valid) {
                v[sg][q][0] = reinterpret_cast<const float4*>(row[sg])[2 * j];
                v[sg][q][1] = reinterpret_cast<const float4*>(row[sg])[2 * j + 1];
            } else {
                v[sg][q][0] = v[sg][q][1] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
    for (int sg = 0; sg < SEG; ++sg)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int j = (lane >> 3) + 4 * q;
            *reinterpret_cast<uint4*>(sA + sg * kKBlock + tc::core_offset(r, 8 * j)) = pack8(v[sg][q][0], v[sg][q][1]);
        }
}

// issue the K/16 MMAs of one tile (thread 0) and wait for them (every thread);
// false when the bounded wait gave up (then the copies in flight are waited
// for once more, so TMEM can be freed)
__device__ __forceinline__ bool mma_tile(uint32_t tmem, const unsigned char* sA, const unsigned char* sB, int kblocks,
                                         uint64_t* bar, uint32_t& phase, int* status, long long limit) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor-core reads
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc = tc::instr_desc(kRows, 64);
        for (int kb = 0; kb < kblocks; ++kb)
#pragma unroll
            for (int st = 0; st < 4; ++st)
                tc::mma_bf16(tmem, tc::smem_desc(tc::s_u32(sA + kb * kKBlock) + st * 256, 128, 1024),
                             tc::smem_desc(tc::s_u32(sB + kb * kWBlock) + st * 256, 128, 1024), idesc,
                             (kb > 0 || st > 0) ? 1u : 0u);
        tc::mma_commit(bar);
    }
    const int timed_out = __syncthreads_or(!tc::mbar_wait(bar, phase, limit));
    if (timed_out) {
        if (threadIdx.x == 0) atomicOr(status, 1);
        tc::mbar_wait(bar, phase, limit);
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return !timed_out;
}

struct EdgeLayerArgs {
    int B;
    int64_t N, E;
    const int32_t *src, *dst, *in_ptr;
    const EdgeTile* tiles;
    int n_tiles;
    const float* e_in;        // B x E x H, or the shared E x H encoder output (e_in_stride 0)
    int64_t e_in_stride;
    float* e_out;             // B x E x H (may alias e_in); null on the last layer
    const float* h;           // B x N x H
    float* a;                 // B x N x H
    const bf16* W;            // H x 3H
    const float* bias;
    int* status;
    long long limit;
};

constexpr int kFusedThreads = 256;   // 8 warps: two per TMEM lane quadrant, one per 32-column half

// epilogue coordinates of this thread: TMEM lane quadrant (rows 32q..32q+31) and column half
__device__ __forceinline__ int epi_row() { return 32 * ((threadIdx.x >> 5) & 3) + (threadIdx.x & 31); }
__device__ __forceinline__ int epi_col0() { return 32 * (threadIdx.x >> 7); }

__global__ void __launch_bounds__(kFusedThreads, 3) k_edge_layer(EdgeLayerArgs g) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                          // 3 K-blocks; after the MMAs: messages, 128 x kPad FP32
    unsigned char* sB = smem + 3 * kKBlock;            // W_e, 3 K-blocks
    float* msgS = reinterpret_cast<float*>(sA);
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(tc::s_u32(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) tc::mbar_init(&bar);
    stage_weights(sB, g.W, 3 * H);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    uint32_t phase = 0;
    const int nw = blockDim.x >> 5;
    const int64_t items = (int64_t)g.n_tiles * g.B;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int t = (int)(item % g.n_tiles);
        const int64_t b = item / g.n_tiles;
        const EdgeTile T = g.tiles[t];
        for (int i = warp; i < kRows / 8; i += nw) {
            const int r = 8 * i + (lane & 7);
            const bool valid = r < T.count;
            const int64_t m = T.m0 + (valid ? r : 0);   // read only for valid rows
            const int32_t s = valid ? g.src[m] : 0, d = valid ? g.dst[m] : 0;
            const float* const rows[3] = {g.e_in + b * g.e_in_stride + m * H, g.h + (b * g.N + s) * H,
                                          g.h + (b * g.N + d) * H};
            stage_rows<3>(sA, r, rows, valid);
        }
        if (!mma_tile(tmem, sA, sB, 3, &bar, phase, g.status, g.limit)) break;
        // epilogue: row r (TMEM lane r), columns c0..c0+31; e is re-read (it was
        // just staged, so it comes from L2) and written back, the messages go to
        // shared memory (over the A operand, which the MMAs no longer read)
        {
            const int r = epi_row(), c0 = epi_col0();
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(r & ~31) << 16) + (uint32_t)c0, v);
            if (r < T.count) {
                const int64_t m = T.m0 + r;
                const float* er = g.e_in + b * g.e_in_stride + m * H + c0;
                float* mr = msgS + r * kPad + c0;
                float* eo = g.e_out ? g.e_out + (b * g.E + m) * H + c0 : nullptr;
#pragma unroll
                for (int c = 0; c < 32; c += 4) {
                    float4 msg;
                    msg.x = tc::silu(v[c] + g.bias[c0 + c]);
                    msg.y = tc::silu(v[c + 1] + g.bias[c0 + c + 1]);
                    msg.z = tc::silu(v[c + 2] + g.bias[c0 + c + 2]);
                    msg.w = tc::silu(v[c + 3] + g.bias[c0 + c + 3]);
                    *reinterpret_cast<float4*>(mr + c) = msg;
                    if (eo) {
                        float4 ev = *reinterpret_cast<const float4*>(er + c);
                        ev.x = ev.x + msg.x; ev.y = ev.y + msg.y; ev.z = ev.z + msg.z; ev.w = ev.w + msg.w;
                        *reinterpret_cast<float4*>(eo + c) = ev;
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        // a_n = sum of the messages over n's in-edges, in edge order
        {
            const int c = threadIdx.x & 63;
            for (int n = T.n0 + (threadIdx.x >> 6); n < T.n1; n += blockDim.x >> 6) {
                float acc = 0.0f;
                for (int32_t m = g.in_ptr[n]; m < g.in_ptr[n + 1]; ++m) acc += msgS[(m - T.m0) * kPad + c];
                g.a[(b * g.N + n) * H + c] = acc;
            }
        }
        __syncthreads();   // shared buffers are restaged by the next item
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

struct NodeLayerArgs {
    int64_t R;                // rows: batch x nodes
    float* h;                 // R x H, updated in place
    const float* a;           // R x H
    const bf16* W;            // H x 2H
    const float* bias;
    const float* wd;          // decoder (last layer), else null
    const float* bd;
    float* y;                 // R decoder outputs (last layer)
    int* status;
    long long limit;
};

__global__ void __launch_bounds__(kFusedThreads, 3) k_node_layer(NodeLayerArgs g) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                          // 2 K-blocks: [h | a]
    unsigned char* sB = smem + 2 * kKBlock;            // W_n, 2 K-blocks
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(tc::s_u32(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) tc::mbar_init(&bar);
    stage_weights(sB, g.W, 2 * H);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    uint32_t phase = 0;
    const int nw = blockDim.x >> 5;
    const int64_t tiles = (g.R + kRows - 1) / kRows;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t row0 = tile * kRows;
        for (int i = warp; i < kRows / 8; i += nw) {
            const int r = 8 * i + (lane & 7);
            const bool valid = row0 + r < g.R;
            const int64_t row = valid ? row0 + r : 0;
            const float* const rows[2] = {g.h + row * H, g.a + row * H};
            stage_rows<2>(sA, r, rows, valid);
        }
        if (!mma_tile(tmem, sA, sB, 2, &bar, phase, g.status, g.limit)) break;
        {   // h += SiLU(acc + b_n), in place: each (row, column half) belongs to one thread
            const int r = epi_row(), c0 = epi_col0();
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(r & ~31) << 16) + (uint32_t)c0, v);
            if (row0 + r < g.R) {
                float* hr = g.h + (row0 + r) * H + c0;
#pragma unroll
                for (int c = 0; c < 32; c += 4) {
                    float4 hv = *reinterpret_cast<const float4*>(hr + c);
                    hv.x = hv.x + tc::silu(v[c] + g.bias[c0 + c]);
                    hv.y = hv.y + tc::silu(v[c + 1] + g.bias[c0 + c + 1]);
                    hv.z = hv.z + tc::silu(v[c + 2] + g.bias[c0 + c + 2]);
                    hv.w = hv.w + tc::silu(v[c + 3] + g.bias[c0 + c + 3]);
                    *reinterpret_cast<float4*>(hr + c) = hv;
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();   // the new rows are visible to the block; A is restaged next
        if (g.y && threadIdx.x < kRows && row0 + threadIdx.x < g.R) {   // decoder, in the unfused order
            const float* hr = g.h + (row0 + threadIdx.x) * H;
            float acc = g.bd[0];
            for (int k = 0; k < H; ++k) acc += g.wd[k] * hr[k];
            g.y[row0 + threadIdx.x] = acc;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

constexpr size_t kEdgeSmem = 3 * kKBlock + 3 * kWBlock;   // the messages reuse the A operand
constexpr size_t kNodeSmem = 2 * kKBlock + 2 * kWBlock;
static_assert((size_t)kRows * kPad * 4 <= 3 * kKBlock, "messages fit over the edge A operand");

}  // namespace
}  // namespace fedfem

using namespace fedfem;

struct fedfem_mpnn {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t N = 0, E = 0;
    int L = 4, Bmax = 1;
    std::string err;
    std::vector<void*> allocs;
    int32_t *src = nullptr, *dst = nullptr, *in_ptr = nullptr, *out_ptr = nullptr, *out_edge = nullptr;
    float* efeat = nullptr;
    int64_t nP = 0;
    std::vector<int64_t> off;               // tensor offsets in P (order of the flat layout)
    float *P = nullptr, *G = nullptr, *Am = nullptr, *Av = nullptr;
    std::vector<bf16*> We, WeT, Wn, WnT;
    int64_t adam_t = 0;
    // workspace (Bmax)
    float *zne = nullptr, *zee = nullptr, *e0 = nullptr, *e = nullptr, *msg = nullptr, *a = nullptr, *u = nullptr;
    std::vector<float*> hL, ze, zn;         // h at the input of each layer (L + 1), pre-activations
    std::vector<bf16*> Xe, Xn;
    float *y = nullptr, *dy = nullptr, *dh = nullptr, *de = nullptr, *dz_e = nullptr, *dz_n = nullptr;
    float *dXe = nullptr, *dXn = nullptr, *dzee = nullptr, *dzne = nullptr;
    bf16 *dzb_e = nullptr, *dzb_n = nullptr, *T1 = nullptr, *T2 = nullptr;
    float *part = nullptr, *colpart = nullptr, *lossp = nullptr;
    int* status = nullptr;
    // fused inference: edge tiles (in-edges of consecutive destination nodes)
    void* edge_tiles = nullptr;
    int n_edge_tiles = 0;
    int sm_count = 0;
    long long spin_limit = 2000000000LL;
    int64_t part_floats = 0, colpart_floats = 0;
};

namespace {

enum { P_WNE = 0, P_BNE, P_WEE, P_BEE };
inline int64_t p_We(int l) { return 4 + 4 * l; }
inline int64_t p_be(int l) { return 5 + 4 * l; }
inline int64_t p_Wn(int l) { return 6 + 4 * l; }
inline int64_t p_bn(int l) { return 7 + 4 * l; }

template <typename T>
cudaError_t ma(fedfem_mpnn* m, T** p, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n * sizeof(T), 16));
    if (e == cudaSuccess) { m->allocs.push_back(q); *p = (T*)q; }
    return e;
}

int mfail(fedfem_mpnn* m, int code, const std::string& s) {
    if (m) m->err = s;
    return code;
}

#define MC(x)                                                                             \
    do {                                                                                  \
        cudaError_t _e = (x);                                                             \
        if (_e != cudaSuccess) return mfail(m, FEDFEM_E_CUDA, std::string(#x) + ": " + cudaGetErrorString(_e)); \
    } while (0)

inline int64_t pad64(int64_t n) { return (n + 63) / 64 * 64; }

int refresh_bf16(fedfem_mpnn* m) {
    for (int l = 0; l < m->L; ++l) {
        k_weights_bf16<<<grid(H * 3 * H), kT, 0, m->stream>>>(H, 3 * H, m->P + m->off[p_We(l)], m->We[l], m->WeT[l]);
        k_weights_bf16<<<grid(H * 2 * H), kT, 0, m->stream>>>(H, 2 * H, m->P + m->off[p_Wn(l)], m->Wn[l], m->WnT[l]);
    }
    MC(cudaGetLastError());
    return FEDFEM_OK;
}

int gemm(fedfem_mpnn* m, const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K, int k_chunk,
         const float* bias, int act, float* Z, int64_t ldz, float* Cf, int64_t ldc) {
    GemmArgs g{};
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.M = M; g.N = N; g.K = K; g.k_chunk = k_chunk;
    g.bias = bias; g.act = act; g.Z = Z; g.ldz = ldz; g.Cf = Cf; g.ldc = ldc; g.partial = m->part;
    g.status = m->status;
    if (k_chunk > 0 && k_chunk < K && gemm_partial_floats(M, N, K, k_chunk) > (size_t)m->part_floats)
        return mfail(m, FEDFEM_E_ARG, "split-K scratch too small");
    MC(launch_gemm_tc(g, m->stream));
    return FEDFEM_OK;
}

int colsum(fedfem_mpnn* m, int64_t R, int K, int J, const float* A, int lda, const float* X, int ldx, float* out) {
    const int chunks = (int)((R + kChunk - 1) / kChunk);
    if ((int64_t)chunks * K * J > m->colpart_floats) return mfail(m, FEDFEM_E_ARG, "column-sum scratch too small");
    dim3 g((unsigned)chunks, (unsigned)((K * J + kT - 1) / kT));
    k_colsum_part<<<g, kT, 0, m->stream>>>(R, K, J, A, lda, X, ldx, m->colpart);
    k_colsum_final<<<grid(K * J), kT, 0, m->stream>>>(chunks, K * J, m->colpart, out);
    MC(cudaGetLastError());
    return FEDFEM_OK;
}

int transpose(fedfem_mpnn* m, int64_t R, int C, const bf16* in, int64_t ldi, bf16* out) {
    const int64_t Rp = pad64(R);
    dim3 g((unsigned)((Rp + 31) / 32), (unsigned)((C + 31) / 32));
    k_transpose<<<g, dim3(32, 8), 0, m->stream>>>(R, Rp, C, in, ldi, out, Rp);
    MC(cudaGetLastError());
    return FEDFEM_OK;
}

// forward for a batch; keeps what backward needs
int forward(fedfem_mpnn* m, int B, const float* x) {
    const int64_t N = m->N, E = m->E, RN = B * N, RE = B * E;
    const float* P = m->P;
    cudaStream_t s = m->stream;
    k_encode<<<grid(RN * H), kT, 0, s>>>(RN, NIN, x, P + m->off[P_WNE], P + m->off[P_BNE], m->zne, m->hL[0]);
    k_encode<<<grid(E * H), kT, 0, s>>>(E, EIN, m->efeat, P + m->off[P_WEE], P + m->off[P_BEE], m->zee, m->e0);
    k_bcast_edges<<<grid(RE * H), kT, 0, s>>>(B, E, m->e0, m->e);
    MC(cudaGetLastError());
    for (int l = 0; l < m->L; ++l) {
        float* h = m->hL[l];
        k_build_xe<<<grid(RE * 3 * H), kT, 0, s>>>(B, E, N, m->src, m->dst, m->e, h, m->Xe[l]);
        MC(cudaGetLastError());
        if (int r = gemm(m, m->Xe[l], 3 * H, m->We[l], 3 * H, (int)RE, H, 3 * H, 0, P + m->off[p_be(l)], 1,
                         m->ze[l], H, m->msg, H))
            return r;
        k_add<<<grid(RE * H), kT, 0, s>>>(RE * H, m->e, m->msg);
        k_aggregate<<<grid(RN * H), kT, 0, s>>>(B, E, N, m->in_ptr, m->msg, m->a);
        k_build_xn<<<grid(RN * 2 * H), kT, 0, s>>>(RN, h, m->a, m->Xn[l]);
        MC(cudaGetLastError());
        if (int r = gemm(m, m->Xn[l], 2 * H, m->Wn[l], 2 * H, (int)RN, H, 2 * H, 0, P + m->off[p_bn(l)], 1,
                         m->zn[l], H, m->u, H))
            return r;
        MC(cudaMemcpyAsync(m->hL[l + 1], h, sizeof(float) * RN * H, cudaMemcpyDeviceToDevice, s));
        k_add<<<grid(RN * H), kT, 0, s>>>(RN * H, m->hL[l + 1], m->u);
    }
    k_decode<<<grid(RN), kT, 0, s>>>(RN, m->hL[m->L], P + m->off[p_We(m->L)], P + m->off[p_We(m->L) + 1], m->y);
    MC(cudaGetLastError());
    return FEDFEM_OK;
}

int backward(fedfem_mpnn* m, int B, const float* x) {
    const int64_t N = m->N, E = m->E, RN = B * N, RE = B * E;
    const int64_t REp = pad64(RE), RNp = pad64(RN);
    float* G = m->G;
    const float* P = m->P;
    cudaStream_t s = m->stream;
    const int64_t od = m->off[p_We(m->L)];           // w_d, then b_d
    if (int r = colsum(m, RN, H, 1, m->hL[m->L], H, m->dy, 1, G + od)) return r;
    if (int r = colsum(m, RN, 1, 1, m->dy, 1, nullptr, 0, G + m->off[p_We(m->L) + 1])) return r;
    k_dec_bwd<<<grid(RN * H), kT, 0, s>>>(RN, m->dy, P + od, m->dh);
    MC(cudaMemsetAsync(m->de, 0, sizeof(float) * RE * H, s));
    const int kc_n = (int)std::min<int64_t>(RNp, 4096), kc_e = (int)std::min<int64_t>(REp, 32768);
    for (int l = m->L - 1; l >= 0; --l) {
        // node update
        k_dsilu<<<grid(RN * H), kT, 0, s>>>(RN * H, m->dh, m->zn[l], m->dz_n, m->dzb_n);
        MC(cudaGetLastError());
        if (int r = colsum(m, RN, H, 1, m->dz_n, H, nullptr, 0, G + m->off[p_bn(l)])) return r;
        if (int r = transpose(m, RN, H, m->dzb_n, H, m->T1)) return r;              // 64 x RNp
        if (int r = transpose(m, RN, 2 * H, m->Xn[l], 2 * H, m->T2)) return r;      // 128 x RNp
        if (int r = gemm(m, m->T1, RNp, m->T2, RNp, H, 2 * H, (int)RNp, kc_n, nullptr, 0, nullptr, 0,
                         G + m->off[p_Wn(l)], 2 * H))
            return r;
        if (int r = gemm(m, m->dzb_n, H, m->WnT[l], H, (int)RN, 2 * H, H, 0, nullptr, 0, nullptr, 0, m->dXn, 2 * H))
            return r;
        k_node_bwd<<<grid(RN * H), kT, 0, s>>>(RN, m->dXn, m->dh);
        // edge update
        k_dmsg<<<grid(RE * H), kT, 0, s>>>(B, E, N, m->dst, m->de, m->dXn, m->ze[l], m->dz_e, m->dzb_e);
        MC(cudaGetLastError());
        if (int r = colsum(m, RE, H, 1, m->dz_e, H, nullptr, 0, G + m->off[p_be(l)])) return r;
        if (int r = transpose(m, RE, H, m->dzb_e, H, m->T1)) return r;              // 64 x REp
        if (int r = transpose(m, RE, 3 * H, m->Xe[l], 3 * H, m->T2)) return r;      // 192 x REp
        if (int r = gemm(m, m->T1, REp, m->T2, REp, H, 3 * H, (int)REp, kc_e, nullptr, 0, nullptr, 0,
                         G + m->off[p_We(l)], 3 * H))
            return r;
        if (int r = gemm(m, m->dzb_e, H, m->WeT[l], H, (int)RE, 3 * H, H, 0, nullptr, 0, nullptr, 0, m->dXe, 3 * H))
            return r;
        k_edge_bwd<<<grid(RE * H), kT, 0, s>>>(RE, m->dXe, m->de);
        k_node_scatter<<<grid(RN * H), kT, 0, s>>>(B, E, N, m->out_ptr, m->out_edge, m->in_ptr, m->dXe, m->dh);
        MC(cudaGetLastError());
    }
    k_edge_enc_bwd<<<grid(E * H), kT, 0, s>>>(B, E, m->de, m->zee, m->dzee);
    if (int r = colsum(m, E, H, EIN, m->dzee, H, m->efeat, EIN, G + m->off[P_WEE])) return r;
    if (int r = colsum(m, E, H, 1, m->dzee, H, nullptr, 0, G + m->off[P_BEE])) return r;
    k_dsilu_f32<<<grid(RN * H), kT, 0, s>>>(RN * H, m->dh, m->zne, m->dzne);
    if (int r = colsum(m, RN, H, NIN, m->dzne, H, x, NIN, G + m->off[P_WNE])) return r;
    if (int r = colsum(m, RN, H, 1, m->dzne, H, nullptr, 0, G + m->off[P_BNE])) return r;
    MC(cudaGetLastError());
    return FEDFEM_OK;
}

// fused inference forward: encoders, then per layer the edge and node kernels
int infer(fedfem_mpnn* m, int B, const float* x, float* y) {
    const int64_t N = m->N, E = m->E, RN = B * N;
    const float* P = m->P;
    cudaStream_t s = m->stream;
    float* h = m->hL[0];
    k_encode<<<grid(RN * H), kT, 0, s>>>(RN, NIN, x, P + m->off[P_WNE], P + m->off[P_BNE], m->zne, h);
    k_encode<<<grid(E * H), kT, 0, s>>>(E, EIN, m->efeat, P + m->off[P_WEE], P + m->off[P_BEE], m->zee, m->e0);
    MC(cudaGetLastError());
    MC(cudaFuncSetAttribute(k_edge_layer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEdgeSmem));
    MC(cudaFuncSetAttribute(k_node_layer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNodeSmem));
    const int64_t edge_items = (int64_t)m->n_edge_tiles * B;
    const int64_t node_tiles = (RN + kRows - 1) / kRows;
    const int resident = 3 * std::max(1, m->sm_count);
    for (int l = 0; l < m->L; ++l) {
        EdgeLayerArgs ea{};
        ea.B = B; ea.N = N; ea.E = E;
        ea.src = m->src; ea.dst = m->dst; ea.in_ptr = m->in_ptr;
        ea.tiles = (const EdgeTile*)m->edge_tiles; ea.n_tiles = m->n_edge_tiles;
        ea.e_in = l == 0 ? m->e0 : m->e;
        ea.e_in_stride = l == 0 ? 0 : E * H;
        ea.e_out = l + 1 < m->L ? m->e : nullptr;
        ea.h = h; ea.a = m->a;
        ea.W = m->We[l]; ea.bias = P + m->off[p_be(l)];
        ea.status = m->status; ea.limit = m->spin_limit;
        k_edge_layer<<<(unsigned)std::min<int64_t>(edge_items, resident), kFusedThreads, kEdgeSmem, s>>>(ea);
        MC(cudaGetLastError());
        NodeLayerArgs na{};
        na.R = RN; na.h = h; na.a = m->a;
        na.W = m->Wn[l]; na.bias = P + m->off[p_bn(l)];
        const bool last = l + 1 == m->L;
        na.wd = last ? P + m->off[p_We(m->L)] : nullptr;
        na.bd = last ? P + m->off[p_We(m->L) + 1] : nullptr;
        na.y = last ? y : nullptr;
        na.status = m->status; na.limit = m->spin_limit;
        k_node_layer<<<(unsigned)std::min<int64_t>(node_tiles, resident), kFusedThreads, kNodeSmem, s>>>(na);
        MC(cudaGetLastError());
    }
    return FEDFEM_OK;
}

}  // namespace

extern "C" {

int fedfem_mpnn_create(fedfem_mpnn** out, int device, int64_t n_nodes, int64_t n_edges, const int32_t* src,
                       const int32_t* dst, const double* xyz, double length_scale, int layers, int max_batch,
                       void* stream) {
    if (!out || n_nodes <= 0 || n_edges <= 0 || !src || !dst || !xyz || !(length_scale > 0) || layers < 1 ||
        layers > 8 || max_batch < 1)
        return FEDFEM_E_ARG;
    *out = nullptr;
    for (int64_t i = 0; i < n_edges; ++i) {
        if (src[i] < 0 || src[i] >= n_nodes || dst[i] < 0 || dst[i] >= n_nodes) return FEDFEM_E_ARG;
        if (i > 0 && (dst[i] < dst[i - 1] || (dst[i] == dst[i - 1] && src[i] <= src[i - 1]))) return FEDFEM_E_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return FEDFEM_E_CUDA;
    fedfem_mpnn* m = new fedfem_mpnn();
    m->device = device;
    m->stream = (cudaStream_t)stream;
    m->N = n_nodes; m->E = n_edges; m->L = layers; m->Bmax = max_batch;
    // parameter layout
    std::vector<int64_t> sizes = {H * NIN, H, H * EIN, H};
    for (int l = 0; l < layers; ++l) { sizes.push_back(H * 3 * H); sizes.push_back(H); sizes.push_back(H * 2 * H); sizes.push_back(H); }
    sizes.push_back(H);
    sizes.push_back(1);
    int64_t o = 0;
    for (int64_t s : sizes) { m->off.push_back(o); o += s; }
    m->nP = o;
    // graph: CSR by destination, edges out of each node
    std::vector<int32_t> in_ptr(n_nodes + 1, 0), out_ptr(n_nodes + 1, 0), out_edge(n_edges);
    for (int64_t i = 0; i < n_edges; ++i) { in_ptr[dst[i] + 1]++; out_ptr[src[i] + 1]++; }
    for (int64_t i = 0; i < n_nodes; ++i) { in_ptr[i + 1] += in_ptr[i]; out_ptr[i + 1] += out_ptr[i]; }
    {
        std::vector<int32_t> pos(out_ptr.begin(), out_ptr.end() - 1);
        for (int64_t i = 0; i < n_edges; ++i) out_edge[pos[src[i]]++] = (int32_t)i;
    }
    // edge tiles of the fused forward: whole in-edge lists of consecutive nodes, at most 128 edges
    std::vector<EdgeTile> tiles;
    for (int64_t n = 0; n < n_nodes;) {
        EdgeTile t{in_ptr[n], 0, (int32_t)n, (int32_t)n};
        while (n < n_nodes && in_ptr[n + 1] - t.m0 <= kRows) ++n;
        if (n == t.n0) {   // one node with more than 128 in-edges
            delete m;
            return FEDFEM_E_UNSUPPORTED;
        }
        t.n1 = (int32_t)n;
        t.count = in_ptr[n] - t.m0;
        tiles.push_back(t);
    }
    m->n_edge_tiles = (int)tiles.size();
    cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, device);
    const int64_t Bm = max_batch, RN = Bm * n_nodes, RE = Bm * n_edges;
    double* xyz_d = nullptr;
    auto fail_alloc = [&](cudaError_t e) {
        for (void* p : m->allocs) cudaFree(p);
        delete m;
        return e == cudaErrorMemoryAllocation ? FEDFEM_E_OOM : FEDFEM_E_CUDA;
    };
#define MA(p, n) do { cudaError_t _e = ma(m, &(p), (size_t)(n)); if (_e != cudaSuccess) return fail_alloc(_e); } while (0)
    MA(m->src, n_edges); MA(m->dst, n_edges); MA(m->in_ptr, n_nodes + 1); MA(m->out_ptr, n_nodes + 1);
    MA(m->out_edge, n_edges); MA(m->efeat, n_edges * EIN); MA(xyz_d, n_nodes * 3);
    MA(m->P, m->nP); MA(m->G, m->nP); MA(m->Am, m->nP); MA(m->Av, m->nP);
    m->We.resize(layers); m->WeT.resize(layers); m->Wn.resize(layers); m->WnT.resize(layers);
    for (int l = 0; l < layers; ++l) {
        MA(m->We[l], H * 3 * H); MA(m->WeT[l], H * 3 * H); MA(m->Wn[l], H * 2 * H); MA(m->WnT[l], H * 2 * H);
    }
    MA(m->zne, RN * H); MA(m->zee, n_edges * H); MA(m->e0, n_edges * H); MA(m->e, RE * H); MA(m->msg, RE * H);
    MA(m->a, RN * H); MA(m->u, RN * H);
    m->hL.resize(layers + 1); m->ze.resize(layers); m->zn.resize(layers); m->Xe.resize(layers); m->Xn.resize(layers);
    for (int l = 0; l <= layers; ++l) MA(m->hL[l], RN * H);
    for (int l = 0; l < layers; ++l) {
        MA(m->ze[l], RE * H); MA(m->zn[l], RN * H); MA(m->Xe[l], RE * 3 * H); MA(m->Xn[l], RN * 2 * H);
    }
    MA(m->y, RN); MA(m->dy, RN); MA(m->dh, RN * H); MA(m->de, RE * H); MA(m->dz_e, RE * H); MA(m->dz_n, RN * H);
    MA(m->dXe, RE * 3 * H); MA(m->dXn, RN * 2 * H); MA(m->dzee, n_edges * H); MA(m->dzne, RN * H);
    MA(m->dzb_e, RE * H); MA(m->dzb_n, RN * H);
    MA(m->T1, H * pad64(std::max(RE, RN))); MA(m->T2, 3 * H * pad64(std::max(RE, RN)));
    m->part_floats = (int64_t)gemm_partial_floats(H, 3 * H, (int)pad64(RE), 32768) +
                     (int64_t)gemm_partial_floats(H, 2 * H, (int)pad64(RN), 4096) + 64;
    MA(m->part, m->part_floats);
    m->colpart_floats = ((std::max(RE, RN) + kChunk - 1) / kChunk) * H * NIN + 64;
    MA(m->colpart, m->colpart_floats);
    MA(m->lossp, (RN + kT - 1) / kT + 1);
    MA(m->status, 1);
    {
        unsigned char* tp = nullptr;
        MA(tp, sizeof(EdgeTile) * tiles.size());
        m->edge_tiles = tp;
    }
#undef MA
    cudaStream_t s = m->stream;
    bool ok = cudaMemcpyAsync(m->src, src, sizeof(int32_t) * n_edges, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(m->dst, dst, sizeof(int32_t) * n_edges, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(m->in_ptr, in_ptr.data(), sizeof(int32_t) * (n_nodes + 1), cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(m->out_ptr, out_ptr.data(), sizeof(int32_t) * (n_nodes + 1), cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(m->out_edge, out_edge.data(), sizeof(int32_t) * n_edges, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(xyz_d, xyz, sizeof(double) * 3 * n_nodes, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaMemcpyAsync(m->edge_tiles, tiles.data(), sizeof(EdgeTile) * tiles.size(), cudaMemcpyHostToDevice,
                              s) == cudaSuccess &&
              cudaMemsetAsync(m->P, 0, sizeof(float) * m->nP, s) == cudaSuccess &&
              cudaMemsetAsync(m->status, 0, sizeof(int), s) == cudaSuccess;
    if (ok) {
        k_edge_features<<<grid(n_edges), kT, 0, s>>>(n_edges, m->src, m->dst, xyz_d, 1.0 / length_scale, m->efeat);
        ok = cudaStreamSynchronize(s) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    }
    if (!ok) return fail_alloc(cudaErrorUnknown);
    *out = m;
    return FEDFEM_OK;
}

void fedfem_mpnn_destroy(fedfem_mpnn* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (void* p : m->allocs) cudaFree(p);
    delete m;
}

int64_t fedfem_mpnn_n_params(const fedfem_mpnn* m) { return m ? m->nP : 0; }

const char* fedfem_mpnn_last_error(const fedfem_mpnn* m) { return m ? m->err.c_str() : "null"; }

int fedfem_mpnn_set_params(fedfem_mpnn* m, const float* host) {
    if (!m || !host) return FEDFEM_E_ARG;
    MC(cudaSetDevice(m->device));
    MC(cudaMemcpyAsync(m->P, host, sizeof(float) * m->nP, cudaMemcpyHostToDevice, m->stream));
    MC(cudaMemsetAsync(m->Am, 0, sizeof(float) * m->nP, m->stream));
    MC(cudaMemsetAsync(m->Av, 0, sizeof(float) * m->nP, m->stream));
    m->adam_t = 0;
    if (int r = refresh_bf16(m)) return r;
    MC(cudaStreamSynchronize(m->stream));
    return FEDFEM_OK;
}

int fedfem_mpnn_get_params(fedfem_mpnn* m, float* host) {
    if (!m || !host) return FEDFEM_E_ARG;
    MC(cudaSetDevice(m->device));
    MC(cudaMemcpyAsync(host, m->P, sizeof(float) * m->nP, cudaMemcpyDeviceToHost, m->stream));
    MC(cudaStreamSynchronize(m->stream));
    return FEDFEM_OK;
}

int fedfem_mpnn_features(fedfem_mpnn* m, int batch, const float* T_dev, const float* q_dev,
                         const unsigned char* dirichlet_dev, const fedfem_material* mat, float* x_dev) {
    if (!m || !T_dev || !q_dev || !mat || !x_dev || batch < 1) return FEDFEM_E_ARG;
    MC(cudaSetDevice(m->device));
    k_features<<<grid((int64_t)batch * m->N), kT, 0, m->stream>>>(batch, m->N, T_dev, q_dev, dirichlet_dev, *mat,
                                                                   x_dev);
    MC(cudaGetLastError());
    return FEDFEM_OK;
}

int fedfem_mpnn_forward(fedfem_mpnn* m, int batch, const float* x_dev, float* y_dev) {
    if (!m || !x_dev || !y_dev || batch < 1 || batch > m->Bmax) return mfail(m, FEDFEM_E_ARG, "bad batch or pointer");
    MC(cudaSetDevice(m->device));
    if (int r = forward(m, batch, x_dev)) return r;
    MC(cudaMemcpyAsync(y_dev, m->y, sizeof(float) * batch * m->N, cudaMemcpyDeviceToDevice, m->stream));
    return FEDFEM_OK;
}

int fedfem_mpnn_infer(fedfem_mpnn* m, int batch, const float* x_dev, float* y_dev) {
    if (!m || !x_dev || !y_dev || batch < 1 || batch > m->Bmax) return mfail(m, FEDFEM_E_ARG, "bad batch or pointer");
    MC(cudaSetDevice(m->device));
    return infer(m, batch, x_dev, y_dev);
}

int fedfem_mpnn_sync(fedfem_mpnn* m) {
    if (!m) return FEDFEM_E_ARG;
    MC(cudaSetDevice(m->device));
    int st = 0;
    MC(cudaMemcpyAsync(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    MC(cudaStreamSynchronize(m->stream));
    if (st) return mfail(m, FEDFEM_E_TIMEOUT, "a tensor-core wait gave up");
    return FEDFEM_OK;
}

int fedfem_mpnn_loss_grad(fedfem_mpnn* m, int batch, const float* x_dev, const float* target_dev,
                          const float* mask_dev, float* loss_host, float* grad_host) {
    if (!m || !x_dev || !target_dev || !mask_dev || batch < 1 || batch > m->Bmax)
        return mfail(m, FEDFEM_E_ARG, "bad batch or pointer");
    MC(cudaSetDevice(m->device));
    if (int r = forward(m, batch, x_dev)) return r;
    std::vector<float> mask(m->N);
    MC(cudaMemcpyAsync(mask.data(), mask_dev, sizeof(float) * m->N, cudaMemcpyDeviceToHost, m->stream));
    MC(cudaStreamSynchronize(m->stream));
    double cnt = 0;
    for (float v : mask) cnt += v;
    cnt *= batch;
    if (cnt <= 0) return mfail(m, FEDFEM_E_ARG, "empty mask");
    const int64_t RN = (int64_t)batch * m->N;
    const int nb = (int)grid(RN);
    k_loss<<<nb, kT, 0, m->stream>>>(batch, m->N, m->y, target_dev, mask_dev, (float)(1.0 / cnt), m->dy, m->lossp);
    MC(cudaGetLastError());
    if (int r = backward(m, batch, x_dev)) return r;
    std::vector<float> lp(nb);
    MC(cudaMemcpyAsync(lp.data(), m->lossp, sizeof(float) * nb, cudaMemcpyDeviceToHost, m->stream));
    if (grad_host) MC(cudaMemcpyAsync(grad_host, m->G, sizeof(float) * m->nP, cudaMemcpyDeviceToHost, m->stream));
    int st = 0;
    MC(cudaMemcpyAsync(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    MC(cudaStreamSynchronize(m->stream));
    if (st) return mfail(m, FEDFEM_E_TIMEOUT, "a tensor-core wait gave up");
    double s = 0;
    for (float v : lp) s += v;
    if (loss_host) *loss_host = (float)(s / cnt);
    return FEDFEM_OK;
}

int fedfem_mpnn_adam(fedfem_mpnn* m, float lr) {
    if (!m || !(lr > 0)) return FEDFEM_E_ARG;
    MC(cudaSetDevice(m->device));
    m->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)m->adam_t), c2 = 1.0f - powf(b2, (float)m->adam_t);
    k_adam<<<grid(m->nP), kT, 0, m->stream>>>(m->nP, m->P, m->G, m->Am, m->Av, lr, b1, b2, 1e-8f, c1, c2);
    MC(cudaGetLastError());
    return refresh_bf16(m);
}

}  // extern "C"
