// Internal declarations of the FED-FEM library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "fedfem.h"

namespace fedfem {

// ---------------------------------------------------------------------------
// Host-side mesh layout (built once, cold path; host_layout.cpp)
// ---------------------------------------------------------------------------
struct Layout {
    int nv = 0;                      // nodes per element (4 or 8)
    int64_t N = 0, E = 0;
    int64_t N_plain = 0;             // [0, N_plain): free nodes without a film condition
    int64_t N_free = 0;              // [N_plain, N_free): free nodes with a film condition
                                     // [N_free, N): Dirichlet nodes
    std::vector<int32_t> elem_of;    // internal element -> input element
    std::vector<int32_t> node_of;    // internal node -> input node
    std::vector<int32_t> node_at;    // input node -> internal node
    std::vector<int32_t> conn;       // internal connectivity, E x nv, internal node ids
    // Node -> element-slot gather over the free nodes, sliced ELL with slices of
    // 32 consecutive nodes: entry k of node i sits at sell_ids[sell_off[i/32] + 32k + i%32].
    // Each node's list is sorted by INPUT element id; pads point at the zero slot E*nv.
    std::vector<int32_t> sell_off;   // n_slices + 1
    std::vector<int32_t> sell_ids;
    int max_degree = 0;
    // convective nodes [N_plain, N_free): CSR over face ids (input face order)
    std::vector<int32_t> conv_off;   // (N_free - N_plain) + 1
    std::vector<int32_t> conv_face;
};

// Tiles of the tiled time loop: tile t owns free nodes [t*B, min((t+1)*B, N_free))
// and holds every element touching one of them (elements on a tile edge are
// computed by each tile that touches them).  Local node ids: owned nodes
// first (l = i - t*B), then the halo nodes in global order.  Each 16-bit
// local connectivity entry is  local id | rank << rank_shift : for an owned
// corner, rank is the element's position in that node's slot list (input
// element order), i.e. where its load goes in the node's fixed-order sum.
struct Tiles {
    int B = 0, nv = 0;                     // owned nodes per tile, corners
    int64_t n_tiles = 0;
    std::vector<int32_t> e_off;            // n_tiles + 1, into the tile-element arrays
    std::vector<int32_t> e_glob;           // internal element id of each tile element
    std::vector<uint16_t> lconn;           // nv entries per tile element (id | rank << rank_shift)
    std::vector<int32_t> h_off;            // n_tiles + 1
    std::vector<int32_t> halo;             // global node ids
    std::vector<int32_t> deg;              // n_tiles: most elements at one owned node
    int rank_shift = 16;
    int max_local = 0, max_elems = 0, max_deg = 0;
};

std::string build_tiles(const Layout& L, int B, Tiles& out);

struct MeshInput {
    int nv = 0;
    int64_t N = 0, E = 0;
    const double* xyz = nullptr;
    const int32_t* conn = nullptr;
    const std::vector<char>* is_dirichlet = nullptr;   // input node flags
    const std::vector<int32_t>* conv_faces = nullptr;  // n_faces x conv_nverts
    int conv_nverts = 0;
    int order = FEDFEM_ORDER_MORTON;
    const std::vector<int32_t>* groups = nullptr;      // element groups kept apart in the internal order
};

// Returns "" on success, else an error message.  Sets *mesh_error when the
// failure is a mesh defect.
std::string build_layout(const MeshInput& in, Layout& out, bool* mesh_error);

// ---------------------------------------------------------------------------
// Device status word shared by all time-loop kernels
// ---------------------------------------------------------------------------
enum : int { STATUS_RANGE = 1, STATUS_TIMEOUT = 2 };

struct DevStatus {
    int flags;
    int skip_barrier_block;          // testing hook: this block never arrives (-1 = none)
    long long fail_node;             // internal node of the first range failure
    long long fail_step;             // step index (since init) of the first failure
    unsigned long long barrier;      // monotone arrival counter of the grid barrier
    long long steps_done;            // steps completed since init
    unsigned long long bad_input;    // nonzero: the last checked initial field held a non-finite value
    long long pad;
};

// ---------------------------------------------------------------------------
// Kernel parameter block of the time loop
// ---------------------------------------------------------------------------
// R: type of the element matrices and node constants; L: type of one node's
// temperature state -- R itself, or F4 for four scenario lanes.
constexpr int kMaxSegments = 8;   // pieces of a source schedule
constexpr int kMaxTable = 8;      // points of a piecewise-linear property table
constexpr int kMaxRegions = 16;   // tissue regions of a heterogeneous mesh

template <typename R, typename L = R>
struct StepArgs {
    int64_t E, N, N_plain, N_free;
    const int4* conn4;               // nv/4 planes of E int4
    const R* M;                      // 6 planes of E: m00 m11 m22 m01 m02 m12
    R* slots;                        // E*nv + 1 element loads (the last one stays 0)
    const int32_t* sell_off;
    const int32_t* sell_ids;
    const R* V;                      // lumped volume, free nodes
    const L* Q;                      // constant nodal heat flow (W), free nodes (per lane)
    const R* hA;                     // film h * lumped area, nodes [N_plain, N_free)
    L* T;                            // temperature (FP64) or its hi part (FP32), all N nodes
    L* T2;                           // second buffer of the tiled kernel (same layout as T)
    L* Tlo;                          // FP32 compensation, all N nodes (unused in FP64)
    R T_ref, rho0, drho, c0, dc, k0, dk;
    R wbcb, T_a, T_inf;
    R dt, T_lo, T_hi;
    DevStatus* status;
    long long step0;                 // step index (since init) of the first step of this call
    // time-varying regional sources: Q(t) = Q + f(t) Qs with Q the constant part;
    // f(t) = seg_f[k] for the first k with t < seg_end[k] (the last one after the
    // last end), t the step's start time t0 + (step - step0) dt.  Qs null: Q is total.
    const L* Qs;
    double t0, dtd;
    int n_seg;
    double seg_end[kMaxSegments];
    R seg_f[kMaxSegments];
    // thermal dose, dose[i * lanes + l] += dose_dt * rate(T_il): CEM43 minutes
    // (dose_model 0, dose_dt = dt / 60) or the Arrhenius damage integral
    // (dose_model 1, dose_dt = dt, rate = exp(dose_lnA - dose_EaR / T_K)).
    // FP64 state sums in the double; FP32 state keeps each 8-byte slot as a
    // compensated FP32 pair (hi, lo), the dose being hi + lo.
    double* dose;
    double dose_dt;
    float dose_dt32;                 // dose_dt rounded to FP32 (FP32 state)
    int dose_model;
    double dose_lnA, dose_EaR;
    float dose_c43, dose_a2, dose_g2;   // FP32 state: the rate as 2^(c43 s (T - 43) + a2 - g2 / T_K)
    // piecewise-linear laws (n_tab > 0): property P (0 rho, 1 c, 2 k) is
    // linear on each interval between the points tab_T (the end intervals
    // extended beyond the table), written by its kinks:
    //   p(T) = tab_p0[P] + tab_s0[P] (T - T_0) + sum_q tab_d[P][q] max(T - T_q, 0)
    // over the interior points q = 1 .. n_tab - 2, tab_d the change of slope
    // at T_q.  All launch arguments, so that an evaluation reads no memory.
    int n_tab;
    R tab_T[kMaxTable];
    R tab_p0[3], tab_s0[3];
    R tab_d[3][kMaxTable];
    // heterogeneous tissue (emat non-null): each element's region, in internal
    // element order (emat) and in tile-element order (emat_tile, tile t's
    // elements from emat_off[t]); each region's k law (T_ref, k0, dk) in
    // mat_k; per free node i the capacity C_i(T) = Ca + u (Cb + u Cc),
    // u = T - T_ref, and the perfusion beta_i, in Cq = [Ca | Cb | Cc | beta]
    // (planes of N_free)
    const unsigned char* emat;
    const unsigned char* emat_tile;
    const int32_t* emat_off;
    const R* mat_k;
    const R* Cq;
    // fully integrated hex8 (element-parallel kernels only): the 28 entries
    // A_ab, a < b, of each element matrix as planes of E (pair order a-major);
    // the diagonal is implied by the zero row sums.  Null: the factored M.
    const R* A28;
    // hourglass-stabilised one-point hex8: the 12 weights w_ad of each element
    // (planes of E, a-major) and eps / 4; null: no stabilisation.  The tiled
    // kernels read the weights from their tile blocks instead.
    const R* W12;
    R hg_eps4;
};

// Launchers (step.cu).  mode: FEDFEM_FP64 / FEDFEM_FP32_KAHAN / FEDFEM_FP32_PLAIN.
struct LaunchCfg {
    int kernel = FEDFEM_KERNEL_PERSISTENT;
    int block = 256;
    int blocks_per_sm = 0;
    int sm_count = 0;
    long long spin_limit = 4000000000LL;   // clock64 ticks a barrier waits before giving up
    int grid_used = 0;                     // out: grid of the last persistent launch
};

// Packed per-tile blocks of the tiled kernels, each 16-byte aligned (copied
// whole into shared memory by one bulk (TMA) copy in the staged kernel):
//   int32 header {ne, ne_pad, nh, deg}; M: ne_pad x 6 R (one element's six values together);
//   with hourglass stabilisation: ne_pad x 12 R hourglass weights;
//   matrix-free (tet4, FP32): instead of the matrices, room for (B + nh) float4 local node
//   coordinates indexed by local id (owned, then halo; x, y, z relative to the centre of the mesh's
//   bounding box, the same for every tile);
//   local connectivity: ne_pad x nv uint16 (id | rank << rank_shift);
//   halo ids: nh int32.
template <typename R>
struct TileArgs {
    int64_t n_tiles;
    int B, nv;
    int rank_shift;                  // lconn entry = local id | rank << rank_shift
    int max_deg;                     // rows of the per-node load table
    const unsigned char* blocks;
    const int64_t* block_off;        // n_tiles + 1 byte offsets
    int max_block;                   // bytes, multiple of 16
    int max_local;                   // R words of staged temperatures
    int staged;                      // 1: blocks bulk-copied into shared-memory stages; 0: read from global
    int threads;                     // staged kernel: threads per block (256 or 512)
    size_t smem_bytes;
    // replicated-row kernel (rep = 1): codes are byte offsets into rows of stride `threads`
    // (owned corner: rank * threads + l; halo node h: rep_rows * threads + h)
    int rep;
    int rep_rows;                    // rows of the temperature copies and of the load table (largest rank count)
    int max_halo;                    // largest halo of any tile
    int hourglass;                   // 1: each element's 12 hourglass weights follow its 6 matrix values in the block
    int mf;                          // 1: matrix-free tet4 blocks: local coordinates instead of element matrices
};

struct F4;
cudaError_t launch_tiled_f64(const StepArgs<double>& a, const TileArgs<double>& t, int64_t n_steps,
                             LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_tiled_f32(const StepArgs<float>& a, const TileArgs<float>& t, bool kahan, int64_t n_steps,
                             LaunchCfg& cfg, cudaStream_t s);
cudaError_t launch_tiled_f32x4(const StepArgs<float, F4>& a, const TileArgs<float>& t, bool kahan, int64_t n_steps,
                               LaunchCfg& cfg, cudaStream_t s);
// occupancy (blocks per SM) of the tiled kernel for a shared-memory size (lanes: 1 or 4)
int tiled_blocks_per_sm(int precision, int nv, int staged, int threads, int lanes, size_t smem_bytes);
int tiled_threads();   // default threads per block of the staged kernel

cudaError_t launch_steps_f64(const StepArgs<double>& a, int nv, int64_t n_steps, LaunchCfg& cfg,
                             cudaStream_t s);
cudaError_t launch_steps_f32(const StepArgs<float>& a, int nv, bool kahan, int64_t n_steps,
                             LaunchCfg& cfg, cudaStream_t s);

// ---------------------------------------------------------------------------
// BF16 tensor-core GEMM (gemm_tc.cu): C = A B^T (+ bias, SiLU)
// ---------------------------------------------------------------------------
struct GemmArgs {
    const void* A; int64_t lda;      // bf16 M x K, row-major
    const void* B; int64_t ldb;      // bf16 N x K, row-major
    int M, N, K;
    int k_chunk;                     // split-K chunk (multiple of 64; K = no split)
    const float* bias;               // N or null
    int act;                         // 0: none, 1: SiLU
    float* Z; int64_t ldz;           // pre-activation out (fp32) or null
    float* Cf; int64_t ldc;          // activation out fp32 or null
    void* Cb;                        // activation out bf16 (leading dimension ldc) or null
    float* partial;                  // splits x M x N scratch when split
    int* status;                     // bit 0: an mbarrier wait gave up
};
cudaError_t launch_gemm_tc(GemmArgs g, cudaStream_t s);
size_t gemm_partial_floats(int M, int N, int K, int k_chunk);

// ---------------------------------------------------------------------------
// Pre-computation (precompute.cu), FP64
// ---------------------------------------------------------------------------
struct PreArgs {
    int nv;
    int64_t E, N, N_plain, N_free;
    const int4* conn4;
    const double* x; const double* y; const double* z;      // internal node order
    double* M64;                 // 6 planes of E
    double* A28;                 // fully integrated hex8: 28 planes of E (pairs a < b of A_e), else null
    double* W64;                 // hourglass-stabilised hex8: 12 planes of E (weights w_ad), else null
    double hg_eps4;              // its strength / 4
    double* Vshare;              // E + 1 (last = 0): V_e / nv
    int* bad_elem;               // smallest internal element with det <= 0 (init INT_MAX)
    const int32_t* sell_off; const int32_t* sell_ids;
    double* V;                   // free nodes
    double* Q;                   // n_lanes x free nodes
    double* hA;                  // convective nodes
    const double* qr_node;       // n_lanes x free nodes, W/m^3 (nullable)
    const double* flux_node;     // free nodes, W (nullable)
    const double* src;           // n_src x 7: x0 y0 z0 sigma peak lane group (-1: every lane / group)
    int n_src;
    int n_lanes;
    const int32_t* node_group;   // free nodes: element group of the node (nullable)
    double Q_m;
    // film faces
    int64_t n_faces; int face_nv;
    const int32_t* faces;        // internal node ids, n_faces x face_nv
    double* face_share;          // n_faces: h * area / face_nv
    const int32_t* conv_off; const int32_t* conv_face;
    double h_film;
};

cudaError_t launch_geometry(const PreArgs& a, cudaStream_t s);
// fully integrated hex8: A28 and the exact V_e (2 x 2 x 2 Gauss points); run after launch_geometry
cudaError_t launch_geometry_full(const PreArgs& a, cudaStream_t s);
cudaError_t launch_nodal(const PreArgs& a, cudaStream_t s);
// heterogeneous tissue: per-node capacity coefficients and perfusion (Cq, 4
// planes of N_free) and the metabolic heat added to a.Q; coef: 5 per region
cudaError_t launch_regions(const PreArgs& a, const unsigned char* emat, const double* coef, double* Cq,
                           cudaStream_t s);
cudaError_t launch_to_f32(const double* src, float* dst, int64_t n, cudaStream_t s);

// Largest eigenvalue of C0^-1/2 (K0 + diag(beta + hA)) C0^-1/2 on the free
// nodes by Lanczos (FP64); beta = wbcb V, or the given per-node beta (free
// nodes) when not null.  Returns an error message or "".
struct LanczosResult { double lambda = 0; int iterations = 0; };
std::string lanczos_lambda_max(const PreArgs& a, double k0, double rho0c0, double wbcb, const double* beta,
                               int max_iter, double rel_tol, LanczosResult& out, cudaStream_t s);

// Init / output helpers (precompute.cu)
// T_in: input order, n_lanes x N; T / Tlo interleaved by lane
cudaError_t launch_init_state(int precision, int n_lanes, int64_t N, int64_t N_free, const int32_t* node_of,
                              const double* T_in, const double* T_dir, void* T, float* Tlo,
                              cudaStream_t s);
cudaError_t launch_read_state(int precision, int n_lanes, int lane, int64_t N, const int32_t* node_of,
                              const void* T, const float* Tlo, double* out, cudaStream_t s);
// lane-major [lane][n] doubles -> interleaved floats [n][lane]
cudaError_t launch_pack_lanes(const double* src, float* dst, int n_lanes, int64_t n, cudaStream_t s);

}  // namespace fedfem
