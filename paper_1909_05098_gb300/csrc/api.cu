// C ABI of the FED-FEM library: context, input validation, device memory and
// the order of Algorithm 1 (pre-computation, initialisation, time loop).
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fedfem_internal.h"

using namespace fedfem;

struct fedfem_ctx {
    int device = 0;
    int precision = FEDFEM_FP32_KAHAN;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    // ---- inputs (copies) ----
    bool has_mesh = false, has_mat = false;
    int nv = 0;
    int64_t N = 0, E = 0;
    std::vector<double> xyz;
    std::vector<int32_t> conn;
    int order = FEDFEM_ORDER_MORTON;
    fedfem_material mat{};
    fedfem_perfusion perf{0.0, 0.0, 37.0, 0.0};
    std::vector<double> qr;                       // empty: none (applies to every lane)
    std::vector<double> qr_lane[4];               // lane-specific densities (empty: none)
    std::vector<std::array<double, 7>> sources;   // x0 y0 z0 sigma peak lane group (-1: every lane / group)
    int n_lanes = 1;
    std::vector<int32_t> groups;                  // element groups (empty: one group)
    cudaGraphExec_t graph = nullptr;
    int64_t graph_steps = 0;
    double graph_dt = 0.0;
    std::vector<char> is_dir;
    std::vector<double> dir_T;
    std::vector<int32_t> conv_faces;
    int conv_nv = 0;
    double conv_h = 0.0, conv_Tinf = 0.0;
    std::vector<double> flux;                     // empty: none
    std::vector<double> sched_end, sched_f;       // source schedule (empty: sources always on)
    bool dose_on = false;
    int dose_model = FEDFEM_DOSE_CEM43;
    int hex_rule = FEDFEM_HEX_ONE_POINT;
    double hg_eps = 0.0;                          // hourglass stabilisation of the one-point hex (0: off)
    int matrix_free = 0;                          // tet4 FP32: element matrices recomputed in the tiled kernels
    double dose_A = 0.0, dose_Ea = 0.0;           // Arrhenius frequency factor (1/s), activation energy (J/mol)
    int n_reg = 0;                                // heterogeneous tissue regions (0: mat everywhere)
    int lumping = FEDFEM_LUMP_ELEMENT;            // perfusion / metabolic heat per node
    int n_cq = 0;                                 // regions of the per-node coefficient path (pre-computed)
    std::vector<fedfem_material> reg_mat;
    std::vector<fedfem_perfusion> reg_perf;       // w_b, c_b, Q_m per region (T_a from perf)
    std::vector<int32_t> region;                  // per input element
    std::vector<unsigned char> emat_host;         // per internal element (set by precompute)
    int tab_n = 0;                                // piecewise-linear laws (0: linear laws of mat)
    double tab_T[kMaxTable] = {}, tab_p[3][kMaxTable] = {};   // points; P: 0 rho, 1 c, 2 k
    fedfem_tile tile{FEDFEM_KERNEL_PERSISTENT, 256, 0, 0};
    // ---- pre-computed ----
    bool pre = false, inited = false;
    Layout L;
    double T_lo = 0, T_hi = 0, dt_cr = 0, lambda = 0, td_scale = 1;
    int lz_iters = 0;
    // ---- device ----
    std::vector<void*> allocs;
    int64_t dev_bytes = 0;
    int4* conn4 = nullptr;
    double* M64 = nullptr;
    float* M32 = nullptr;
    int32_t *sell_off = nullptr, *sell_ids = nullptr;
    double *V64 = nullptr, *Q64 = nullptr, *hA64 = nullptr, *Qs64 = nullptr;
    float *V32 = nullptr, *Q32 = nullptr, *hA32 = nullptr, *Qs32 = nullptr;
    unsigned char* emat = nullptr;             // regions: per internal element
    double* A28_64 = nullptr;                  // fully integrated hex8: 28 planes of E
    float* A28_32 = nullptr;
    double* W64 = nullptr;                     // hourglass-stabilised hex8: 12 planes of E
    float* W32 = nullptr;
    double *Cq64 = nullptr, *matk64 = nullptr;   // regions: node coefficients (4 x N_free), k laws (3 each)
    float *Cq32 = nullptr, *matk32 = nullptr;
    double* dose = nullptr;                       // CEM43 minutes per free node
    void* T = nullptr;
    void* T2 = nullptr;
    float* Tlo = nullptr;
    // ---- tiled kernel (built on first use) ----
    bool tiles_ok = false;
    int tiles_B = 0;
    Tiles tiles_host;          // host copy kept for the traffic model
    std::vector<void*> tile_allocs;
    unsigned char* t_blocks = nullptr;
    int64_t* t_block_off = nullptr;
    unsigned char* t_emat = nullptr;   // regions of the tile elements
    int32_t* t_emat_off = nullptr;
    int64_t t_block_bytes = 0;
    int t_max_block = 0, t_max_local = 0, t_max_halo = 0;
    size_t t_smem = 0;
    void* slots = nullptr;
    int32_t* node_of = nullptr;
    double* T_dir = nullptr;
    double* io = nullptr;
    DevStatus* st = nullptr;
    int sm_count = 0;
    long long spin_limit = 4000000000LL;
    int skip_block = -1;
    int64_t steps_issued = 0;
    double sim_time = 0.0;
    LaunchCfg last{};
};

namespace {

constexpr double kGasConstant = 8.314462618;   // J/(mol K), CODATA 2018

int fail(fedfem_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_fail(fedfem_ctx* c, cudaError_t e, const char* what) {
    cudaGetLastError();   // a failed call must not surface again in a later, unrelated check
    return fail(c, e == cudaErrorMemoryAllocation ? FEDFEM_E_OOM : FEDFEM_E_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CU(call, what)                                   \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return cuda_fail(c, _e, what); \
    } while (0)

void free_tiles(fedfem_ctx* c) {
    for (void* p : c->tile_allocs) cudaFree(p);
    c->tile_allocs.clear();
    c->t_emat = nullptr;
    c->t_emat_off = nullptr;
    c->tiles_ok = false;
    c->tiles_B = 0;
    c->tiles_host = Tiles();
}

void free_graph(fedfem_ctx* c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    c->graph_steps = 0;
}

void free_device(fedfem_ctx* c) {
    free_graph(c);
    free_tiles(c);
    for (void* p : c->allocs) cudaFree(p);
    c->allocs.clear();
    c->dev_bytes = 0;
    c->conn4 = nullptr; c->M64 = nullptr; c->M32 = nullptr; c->sell_off = c->sell_ids = nullptr;
    c->V64 = c->Q64 = c->hA64 = c->Qs64 = nullptr; c->V32 = c->Q32 = c->hA32 = c->Qs32 = nullptr;
    c->emat = nullptr; c->Cq64 = c->matk64 = nullptr; c->Cq32 = c->matk32 = nullptr;
    c->A28_64 = nullptr; c->A28_32 = nullptr;
    c->W64 = nullptr; c->W32 = nullptr;
    c->dose = nullptr;
    c->T = nullptr; c->T2 = nullptr; c->Tlo = nullptr; c->slots = nullptr; c->node_of = nullptr; c->T_dir = nullptr;
    c->io = nullptr; c->st = nullptr;
    c->pre = false;
    c->inited = false;
}

template <typename P>
cudaError_t dalloc(fedfem_ctx* c, P** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return e;
    c->allocs.push_back(q);
    c->dev_bytes += (int64_t)bytes;
    *p = (P*)q;
    return cudaSuccess;
}

void release(fedfem_ctx* c, void* p, size_t bytes) {
    if (!p) return;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it != c->allocs.end()) { cudaFree(p); c->allocs.erase(it); c->dev_bytes -= (int64_t)bytes; }
}

void invalidate(fedfem_ctx* c) {
    free_graph(c);
    c->pre = false;
    c->inited = false;
}

bool is_finite(double v) { return std::isfinite(v); }

// slope of property P on table interval j
double tab_slope(const fedfem_ctx* c, int P, int j) {
    return (c->tab_p[P][j + 1] - c->tab_p[P][j]) / (c->tab_T[j + 1] - c->tab_T[j]);
}

// property P of the table at T (the interval that holds T, the end ones outside)
double tab_eval(const fedfem_ctx* c, int P, double T) {
    int j = 0;
    while (j + 1 < c->tab_n - 1 && T >= c->tab_T[j + 1]) ++j;
    return c->tab_p[P][j] + tab_slope(c, P, j) * (T - c->tab_T[j]);
}

// property_scale for tables: k is largest at an end point or a table point;
// rho c is a quadratic on every interval, smallest at an end point, a table
// point or the vertex of an interval's quadratic inside it.
int property_scale_table(fedfem_ctx* c, double lo, double hi, double* s_out) {
    std::vector<double> pts{lo, hi};
    for (int j = 0; j < c->tab_n; ++j)
        if (lo < c->tab_T[j] && c->tab_T[j] < hi) pts.push_back(c->tab_T[j]);
    double kmax = -INFINITY, kmin = INFINITY;
    for (double T : pts) {
        kmax = std::max(kmax, tab_eval(c, 2, T));
        kmin = std::min(kmin, tab_eval(c, 2, T));
    }
    std::vector<double> cand = pts;
    for (int j = 0; j + 1 < c->tab_n; ++j) {
        const double sr = tab_slope(c, 0, j), sc = tab_slope(c, 1, j);
        if (sr * sc == 0.0) continue;
        const double tv = c->tab_T[j] - (c->tab_p[0][j] * sc + c->tab_p[1][j] * sr) / (2.0 * sr * sc);
        const double a = j == 0 ? -INFINITY : c->tab_T[j];
        const double b = j + 2 == c->tab_n ? INFINITY : c->tab_T[j + 1];
        if (std::max(a, lo) < tv && tv < std::min(b, hi)) cand.push_back(tv);
    }
    double rc_min = INFINITY;
    for (double T : cand) rc_min = std::min(rc_min, tab_eval(c, 0, T) * tab_eval(c, 1, T));
    if (!(rc_min > 0) || !(kmin > 0)) return fail(c, FEDFEM_E_RANGE, "rho(T) c(T) or k(T) is not positive on [T_lo, T_hi]");
    const double rc0 = c->tab_p[0][0] * c->tab_p[1][0];
    *s_out = std::max(1.0, kmax / c->tab_p[2][0]) * std::max(1.0, rc0 / rc_min);
    return FEDFEM_OK;
}

// s = max(1, max k/k0) * max(1, max rho0 c0 / (rho c)) over [lo, hi]; rho c is
// quadratic in T, so its minimum is at an end point or the vertex.
int property_scale(fedfem_ctx* c, double lo, double hi, double* s_out);

// property_scale for regions, against the first region's reference state:
// the largest k of any region over [lo, hi] and the smallest rho c of any
// region (each a linear law: k at an end point, rho c at an end point or its
// vertex).  Every C_i is a positive combination of the regions' rho c and
// every k_e a region's k, so the bound of the homogeneous case carries over.
int property_scale_regions(fedfem_ctx* c, double lo, double hi, double* s_out) {
    const fedfem_material ref = c->reg_mat[0];
    double kmax = -INFINITY, rc_min = INFINITY;
    for (const fedfem_material& m : c->reg_mat) {
        auto k = [&](double T) { return m.k0 + m.dk * (T - m.T_ref); };
        auto rc = [&](double T) { return (m.rho0 + m.drho * (T - m.T_ref)) * (m.c0 + m.dc * (T - m.T_ref)); };
        if (!(k(lo) > 0 && k(hi) > 0)) return fail(c, FEDFEM_E_RANGE, "a region's k(T) is not positive on [T_lo, T_hi]");
        kmax = std::max(kmax, std::max(k(lo), k(hi)));
        rc_min = std::min(rc_min, std::min(rc(lo), rc(hi)));
        const double qa = m.drho * m.dc;
        if (qa != 0.0) {
            const double u = -(m.rho0 * m.dc + m.c0 * m.drho) / (2.0 * qa);
            if (lo < m.T_ref + u && m.T_ref + u < hi) rc_min = std::min(rc_min, rc(m.T_ref + u));
        }
    }
    if (!(rc_min > 0)) return fail(c, FEDFEM_E_RANGE, "a region's rho(T) c(T) is not positive on [T_lo, T_hi]");
    *s_out = std::max(1.0, kmax / ref.k0) * std::max(1.0, ref.rho0 * ref.c0 / rc_min);
    return FEDFEM_OK;
}

int property_scale(fedfem_ctx* c, double lo, double hi, double* s_out) {
    if (c->tab_n > 0) return property_scale_table(c, lo, hi, s_out);
    if (c->n_reg > 0) return property_scale_regions(c, lo, hi, s_out);
    const fedfem_material& m = c->mat;
    auto k = [&](double T) { return m.k0 + m.dk * (T - m.T_ref); };
    auto rc = [&](double T) { return (m.rho0 + m.drho * (T - m.T_ref)) * (m.c0 + m.dc * (T - m.T_ref)); };
    if (!(k(lo) > 0 && k(hi) > 0)) return fail(c, FEDFEM_E_RANGE, "k(T) is not positive on [T_lo, T_hi]");
    double rc_min = std::min(rc(lo), rc(hi));
    const double qa = m.drho * m.dc;
    if (qa != 0.0) {
        const double u = -(m.rho0 * m.dc + m.c0 * m.drho) / (2.0 * qa);
        if (lo < m.T_ref + u && m.T_ref + u < hi) rc_min = std::min(rc_min, rc(m.T_ref + u));
    }
    if (!(rc_min > 0)) return fail(c, FEDFEM_E_RANGE, "rho(T) c(T) is not positive on [T_lo, T_hi]");
    const double kmax = std::max(k(lo), k(hi));
    *s_out = std::max(1.0, kmax / m.k0) * std::max(1.0, m.rho0 * m.c0 / rc_min);
    return FEDFEM_OK;
}

int reset_status(fedfem_ctx* c) {
    DevStatus h{};
    h.flags = 0;
    h.skip_barrier_block = c->skip_block;
    h.fail_node = LLONG_MAX;
    h.fail_step = LLONG_MAX;
    h.barrier = 0;
    h.steps_done = 0;
    CU(cudaMemcpyAsync(c->st, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream), "status reset");
    CU(cudaStreamSynchronize(c->stream), "status reset");
    return FEDFEM_OK;
}

template <typename R, typename L = R>
StepArgs<R, L> make_args(fedfem_ctx* c, const R* M, const R* V, const R* Q, const R* hA, double dt,
                         const R* Qs = nullptr) {
    StepArgs<R, L> a{};
    a.Qs = c->sched_f.empty() ? nullptr : (const L*)Qs;
    a.t0 = c->sim_time;
    a.dtd = dt;
    a.n_seg = (int)c->sched_f.size();
    for (int k = 0; k < a.n_seg; ++k) {
        a.seg_end[k] = c->sched_end[k];
        a.seg_f[k] = (R)c->sched_f[k];
    }
    a.dose = c->dose;
    a.dose_model = c->dose_model;
    a.dose_dt = c->dose_model == FEDFEM_DOSE_ARRHENIUS ? dt : dt / 60.0;
    a.dose_dt32 = (float)a.dose_dt;
    a.dose_lnA = c->dose_model == FEDFEM_DOSE_ARRHENIUS ? std::log(c->dose_A) : 0.0;
    a.dose_EaR = c->dose_Ea / kGasConstant;
    const bool arr = c->dose_model == FEDFEM_DOSE_ARRHENIUS;
    a.dose_c43 = arr ? 0.0f : 1.0f;
    a.dose_a2 = arr ? (float)std::log2(c->dose_A) : 0.0f;
    a.dose_g2 = arr ? (float)(a.dose_EaR / std::log(2.0)) : 0.0f;
    a.E = c->E; a.N = c->N; a.N_plain = c->L.N_plain; a.N_free = c->L.N_free;
    a.conn4 = c->conn4; a.M = M; a.slots = (R*)c->slots;
    a.sell_off = c->sell_off; a.sell_ids = c->sell_ids;
    a.V = V; a.Q = (const L*)Q; a.hA = hA;
    a.T = (L*)c->T; a.T2 = (L*)c->T2; a.Tlo = (L*)c->Tlo;
    a.T_ref = (R)c->mat.T_ref; a.rho0 = (R)c->mat.rho0; a.drho = (R)c->mat.drho;
    a.c0 = (R)c->mat.c0; a.dc = (R)c->mat.dc; a.k0 = (R)c->mat.k0; a.dk = (R)c->mat.dk;
    a.wbcb = (R)(c->perf.w_b * c->perf.c_b); a.T_a = (R)c->perf.T_a; a.T_inf = (R)c->conv_Tinf;
    a.dt = (R)dt; a.T_lo = (R)c->T_lo; a.T_hi = (R)c->T_hi;
    a.status = c->st;
    a.step0 = c->steps_issued;
    a.n_tab = c->tab_n;
    for (int j = 0; j < c->tab_n; ++j) a.tab_T[j] = (R)c->tab_T[j];
    for (int P = 0; P < 3 && c->tab_n > 1; ++P) {
        a.tab_p0[P] = (R)c->tab_p[P][0];
        a.tab_s0[P] = (R)tab_slope(c, P, 0);
        for (int q = 1; q + 1 < c->tab_n; ++q) a.tab_d[P][q] = (R)(tab_slope(c, P, q) - tab_slope(c, P, q - 1));
    }
    a.A28 = std::is_same<R, double>::value ? (const R*)c->A28_64 : (const R*)c->A28_32;
    a.W12 = std::is_same<R, double>::value ? (const R*)c->W64 : (const R*)c->W32;
    a.hg_eps4 = (R)(0.25 * c->hg_eps);
    if (c->n_cq > 0 && c->emat) {
        a.emat = c->emat;
        a.emat_tile = c->t_emat;
        a.emat_off = c->t_emat_off;
        a.mat_k = std::is_same<R, double>::value ? (const R*)c->matk64 : (const R*)c->matk32;
        a.Cq = std::is_same<R, double>::value ? (const R*)c->Cq64 : (const R*)c->Cq32;
    }
    return a;
}

template <typename P>
cudaError_t talloc(fedfem_ctx* c, P** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return e;
    c->tile_allocs.push_back(q);
    *p = (P*)q;
    return cudaSuccess;
}

// bytes of tile t's packed block: int4 header {elements, padded elements,
// halo nodes, most elements at one owned node}, the 6 element-matrix rows
// (padded element count each), the 16-bit local connectivity (nv per padded
// element), the halo node ids; 16-byte multiple
int64_t tile_block_bytes(const Tiles& t, int64_t i, size_t rs, bool hg = false, bool mf = false) {
    const int64_t ne = t.e_off[i + 1] - t.e_off[i], ne_pad = (ne + 7) / 8 * 8;
    const int64_t nh = t.h_off[i + 1] - t.h_off[i];
    const int64_t geo = mf ? 16 * ((int64_t)t.B + nh) : (hg ? 18 : 6) * ne_pad * (int64_t)rs;
    const int64_t b = 16 + geo + ne_pad * t.nv * 2 + nh * 4;
    return (b + 15) / 16 * 16;
}

// largest halo of any tile
int tile_max_halo(const Tiles& t) {
    int h = 0;
    for (int64_t i = 0; i < t.n_tiles; ++i) h = std::max(h, t.h_off[i + 1] - t.h_off[i]);
    return h;
}

// bytes of one replicated-row array (temperature copies or load table): rows
// of stride S plus the halo, 16-byte multiple
size_t rep_bytes(const Tiles& t, size_t ls, int S) {
    return (((size_t)std::max(1, t.max_deg) * S + tile_max_halo(t)) * ls + 15) / 16 * 16;
}

// dynamic shared memory of the tiled kernels (kind: 0 direct, 1 staged, 2 staged
// with replicated rows of stride S): two block stages when staged; the tile
// temperatures and the per-node load table (max_deg rows of B + 1), or the two
// replicated-row arrays
size_t tile_smem(const Tiles& t, size_t rs, size_t ls, int* max_block, int kind, int S, bool hg, bool mf) {
    int64_t mb = 0;
    for (int64_t i = 0; i < t.n_tiles; ++i) mb = std::max(mb, tile_block_bytes(t, i, rs, hg, mf));
    *max_block = (int)mb;
    if (kind == 2) return 128 + 2 * rep_bytes(t, ls, S) + 2 * (size_t)mb;
    const size_t ts = ((size_t)t.max_local * ls + 15) / 16 * 16;
    const size_t b = (kind ? 128 + 2 * (size_t)mb : 0) + ts + ls * (size_t)std::max(1, t.max_deg) * (t.B + 1);
    return (b + 15) / 16 * 16;
}

// threads per block of the staged kernels: the block knob if it names a built
// size.  The replicated-row kernel is built for 128, 256 and 512; its rows have
// one entry per thread, so its default shrinks with the rows' size: 512 for
// hex8 (8 rows), 256 for tet4 (up to 32 rows), halved in FP64.
int staged_threads(const fedfem_ctx* c) {
    if (c->tile.kernel == FEDFEM_KERNEL_TILED_REP) {
        if (c->tile.block == 128 || c->tile.block == 256 || c->tile.block == 512) return c->tile.block;
        const int d = c->nv == 8 ? 512 : 256;
        return c->precision == FEDFEM_FP64 ? d / 2 : d;
    }
    return c->tile.block == 256 || c->tile.block == 1024 ? c->tile.block : tiled_threads();
}

// kind of tiled kernel selected: 0 direct, 1 staged, 2 replicated rows
int tile_kind(const fedfem_ctx* c) {
    return c->tile.kernel == FEDFEM_KERNEL_TILED_REP ? 2 : c->tile.kernel == FEDFEM_KERNEL_TILED_STAGED ? 1 : 0;
}

// Tiles for the tiled kernels.  The requested size is used as given; the
// default (512 owned hex nodes staged, 256 direct; 256 / 128 tet nodes; halved
// in FP64 and with scenario lanes, and again while its tiles do not fit in
// shared memory) is moved to the nearest size that gives every resident block
// the same number of tiles.  Each tile's constant data
// is packed into one 16-byte-aligned block (see tile_block_bytes).
int plan_tiles(fedfem_ctx* c) {
    if (c->tiles_ok) return FEDFEM_OK;
    const int kind = tile_kind(c);
    const bool staged = kind != 0;
    const int S = staged_threads(c);    // replicated-row stride: one owned node per thread
    const size_t rs = c->precision == FEDFEM_FP64 ? sizeof(double) : sizeof(float);
    const size_t ls = rs * c->n_lanes;
    const bool hg = c->W64 || c->W32;   // blocks carry the hourglass weights
    const bool mf = c->matrix_free != 0;  // blocks carry local coordinates instead of the matrices
    if (mf && (c->nv != 4 || c->precision == FEDFEM_FP64 || kind == 2))
        return fail(c, FEDFEM_E_UNSUPPORTED, "matrix-free geometry: tet4, FP32 state, the tiled and staged tiled kernels");
    if (kind == 2 && c->n_lanes > 1) return fail(c, FEDFEM_E_UNSUPPORTED, "the replicated-row kernel takes one lane");
    const int64_t NF = c->L.N_free;
    if (NF == 0) return fail(c, FEDFEM_E_ARG, "no free nodes");
    int B = c->tile.tile_nodes;
    Tiles t;
    std::string m;
    int mb = 0;
    {
        // the requested size exactly; the default size is moved to the nearest one
        // that gives every resident block the same number of tiles at the same
        // occupancy
        int B0 = B;
        if (B0 <= 0) {
            B0 = c->nv == 8 ? (staged ? 512 : 256) : (staged ? 256 : 128);
            if (c->precision == FEDFEM_FP64) B0 /= 2;
            if (c->n_lanes > 1) B0 /= 2;
            if (kind == 2) B0 = std::min(B0, S);
        }
        if (kind == 2 && B0 > S) return fail(c, FEDFEM_E_ARG, "replicated-row tiles hold at most one owned node per thread");
        B0 = (int)std::max<int64_t>(8, std::min<int64_t>(B0, (NF + 7) / 8 * 8));
        int per_sm = 0;
        for (;;) {   // the default size halves while its tiles do not fit (meshes whose tiles hold many elements)
            m = build_tiles(c->L, B0, t);
            if (!m.empty()) return fail(c, FEDFEM_E_ARG, m);
            size_t smem = tile_smem(t, rs, ls, &mb, kind, S, hg, mf);
            per_sm = tiled_blocks_per_sm(c->precision, c->nv, kind, S, c->n_lanes, smem);
            if (c->tile.blocks_per_sm > 0) per_sm = std::min(per_sm, c->tile.blocks_per_sm);
            if (per_sm >= 1 || c->tile.tile_nodes > 0 || B0 <= 32) break;
            B0 = std::max(32, B0 / 2 / 8 * 8);
        }
        if (per_sm < 1) return fail(c, FEDFEM_E_UNSUPPORTED, "tile does not fit in shared memory; use smaller tile_nodes");
        B = B0;
        const int64_t grid = (int64_t)per_sm * c->sm_count;
        const int64_t w0 = std::max<int64_t>(1, (int64_t)std::llround((double)NF / ((double)B0 * grid)));
        for (int64_t waves = w0; waves <= w0 + 1 && c->tile.tile_nodes <= 0; ++waves) {
            const int64_t Bw = ((NF + waves * grid - 1) / (waves * grid) + 7) / 8 * 8;
            if (Bw < 32 || Bw > 2 * (int64_t)B0) continue;                 // small meshes: keep the target
            if (kind == 2 && Bw > S) continue;
            Tiles tw;
            if (!build_tiles(c->L, (int)Bw, tw).empty()) continue;
            int mbw = 0;
            int pw = tiled_blocks_per_sm(c->precision, c->nv, kind, S, c->n_lanes, tile_smem(tw, rs, ls, &mbw, kind, S, hg, mf));
            if (c->tile.blocks_per_sm > 0) pw = std::min(pw, c->tile.blocks_per_sm);
            if (pw != per_sm) continue;
            B = (int)Bw;
            t = std::move(tw);
            break;
        }
    }
    if (t.B != B) {
        m = build_tiles(c->L, B, t);
        if (!m.empty()) return fail(c, FEDFEM_E_ARG, m);
    }
    const size_t smem = tile_smem(t, rs, ls, &mb, kind, S, hg, mf);
    if (kind == 2 && t.max_deg > (c->nv == 8 ? 8 : 32))
        return fail(c, FEDFEM_E_UNSUPPORTED, "the replicated-row kernel takes at most 8 (hex) or 32 (tet) elements per node");
    if (kind == 2 && ls * ((size_t)std::max(1, t.max_deg) * S + tile_max_halo(t)) > 65536)
        return fail(c, FEDFEM_E_UNSUPPORTED, "replicated-row offsets exceed 16 bits; use smaller tiles or 256 threads");
    if (tiled_blocks_per_sm(c->precision, c->nv, kind, S, c->n_lanes, smem) < 1)
        return fail(c, FEDFEM_E_UNSUPPORTED, "tile does not fit in shared memory; use smaller tile_nodes");
    free_tiles(c);
    cudaStream_t st = c->stream;
    // element matrices (and hourglass weights) back to the host once, to pack them per tile
    const int64_t E = c->E;
    std::vector<unsigned char> Mh(rs * 6 * E), Wh(hg ? rs * 12 * E : 0);
    CU(cudaMemcpyAsync(Mh.data(), c->precision == FEDFEM_FP64 ? (void*)c->M64 : (void*)c->M32, rs * 6 * E,
                       cudaMemcpyDeviceToHost, st), "tile pack");
    if (hg)
        CU(cudaMemcpyAsync(Wh.data(), c->precision == FEDFEM_FP64 ? (void*)c->W64 : (void*)c->W32, rs * 12 * E,
                           cudaMemcpyDeviceToHost, st), "tile pack");
    CU(cudaStreamSynchronize(st), "tile pack");
    std::vector<int64_t> off(t.n_tiles + 1, 0);
    for (int64_t i = 0; i < t.n_tiles; ++i) off[i + 1] = off[i] + tile_block_bytes(t, i, rs, hg, mf);
    std::vector<unsigned char> blob(off[t.n_tiles], 0);
    // matrix-free blocks: one origin for every tile, so that a node's stored
    // coordinates (and every element matrix recomputed from them) do not
    // depend on the tiling
    double mf_origin[3] = {0.0, 0.0, 0.0};
    if (mf) {
        for (int d = 0; d < 3; ++d) {
            double lo = c->xyz[d], hi = c->xyz[d];
            for (int64_t n = 1; n < c->N; ++n) {
                lo = std::min(lo, c->xyz[3 * n + d]);
                hi = std::max(hi, c->xyz[3 * n + d]);
            }
            mf_origin[d] = 0.5 * (lo + hi);
        }
    }
    for (int64_t i = 0; i < t.n_tiles; ++i) {
        unsigned char* b = blob.data() + off[i];
        const int64_t e0 = t.e_off[i], ne = t.e_off[i + 1] - e0, ne_pad = (ne + 7) / 8 * 8;
        const int64_t h0 = t.h_off[i], nh = t.h_off[i + 1] - h0;
        const int32_t hdr[4] = {(int32_t)ne, (int32_t)ne_pad, (int32_t)nh, t.deg[i]};
        std::memcpy(b, hdr, 16);
        if (mf) {   // node coordinates relative to the mesh's bounding-box centre, rounded once from FP64
            const int64_t base = i * (int64_t)t.B, own = std::min<int64_t>(t.B, NF - base);
            const double* a0 = mf_origin;
            float* X = (float*)(b + 16);
            auto put = [&](int64_t slot, int64_t internal) {
                const double* x = &c->xyz[3 * (int64_t)c->L.node_of[internal]];
                for (int d = 0; d < 3; ++d) X[4 * slot + d] = (float)(x[d] - a0[d]);
                X[4 * slot + 3] = 0.0f;
            };
            for (int64_t l = 0; l < own; ++l) put(l, base + l);
            for (int64_t h = 0; h < nh; ++h) put(own + h, t.halo[h0 + h]);   // local id own + h
            uint16_t* lc = (uint16_t*)(b + 16 + 16 * ((int64_t)t.B + nh));
            std::memcpy(lc, t.lconn.data() + e0 * t.nv, sizeof(uint16_t) * ne * t.nv);
            int32_t* hh = (int32_t*)(lc + t.nv * ne_pad);
            std::memcpy(hh, t.halo.data() + h0, sizeof(int32_t) * nh);
            continue;
        }
        unsigned char* Mb = b + 16;
        for (int q = 0; q < 6; ++q)
            for (int64_t j = 0; j < ne; ++j)
                std::memcpy(Mb + rs * (6 * j + q), Mh.data() + rs * (q * E + t.e_glob[e0 + j]), rs);
        if (hg) {   // an element's 12 weights together, after the matrices
            unsigned char* Wb = Mb + rs * 6 * ne_pad;
            for (int q = 0; q < 12; ++q)
                for (int64_t j = 0; j < ne; ++j)
                    std::memcpy(Wb + rs * (12 * j + q), Wh.data() + rs * (q * E + t.e_glob[e0 + j]), rs);
        }
        uint16_t* lc = (uint16_t*)(Mb + rs * (hg ? 18 : 6) * ne_pad);
        if (kind == 2) {   // byte offsets into the replicated rows (see TileArgs::rep)
            const int64_t own = std::min<int64_t>(t.B, NF - i * (int64_t)t.B);
            const int id_mask = (1 << t.rank_shift) - 1, D = std::max(1, t.max_deg);
            for (int64_t q = 0; q < ne * t.nv; ++q) {
                const int code = t.lconn[e0 * t.nv + q];
                const int lid = code & id_mask, rank = code >> t.rank_shift;
                const int64_t slot = lid < own ? (int64_t)rank * S + lid : (int64_t)D * S + (lid - own);
                lc[q] = (uint16_t)(slot * (int64_t)ls);
            }
        } else {
            std::memcpy(lc, t.lconn.data() + e0 * t.nv, sizeof(uint16_t) * ne * t.nv);
        }
        int32_t* h = (int32_t*)(lc + t.nv * ne_pad);
        std::memcpy(h, t.halo.data() + h0, sizeof(int32_t) * nh);
    }
    CU(talloc(c, &c->t_blocks, blob.size()), "tile alloc");
    CU(talloc(c, &c->t_block_off, sizeof(int64_t) * off.size()), "tile alloc");
    CU(cudaMemcpyAsync(c->t_blocks, blob.data(), blob.size(), cudaMemcpyHostToDevice, st), "tile copy");
    CU(cudaMemcpyAsync(c->t_block_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, st),
       "tile copy");
    if (c->n_cq > 0 && !c->emat_host.empty()) {   // regions of the tile elements, tile t's from e_off[t]
        std::vector<unsigned char> te(std::max<size_t>(1, t.e_glob.size()));
        for (size_t j = 0; j < t.e_glob.size(); ++j) te[j] = c->emat_host[t.e_glob[j]];
        CU(talloc(c, &c->t_emat, te.size()), "tile alloc");
        CU(talloc(c, &c->t_emat_off, sizeof(int32_t) * t.e_off.size()), "tile alloc");
        CU(cudaMemcpyAsync(c->t_emat, te.data(), te.size(), cudaMemcpyHostToDevice, st), "tile copy");
        CU(cudaMemcpyAsync(c->t_emat_off, t.e_off.data(), sizeof(int32_t) * t.e_off.size(), cudaMemcpyHostToDevice,
                           st), "tile copy");
        CU(cudaStreamSynchronize(st), "tile copy");   // te is a host vector of this frame
    }
    CU(cudaStreamSynchronize(st), "tile build");
    c->t_block_bytes = (int64_t)blob.size();
    c->t_max_block = mb;
    c->t_max_local = t.max_local;
    c->t_max_halo = tile_max_halo(t);
    c->t_smem = smem;
    c->tiles_B = t.B;
    c->tiles_host = std::move(t);
    c->tiles_ok = true;
    return FEDFEM_OK;
}

template <typename R>
TileArgs<R> make_tile_args(fedfem_ctx* c) {
    TileArgs<R> t{};
    const Tiles& h = c->tiles_host;
    t.n_tiles = h.n_tiles; t.B = h.B; t.nv = h.nv;
    t.rank_shift = h.rank_shift; t.max_deg = std::max(1, h.max_deg);
    t.blocks = c->t_blocks; t.block_off = c->t_block_off;
    t.max_block = c->t_max_block; t.max_local = c->t_max_local;
    t.smem_bytes = c->t_smem;
    t.staged = tile_kind(c) != 0;
    t.threads = staged_threads(c);
    t.rep = tile_kind(c) == 2;
    t.rep_rows = std::max(1, h.max_deg);
    t.max_halo = c->t_max_halo;
    t.hourglass = (c->W64 || c->W32) ? 1 : 0;
    t.mf = c->matrix_free;
    return t;
}

// Launch knobs of the next time-loop launch; plans tiles when a tiled kernel
// is selected (host work and allocation: never inside a graph capture).
int prepare_launch(fedfem_ctx* c, LaunchCfg& cfg) {
    cfg.kernel = c->tile.kernel;
    cfg.block = c->tile.block;
    cfg.blocks_per_sm = c->tile.blocks_per_sm;
    cfg.sm_count = c->sm_count;
    cfg.spin_limit = c->spin_limit;
    const bool tiled = cfg.kernel == FEDFEM_KERNEL_TILED || cfg.kernel == FEDFEM_KERNEL_TILED_STAGED ||
                       cfg.kernel == FEDFEM_KERNEL_TILED_REP;
    if (c->n_lanes > 1 && !tiled) return fail(c, FEDFEM_E_UNSUPPORTED, "scenario lanes need a tiled kernel");
    if (!tiled && c->matrix_free)
        return fail(c, FEDFEM_E_UNSUPPORTED, "matrix-free geometry runs on the tiled kernels");
    if (tiled && (c->A28_64 || c->A28_32))
        return fail(c, FEDFEM_E_UNSUPPORTED, "the fully integrated hexahedron runs on the two-phase and persistent kernels");
    if (tiled) return plan_tiles(c);
    return FEDFEM_OK;
}

// Enqueue n_steps of the selected kernel on the context's stream.
cudaError_t launch_all(fedfem_ctx* c, double dt, int64_t n_steps, LaunchCfg& cfg) {
    const bool tiled = cfg.kernel == FEDFEM_KERNEL_TILED || cfg.kernel == FEDFEM_KERNEL_TILED_STAGED ||
                       cfg.kernel == FEDFEM_KERNEL_TILED_REP;
    if (tiled) {
        if (c->precision == FEDFEM_FP64) {
            StepArgs<double> a = make_args<double>(c, c->M64, c->V64, c->Q64, c->hA64, dt, c->Qs64);
            return launch_tiled_f64(a, make_tile_args<double>(c), n_steps, cfg, c->stream);
        }
        const bool kahan = c->precision == FEDFEM_FP32_KAHAN;
        if (c->n_lanes == 4) {
            StepArgs<float, F4> a = make_args<float, F4>(c, c->M32, c->V32, c->Q32, c->hA32, dt, c->Qs32);
            return launch_tiled_f32x4(a, make_tile_args<float>(c), kahan, n_steps, cfg, c->stream);
        }
        StepArgs<float> a = make_args<float>(c, c->M32, c->V32, c->Q32, c->hA32, dt, c->Qs32);
        return launch_tiled_f32(a, make_tile_args<float>(c), kahan, n_steps, cfg, c->stream);
    }
    if (c->precision == FEDFEM_FP64) {
        StepArgs<double> a = make_args<double>(c, c->M64, c->V64, c->Q64, c->hA64, dt, c->Qs64);
        return launch_steps_f64(a, c->nv, n_steps, cfg, c->stream);
    }
    StepArgs<float> a = make_args<float>(c, c->M32, c->V32, c->Q32, c->hA32, dt, c->Qs32);
    return launch_steps_f32(a, c->nv, c->precision == FEDFEM_FP32_KAHAN, n_steps, cfg, c->stream);
}

}  // namespace

// One NVTX range per public call, named after it, so that a profiler's
// timeline shows which library call the kernels and copies belong to (no
// cost unless a tool is attached).
struct ApiRange {
    explicit ApiRange(const char* name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
    ApiRange(const ApiRange&) = delete;
    ApiRange& operator=(const ApiRange&) = delete;
};

extern "C" {

int fedfem_plan_layout(int elem_type, int64_t n_nodes, const double* xyz, int64_t n_elems, const int32_t* conn,
                       const int32_t* groups, int order, int64_t n_dirichlet, const int32_t* dirichlet_nodes,
                       int64_t n_faces, int nverts, const int32_t* faces, int tile_nodes,
                       fedfem_layout_info* info, int32_t* node_of,
                       int32_t* elem_of, int32_t* slice_off, int32_t* gather, int32_t* tile_elem_off,
                       int32_t* tile_elems, uint16_t* tile_lconn, int32_t* tile_halo_off, int32_t* tile_halo,
                       int32_t* tile_degree) {
    if (!info || !xyz || !conn || n_nodes <= 0 || n_elems <= 0) return FEDFEM_E_ARG;
    if (elem_type != FEDFEM_HEX8 && elem_type != FEDFEM_TET4) return FEDFEM_E_ARG;
    if (order < FEDFEM_ORDER_INPUT || order > FEDFEM_ORDER_RCM) return FEDFEM_E_ARG;
    if (n_dirichlet < 0 || (n_dirichlet > 0 && !dirichlet_nodes)) return FEDFEM_E_ARG;
    if (n_faces < 0 || (n_faces > 0 && (!faces || (nverts != 3 && nverts != 4)))) return FEDFEM_E_ARG;
    std::vector<char> dir(n_nodes, 0);
    for (int64_t i = 0; i < n_dirichlet; ++i) {
        if (dirichlet_nodes[i] < 0 || dirichlet_nodes[i] >= n_nodes) return FEDFEM_E_ARG;
        dir[dirichlet_nodes[i]] = 1;
    }
    std::vector<int32_t> fv;
    if (n_faces > 0) {
        fv.assign(faces, faces + n_faces * nverts);
        for (int32_t v : fv)
            if (v < 0 || v >= n_nodes) return FEDFEM_E_ARG;
    }
    MeshInput in;
    in.nv = elem_type; in.N = n_nodes; in.E = n_elems; in.xyz = xyz; in.conn = conn;
    in.is_dirichlet = &dir; in.conv_faces = n_faces > 0 ? &fv : nullptr; in.conv_nverts = n_faces > 0 ? nverts : 0;
    in.order = order;
    std::vector<int32_t> grp;
    if (groups) { grp.assign(groups, groups + n_elems); in.groups = &grp; }
    Layout L;
    bool mesh_err = false;
    std::string m = build_layout(in, L, &mesh_err);
    if (!m.empty()) return mesh_err ? FEDFEM_E_MESH : FEDFEM_E_ARG;
    Tiles t;
    if (tile_nodes > 0) {
        m = build_tiles(L, tile_nodes, t);
        if (!m.empty()) return FEDFEM_E_ARG;
    }
    std::memset(info, 0, sizeof(*info));
    info->n_nodes = n_nodes; info->n_elems = n_elems; info->n_plain = L.N_plain; info->n_free = L.N_free;
    info->n_slices = (int64_t)L.sell_off.size() - 1; info->n_gather = (int64_t)L.sell_ids.size();
    info->max_degree = L.max_degree;
    info->tile_nodes = tile_nodes > 0 ? tile_nodes : 0;
    info->n_tiles = t.n_tiles; info->n_tile_elems = (int64_t)t.e_glob.size(); info->n_halo = (int64_t)t.halo.size();
    info->max_tile_local = t.max_local; info->max_tile_elems = t.max_elems;
    info->max_tile_degree = t.max_deg; info->tile_rank_shift = tile_nodes > 0 ? t.rank_shift : 0;
    auto put = [](auto* dst, const auto& v) { if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(v[0])); };
    put(node_of, L.node_of); put(elem_of, L.elem_of); put(slice_off, L.sell_off); put(gather, L.sell_ids);
    put(tile_elem_off, t.e_off); put(tile_elems, t.e_glob); put(tile_lconn, t.lconn); put(tile_halo_off, t.h_off);
    put(tile_halo, t.halo); put(tile_degree, t.deg);
    return FEDFEM_OK;
}

const char* fedfem_version(void) { return "fedfem-gb300 0.1 (sm_103a)"; }

int fedfem_create(fedfem_ctx** out, int device, int precision, void* cuda_stream) {
    if (!out) return FEDFEM_E_ARG;
    *out = nullptr;
    if (precision < FEDFEM_FP64 || precision > FEDFEM_FP32_PLAIN) return FEDFEM_E_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FEDFEM_E_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return FEDFEM_E_CUDA;
    int major = 0, minor = 0, coop = 0, sms = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (major != 10 || minor != 3 || !coop) return FEDFEM_E_UNSUPPORTED;
    fedfem_ctx* c = new fedfem_ctx();
    c->device = device;
    c->precision = precision;
    c->sm_count = sms;
    if (const char* s = std::getenv("FEDFEM_BARRIER_SPIN_LIMIT")) c->spin_limit = std::max(1000LL, std::atoll(s));
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return FEDFEM_E_CUDA; }
        c->own_stream = true;
    }
    *out = c;
    return FEDFEM_OK;
}

void fedfem_destroy(fedfem_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_device(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* fedfem_last_error(const fedfem_ctx* c) { return c ? c->err.c_str() : "null context"; }

int fedfem_set_mesh(fedfem_ctx* c, int elem_type, int64_t n_nodes, const double* xyz, int64_t n_elems,
                    const int32_t* conn) {
    ApiRange nvtx_range("fedfem_set_mesh");
    if (!c) return FEDFEM_E_ARG;
    if (elem_type != FEDFEM_HEX8 && elem_type != FEDFEM_TET4) return fail(c, FEDFEM_E_ARG, "elem_type must be 4 or 8");
    if (n_nodes <= 0 || n_elems <= 0 || !xyz || !conn) return fail(c, FEDFEM_E_ARG, "empty mesh or null array");
    if (n_nodes >= INT32_MAX) return fail(c, FEDFEM_E_ARG, "n_nodes must fit in int32");
    for (int64_t i = 0; i < 3 * n_nodes; ++i)
        if (!is_finite(xyz[i])) return fail(c, FEDFEM_E_ARG, "non-finite coordinate");
    for (int64_t i = 0; i < n_elems * elem_type; ++i)
        if (conn[i] < 0 || conn[i] >= n_nodes)
            return fail(c, FEDFEM_E_MESH, "element " + std::to_string(i / elem_type) + " has a node id out of range");
    c->nv = elem_type; c->N = n_nodes; c->E = n_elems;
    c->xyz.assign(xyz, xyz + 3 * n_nodes);
    c->conn.assign(conn, conn + n_elems * elem_type);
    c->is_dir.assign(n_nodes, 0);
    c->dir_T.assign(n_nodes, 0.0);
    c->conv_faces.clear(); c->conv_nv = 0; c->conv_h = 0; c->conv_Tinf = 0;
    c->flux.clear(); c->qr.clear(); c->sources.clear(); c->groups.clear();
    c->n_reg = 0; c->region.clear(); c->reg_mat.clear(); c->reg_perf.clear();
    for (auto& q : c->qr_lane) q.clear();
    c->has_mesh = true;
    free_device(c);
    c->err.clear();
    return FEDFEM_OK;
}

int fedfem_set_order(fedfem_ctx* c, int order) {
    if (!c) return FEDFEM_E_ARG;
    if (order < FEDFEM_ORDER_INPUT || order > FEDFEM_ORDER_RCM) return fail(c, FEDFEM_E_ARG, "unknown order");
    c->order = order;
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_material(fedfem_ctx* c, const fedfem_material* m) {
    if (!c || !m) return fail(c, FEDFEM_E_ARG, "null material");
    const double v[7] = {m->T_ref, m->rho0, m->drho, m->c0, m->dc, m->k0, m->dk};
    for (double x : v)
        if (!is_finite(x)) return fail(c, FEDFEM_E_ARG, "non-finite material value");
    if (!(m->rho0 > 0 && m->c0 > 0 && m->k0 > 0)) return fail(c, FEDFEM_E_ARG, "rho0, c0 and k0 must be positive");
    c->mat = *m;
    c->has_mat = true;
    c->tab_n = 0;
    c->n_reg = 0;
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_regions(fedfem_ctx* c, int n, const fedfem_material* mats, const fedfem_perfusion* perf,
                       const int32_t* region) {
    if (!c) return FEDFEM_E_ARG;
    if (!c->has_mesh) return fail(c, FEDFEM_E_STATE, "set_mesh first");
    if (n < 1 || n > kMaxRegions || !mats || !perf || !region)
        return fail(c, FEDFEM_E_ARG, "regions: 1.." + std::to_string(kMaxRegions) + " materials and an id per element");
    for (int r = 0; r < n; ++r) {
        const fedfem_material& m = mats[r];
        const double v[7] = {m.T_ref, m.rho0, m.drho, m.c0, m.dc, m.k0, m.dk};
        for (double x : v)
            if (!is_finite(x)) return fail(c, FEDFEM_E_ARG, "regions: non-finite material value");
        if (!(m.rho0 > 0 && m.c0 > 0 && m.k0 > 0)) return fail(c, FEDFEM_E_ARG, "regions: rho0, c0, k0 must be positive");
        const fedfem_perfusion& p = perf[r];
        if (!(is_finite(p.w_b) && is_finite(p.c_b) && is_finite(p.Q_m)) || p.w_b < 0 || p.c_b < 0)
            return fail(c, FEDFEM_E_ARG, "regions: perfusion values must be finite, w_b and c_b non-negative");
    }
    for (int64_t e = 0; e < c->E; ++e)
        if (region[e] < 0 || region[e] >= n) return fail(c, FEDFEM_E_ARG, "regions: element region out of range");
    c->n_reg = n;
    c->reg_mat.assign(mats, mats + n);
    c->reg_perf.assign(perf, perf + n);
    c->region.assign(region, region + c->E);
    c->mat = mats[0];
    c->has_mat = true;
    c->tab_n = 0;
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_material_table(fedfem_ctx* c, int n, const double* T, const double* rho, const double* cp,
                              const double* k) {
    if (!c) return FEDFEM_E_ARG;
    if (n < 2 || n > kMaxTable || !T || !rho || !cp || !k)
        return fail(c, FEDFEM_E_ARG, "material table: 2.." + std::to_string(kMaxTable) + " points");
    for (int j = 0; j < n; ++j) {
        if (!(is_finite(T[j]) && is_finite(rho[j]) && is_finite(cp[j]) && is_finite(k[j])))
            return fail(c, FEDFEM_E_ARG, "material table: non-finite value");
        if (j > 0 && !(T[j] > T[j - 1])) return fail(c, FEDFEM_E_ARG, "material table: T must increase");
    }
    if (!(rho[0] > 0 && cp[0] > 0 && k[0] > 0))
        return fail(c, FEDFEM_E_ARG, "material table: rho, c and k at the first point must be positive");
    c->tab_n = n;
    for (int j = 0; j < n; ++j) {
        c->tab_T[j] = T[j];
        c->tab_p[0][j] = rho[j];
        c->tab_p[1][j] = cp[j];
        c->tab_p[2][j] = k[j];
    }
    c->mat = fedfem_material{T[0], rho[0], 0.0, cp[0], 0.0, k[0], 0.0};
    c->has_mat = true;
    c->n_reg = 0;
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_perfusion(fedfem_ctx* c, const fedfem_perfusion* p) {
    if (!c || !p) return fail(c, FEDFEM_E_ARG, "null perfusion");
    if (!(is_finite(p->w_b) && is_finite(p->c_b) && is_finite(p->T_a) && is_finite(p->Q_m)) || p->w_b < 0 || p->c_b < 0)
        return fail(c, FEDFEM_E_ARG, "perfusion values must be finite, w_b and c_b non-negative");
    c->perf = *p;
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_source(fedfem_ctx* c, const double* q_r) {
    if (!c) return FEDFEM_E_ARG;
    if (!c->has_mesh) return fail(c, FEDFEM_E_STATE, "set_mesh first");
    if (!q_r) { c->qr.clear(); invalidate(c); return FEDFEM_OK; }
    for (int64_t i = 0; i < c->N; ++i)
        if (!is_finite(q_r[i])) return fail(c, FEDFEM_E_ARG, "non-finite source density");
    c->qr.assign(q_r, q_r + c->N);
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_add_gaussian_source(fedfem_ctx* c, const double x0[3], double sigma, double peak) {
    if (!c || !x0) return fail(c, FEDFEM_E_ARG, "null source centre");
    if (!(is_finite(x0[0]) && is_finite(x0[1]) && is_finite(x0[2]) && is_finite(peak)) || !(sigma > 0) || !is_finite(sigma))
        return fail(c, FEDFEM_E_ARG, "source needs a finite centre and peak and sigma > 0");
    c->sources.push_back({x0[0], x0[1], x0[2], sigma, peak, -1.0, -1.0});
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_add_gaussian_source_lane(fedfem_ctx* c, int lane, int group, const double x0[3], double sigma,
                                    double peak) {
    if (!c) return FEDFEM_E_ARG;
    if (lane < 0 || lane >= c->n_lanes) return fail(c, FEDFEM_E_ARG, "lane out of range (set_lanes first)");
    if (group < -1) return fail(c, FEDFEM_E_ARG, "group must be -1 or a group id");
    int r = fedfem_add_gaussian_source(c, x0, sigma, peak);
    if (r) return r;
    c->sources.back()[5] = (double)lane;
    c->sources.back()[6] = (double)group;
    return FEDFEM_OK;
}

int fedfem_set_source_lane(fedfem_ctx* c, int lane, const double* q_r) {
    if (!c) return FEDFEM_E_ARG;
    if (!c->has_mesh) return fail(c, FEDFEM_E_STATE, "set_mesh first");
    if (lane < 0 || lane >= c->n_lanes) return fail(c, FEDFEM_E_ARG, "lane out of range (set_lanes first)");
    if (!q_r) { c->qr_lane[lane].clear(); invalidate(c); return FEDFEM_OK; }
    for (int64_t i = 0; i < c->N; ++i)
        if (!is_finite(q_r[i])) return fail(c, FEDFEM_E_ARG, "non-finite source density");
    c->qr_lane[lane].assign(q_r, q_r + c->N);
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_lanes(fedfem_ctx* c, int n_lanes) {
    if (!c) return FEDFEM_E_ARG;
    if (n_lanes != 1 && n_lanes != 4) return fail(c, FEDFEM_E_ARG, "n_lanes must be 1 or 4");
    if (n_lanes == 4 && c->precision == FEDFEM_FP64) return fail(c, FEDFEM_E_UNSUPPORTED, "lanes need an FP32 precision");
    c->n_lanes = n_lanes;
    for (auto& s : c->sources)
        if (s[5] >= n_lanes) s[5] = -1.0;
    for (int l = n_lanes; l < 4; ++l) c->qr_lane[l].clear();
    if (n_lanes == 4 && (c->tile.kernel == FEDFEM_KERNEL_PERSISTENT || c->tile.kernel == FEDFEM_KERNEL_TWO_PHASE))
        c->tile.kernel = FEDFEM_KERNEL_TILED;
    free_tiles(c);
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_element_groups(fedfem_ctx* c, const int32_t* group) {
    if (!c) return FEDFEM_E_ARG;
    if (!c->has_mesh) return fail(c, FEDFEM_E_STATE, "set_mesh first");
    if (!group) c->groups.clear();
    else c->groups.assign(group, group + c->E);
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_clear_sources(fedfem_ctx* c) {
    if (!c) return FEDFEM_E_ARG;
    c->sources.clear();
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_dirichlet(fedfem_ctx* c, int64_t n, const int32_t* nodes, const double* T) {
    if (!c) return FEDFEM_E_ARG;
    if (!c->has_mesh) return fail(c, FEDFEM_E_STATE, "set_mesh first");
    if (n < 0 || (n > 0 && (!nodes || !T))) return fail(c, FEDFEM_E_ARG, "bad Dirichlet arrays");
    for (int64_t i = 0; i < n; ++i) {
        if (nodes[i] < 0 || nodes[i] >= c->N) return fail(c, FEDFEM_E_ARG, "Dirichlet node out of range");
        if (!is_finite(T[i])) return fail(c, FEDFEM_E_ARG, "non-finite Dirichlet value");
    }
    std::fill(c->is_dir.begin(), c->is_dir.end(), 0);
    for (int64_t i = 0; i < n; ++i) { c->is_dir[nodes[i]] = 1; c->dir_T[nodes[i]] = T[i]; }
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_convective(fedfem_ctx* c, int64_t n_faces, int nverts, const int32_t* faces, double h, double T_inf) {
    if (!c) return FEDFEM_E_ARG;
    if (!c->has_mesh) return fail(c, FEDFEM_E_STATE, "set_mesh first");
    if (n_faces < 0 || (n_faces > 0 && (!faces || (nverts != 3 && nverts != 4))))
        return fail(c, FEDFEM_E_ARG, "faces need 3 or 4 nodes");
    if (!is_finite(h) || h < 0 || !is_finite(T_inf)) return fail(c, FEDFEM_E_ARG, "film h must be finite and >= 0");
    for (int64_t i = 0; i < n_faces * nverts; ++i)
        if (faces[i] < 0 || faces[i] >= c->N) return fail(c, FEDFEM_E_ARG, "face node out of range");
    c->conv_faces.assign(faces, faces + n_faces * nverts);
    c->conv_nv = n_faces > 0 ? nverts : 0;
    c->conv_h = h;
    c->conv_Tinf = T_inf;
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_nodal_flux(fedfem_ctx* c, int64_t n, const int32_t* nodes, const double* q_W) {
    if (!c) return FEDFEM_E_ARG;
    if (!c->has_mesh) return fail(c, FEDFEM_E_STATE, "set_mesh first");
    if (n < 0 || (n > 0 && (!nodes || !q_W))) return fail(c, FEDFEM_E_ARG, "bad flux arrays");
    for (int64_t i = 0; i < n; ++i) {
        if (nodes[i] < 0 || nodes[i] >= c->N) return fail(c, FEDFEM_E_ARG, "flux node out of range");
        if (!is_finite(q_W[i])) return fail(c, FEDFEM_E_ARG, "non-finite flux");
    }
    c->flux.assign(n > 0 ? c->N : 0, 0.0);
    for (int64_t i = 0; i < n; ++i) c->flux[nodes[i]] += q_W[i];
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_source_schedule(fedfem_ctx* c, int n, const double* t_end, const double* factor) {
    if (!c) return FEDFEM_E_ARG;
    if (n < 0 || n > kMaxSegments || (n > 0 && (!t_end || !factor)))
        return fail(c, FEDFEM_E_ARG, "schedule: 0.." + std::to_string(kMaxSegments) + " segments");
    for (int k = 0; k < n; ++k) {
        if (!is_finite(factor[k]) || std::isnan(t_end[k])) return fail(c, FEDFEM_E_ARG, "schedule: bad value");
        if (k > 0 && !(t_end[k] > t_end[k - 1])) return fail(c, FEDFEM_E_ARG, "schedule: ends must increase");
    }
    c->sched_end.assign(t_end, t_end + n);
    c->sched_f.assign(factor, factor + n);
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_enable_dose(fedfem_ctx* c, int on) {
    if (!c) return FEDFEM_E_ARG;
    c->dose_on = on != 0;
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_lumping(fedfem_ctx* c, int mode) {
    if (!c) return FEDFEM_E_ARG;
    if (mode != FEDFEM_LUMP_ELEMENT && mode != FEDFEM_LUMP_UNIFORM) return fail(c, FEDFEM_E_ARG, "unknown lumping");
    c->lumping = mode;
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_matrix_free(fedfem_ctx* c, int on) {
    if (!c) return FEDFEM_E_ARG;
    if (on != 0 && on != 1) return fail(c, FEDFEM_E_ARG, "matrix-free: 0 or 1");
    if (on && c->has_mesh && c->nv != 4) return fail(c, FEDFEM_E_UNSUPPORTED, "matrix-free geometry is for tet4 meshes");
    c->matrix_free = on;
    free_tiles(c);
    return FEDFEM_OK;
}

int fedfem_set_hourglass_control(fedfem_ctx* c, double eps) {
    if (!c) return FEDFEM_E_ARG;
    if (!(eps >= 0.0) || !is_finite(eps)) return fail(c, FEDFEM_E_ARG, "hourglass strength must be >= 0");
    c->hg_eps = eps;
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_hex_integration(fedfem_ctx* c, int rule) {
    if (!c) return FEDFEM_E_ARG;
    if (rule != FEDFEM_HEX_ONE_POINT && rule != FEDFEM_HEX_FULL) return fail(c, FEDFEM_E_ARG, "unknown hex rule");
    c->hex_rule = rule;
    invalidate(c);
    return FEDFEM_OK;
}

int fedfem_set_dose_model(fedfem_ctx* c, int model, double A, double Ea) {
    if (!c) return FEDFEM_E_ARG;
    if (model == FEDFEM_DOSE_CEM43) {
        c->dose_model = model;
        c->dose_A = c->dose_Ea = 0.0;
        return FEDFEM_OK;
    }
    if (model != FEDFEM_DOSE_ARRHENIUS) return fail(c, FEDFEM_E_ARG, "unknown dose model");
    if (!(is_finite(A) && is_finite(Ea) && A > 0 && Ea > 0))
        return fail(c, FEDFEM_E_ARG, "Arrhenius A and Ea must be finite and positive");
    c->dose_model = model;
    c->dose_A = A;
    c->dose_Ea = Ea;
    return FEDFEM_OK;
}

int fedfem_read_dose_lane(fedfem_ctx* c, int lane, double* out) {
    if (!c || !out) return fail(c, FEDFEM_E_ARG, "null output");
    if (!c->dose) return fail(c, FEDFEM_E_STATE, "enable the dose before fedfem_precompute");
    if (!c->inited) return fail(c, FEDFEM_E_STATE, "init first");
    if (lane < 0 || lane >= c->n_lanes) return fail(c, FEDFEM_E_ARG, "lane out of range");
    CU(cudaSetDevice(c->device), "set device");
    const int64_t NF = c->L.N_free, NL = c->n_lanes;
    std::vector<double> d(std::max<int64_t>(1, NF * NL));
    CU(cudaStreamSynchronize(c->stream), "dose read");
    CU(cudaMemcpy(d.data(), c->dose, sizeof(double) * NF * NL, cudaMemcpyDeviceToHost), "dose read");
    if (c->precision == FEDFEM_FP64) {
        for (int64_t i = 0; i < NF; ++i) out[c->L.node_of[i]] = d[i * NL + lane];
    } else {   // FP32 state: each slot holds the pair (hi, lo)
        const float* h = reinterpret_cast<const float*>(d.data());
        for (int64_t i = 0; i < NF; ++i) {
            const int64_t q = 2 * (i * NL + lane);
            out[c->L.node_of[i]] = (double)h[q] + (double)h[q + 1];
        }
    }
    // Dirichlet nodes sit at their fixed temperature for the whole elapsed time
    for (int64_t i = NF; i < c->N; ++i) {
        const int64_t o = c->L.node_of[i];
        const double T = c->dir_T[o];
        out[o] = c->dose_model == FEDFEM_DOSE_ARRHENIUS
                     ? c->sim_time * std::exp(std::log(c->dose_A) - c->dose_Ea / kGasConstant / (T + 273.15))
                     : c->sim_time / 60.0 * std::exp2(T >= 43.0 ? T - 43.0 : 2.0 * (T - 43.0));
    }
    return FEDFEM_OK;
}

int fedfem_read_dose(fedfem_ctx* c, double* out) { return fedfem_read_dose_lane(c, 0, out); }

int fedfem_set_tile(fedfem_ctx* c, const fedfem_tile* t) {
    if (!c || !t) return fail(c, FEDFEM_E_ARG, "null tile");
    if (t->kernel < FEDFEM_KERNEL_TWO_PHASE || t->kernel > FEDFEM_KERNEL_TILED_REP) return fail(c, FEDFEM_E_ARG, "unknown kernel");
    if (t->block != 0 && (t->block < 64 || t->block > 1024 || t->block % 32)) return fail(c, FEDFEM_E_ARG, "block must be 64..1024, multiple of 32");
    if (t->blocks_per_sm < 0 || t->tile_nodes < 0 || t->tile_nodes % 8) return fail(c, FEDFEM_E_ARG, "bad tile knobs");
    if (t->tile_nodes != c->tile.tile_nodes || t->blocks_per_sm != c->tile.blocks_per_sm ||
        t->block != c->tile.block ||
        (t->kernel == FEDFEM_KERNEL_TILED_STAGED) != (c->tile.kernel == FEDFEM_KERNEL_TILED_STAGED) ||
        (t->kernel == FEDFEM_KERNEL_TILED_REP) != (c->tile.kernel == FEDFEM_KERNEL_TILED_REP))
        free_tiles(c);
    c->tile = *t;
    return FEDFEM_OK;
}

int fedfem_debug_set(fedfem_ctx* c, int key, int64_t value) {
    if (!c) return FEDFEM_E_ARG;
    if (key == 1) { c->spin_limit = std::max<long long>(1000, value); return FEDFEM_OK; }
    if (key == 2) { c->skip_block = (int)value; return FEDFEM_OK; }
    return fail(c, FEDFEM_E_ARG, "unknown debug key");
}

int fedfem_precompute(fedfem_ctx* c, double T_lo, double T_hi, double* dt_cr_out) {
    ApiRange nvtx_range("fedfem_precompute");
    if (!c) return FEDFEM_E_ARG;
    if (!c->has_mesh || !c->has_mat) return fail(c, FEDFEM_E_STATE, "set_mesh and set_material first");
    if (!(is_finite(T_lo) && is_finite(T_hi) && T_lo < T_hi)) return fail(c, FEDFEM_E_ARG, "need T_lo < T_hi");
    if (c->lumping == FEDFEM_LUMP_UNIFORM && (c->n_reg > 0 || c->tab_n > 0))
        return fail(c, FEDFEM_E_UNSUPPORTED, "uniform lumping takes one material with linear laws");
    double s = 1.0;
    int rc = property_scale(c, T_lo, T_hi, &s);
    if (rc) return rc;
    CU(cudaSetDevice(c->device), "set device");
    free_device(c);
    // ---- layout (host, integer work) ----
    MeshInput in;
    in.nv = c->nv; in.N = c->N; in.E = c->E; in.xyz = c->xyz.data(); in.conn = c->conn.data();
    in.is_dirichlet = &c->is_dir;
    in.conv_faces = c->conv_nv ? &c->conv_faces : nullptr;
    in.conv_nverts = c->conv_nv;
    in.order = c->order;
    in.groups = c->groups.empty() ? nullptr : &c->groups;
    bool mesh_err = false;
    std::string m = build_layout(in, c->L, &mesh_err);
    if (!m.empty()) return fail(c, mesh_err ? FEDFEM_E_MESH : FEDFEM_E_ARG, m);
    const Layout& L = c->L;
    const int64_t N = c->N, E = c->E, NF = L.N_free, NC = L.N_free - L.N_plain;
    const int nv = c->nv;
    cudaStream_t st = c->stream;
    // ---- device arrays ----
    std::vector<int32_t> c4((size_t)E * nv);
    for (int p = 0; p < nv / 4; ++p)
        for (int64_t e = 0; e < E; ++e)
            for (int k = 0; k < 4; ++k) c4[((size_t)p * E + e) * 4 + k] = L.conn[e * nv + 4 * p + k];
    std::vector<double> xs(N), ys(N), zs(N);
    for (int64_t i = 0; i < N; ++i) {
        const int64_t o = L.node_of[i];
        xs[i] = c->xyz[3 * o]; ys[i] = c->xyz[3 * o + 1]; zs[i] = c->xyz[3 * o + 2];
    }
    double *x = nullptr, *y = nullptr, *z = nullptr, *Vshare = nullptr, *face_share = nullptr, *qr = nullptr,
           *flux = nullptr, *src = nullptr;
    int32_t *faces = nullptr, *conv_off = nullptr, *conv_face = nullptr;
    int* bad = nullptr;
    CU(dalloc(c, &c->conn4, sizeof(int32_t) * E * nv), "alloc");
    CU(dalloc(c, &x, sizeof(double) * N), "alloc");
    CU(dalloc(c, &y, sizeof(double) * N), "alloc");
    CU(dalloc(c, &z, sizeof(double) * N), "alloc");
    CU(dalloc(c, &c->M64, sizeof(double) * 6 * E), "alloc");
    CU(dalloc(c, &Vshare, sizeof(double) * (E + 1)), "alloc");
    CU(dalloc(c, &bad, sizeof(int)), "alloc");
    CU(dalloc(c, &c->sell_off, sizeof(int32_t) * L.sell_off.size()), "alloc");
    CU(dalloc(c, &c->sell_ids, sizeof(int32_t) * L.sell_ids.size()), "alloc");
    const int NL = c->n_lanes;
    CU(dalloc(c, &c->V64, sizeof(double) * NF), "alloc");
    CU(dalloc(c, &c->Q64, sizeof(double) * NF * NL), "alloc");
    CU(dalloc(c, &c->hA64, sizeof(double) * NC), "alloc");
    CU(dalloc(c, &c->node_of, sizeof(int32_t) * N), "alloc");
    CU(dalloc(c, &c->T_dir, sizeof(double) * (N - NF)), "alloc");
    CU(dalloc(c, &c->io, sizeof(double) * N * NL), "alloc");
    CU(dalloc(c, &c->st, sizeof(DevStatus)), "alloc");
    CU(cudaMemcpyAsync(c->conn4, c4.data(), sizeof(int32_t) * E * nv, cudaMemcpyHostToDevice, st), "copy");
    CU(cudaMemcpyAsync(x, xs.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st), "copy");
    CU(cudaMemcpyAsync(y, ys.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st), "copy");
    CU(cudaMemcpyAsync(z, zs.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st), "copy");
    CU(cudaMemcpyAsync(c->sell_off, L.sell_off.data(), sizeof(int32_t) * L.sell_off.size(), cudaMemcpyHostToDevice, st), "copy");
    CU(cudaMemcpyAsync(c->sell_ids, L.sell_ids.data(), sizeof(int32_t) * L.sell_ids.size(), cudaMemcpyHostToDevice, st), "copy");
    CU(cudaMemcpyAsync(c->node_of, L.node_of.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st), "copy");
    {
        std::vector<double> td(N - NF);
        for (int64_t i = NF; i < N; ++i) td[i - NF] = c->dir_T[L.node_of[i]];
        CU(cudaMemcpyAsync(c->T_dir, td.data(), sizeof(double) * td.size(), cudaMemcpyHostToDevice, st), "copy");
        CU(cudaStreamSynchronize(st), "copy");
    }
    const int bad_init = INT_MAX;
    CU(cudaMemcpyAsync(bad, &bad_init, sizeof(int), cudaMemcpyHostToDevice, st), "copy");
    std::vector<int32_t> fint;
    if (c->conv_nv) {
        fint.resize(c->conv_faces.size());
        for (size_t i = 0; i < fint.size(); ++i) fint[i] = L.node_at[c->conv_faces[i]];
        CU(dalloc(c, &faces, sizeof(int32_t) * fint.size()), "alloc");
        CU(dalloc(c, &face_share, sizeof(double) * (fint.size() / c->conv_nv)), "alloc");
        CU(cudaMemcpyAsync(faces, fint.data(), sizeof(int32_t) * fint.size(), cudaMemcpyHostToDevice, st), "copy");
    }
    CU(dalloc(c, &conv_off, sizeof(int32_t) * L.conv_off.size()), "alloc");
    CU(dalloc(c, &conv_face, sizeof(int32_t) * std::max<size_t>(1, L.conv_face.size())), "alloc");
    CU(cudaMemcpyAsync(conv_off, L.conv_off.data(), sizeof(int32_t) * L.conv_off.size(), cudaMemcpyHostToDevice, st), "copy");
    if (!L.conv_face.empty())
        CU(cudaMemcpyAsync(conv_face, L.conv_face.data(), sizeof(int32_t) * L.conv_face.size(), cudaMemcpyHostToDevice, st), "copy");
    std::vector<double> qr_int, flux_int, src_h;
    bool any_qr = !c->qr.empty();
    for (int l = 0; l < NL; ++l) any_qr = any_qr || !c->qr_lane[l].empty();
    if (any_qr) {
        qr_int.assign(NF * NL, 0.0);
        for (int l = 0; l < NL; ++l)
            for (int64_t i = 0; i < NF; ++i) {
                const int64_t o = L.node_of[i];
                qr_int[l * NF + i] = (c->qr.empty() ? 0.0 : c->qr[o]) + (c->qr_lane[l].empty() ? 0.0 : c->qr_lane[l][o]);
            }
        CU(dalloc(c, &qr, sizeof(double) * NF * NL), "alloc");
        CU(cudaMemcpyAsync(qr, qr_int.data(), sizeof(double) * NF * NL, cudaMemcpyHostToDevice, st), "copy");
        CU(cudaStreamSynchronize(st), "copy");
    }
    if (!c->flux.empty()) {
        flux_int.resize(NF);
        for (int64_t i = 0; i < NF; ++i) flux_int[i] = c->flux[L.node_of[i]];
        CU(dalloc(c, &flux, sizeof(double) * NF), "alloc");
        CU(cudaMemcpyAsync(flux, flux_int.data(), sizeof(double) * NF, cudaMemcpyHostToDevice, st), "copy");
    }
    for (auto& sgm : c->sources) src_h.insert(src_h.end(), sgm.begin(), sgm.end());   // 7 per source
    int32_t* node_group = nullptr;
    if (!c->groups.empty()) {
        std::vector<int32_t> ng(NF, -1);
        for (int64_t e = 0; e < E; ++e)
            for (int k = 0; k < nv; ++k) {
                const int32_t n = L.conn[e * nv + k];
                if (n < NF && ng[n] < 0) ng[n] = c->groups[L.elem_of[e]];
            }
        CU(dalloc(c, &node_group, sizeof(int32_t) * std::max<int64_t>(1, NF)), "alloc");
        CU(cudaMemcpyAsync(node_group, ng.data(), sizeof(int32_t) * NF, cudaMemcpyHostToDevice, st), "copy");
        CU(cudaStreamSynchronize(st), "copy");
    }
    CU(dalloc(c, &src, sizeof(double) * std::max<size_t>(1, src_h.size())), "alloc");
    if (!src_h.empty())
        CU(cudaMemcpyAsync(src, src_h.data(), sizeof(double) * src_h.size(), cudaMemcpyHostToDevice, st), "copy");

    PreArgs pa{};
    pa.nv = nv; pa.E = E; pa.N = N; pa.N_plain = L.N_plain; pa.N_free = NF;
    pa.conn4 = c->conn4; pa.x = x; pa.y = y; pa.z = z;
    pa.M64 = c->M64; pa.Vshare = Vshare; pa.bad_elem = bad;
    pa.sell_off = c->sell_off; pa.sell_ids = c->sell_ids;
    pa.V = c->V64; pa.Q = c->Q64; pa.hA = c->hA64;
    pa.qr_node = qr; pa.flux_node = flux; pa.src = src; pa.n_src = (int)c->sources.size(); pa.n_lanes = NL;
    pa.node_group = node_group;
    const bool uniform = c->lumping == FEDFEM_LUMP_UNIFORM;
    pa.Q_m = c->n_reg > 0 || uniform ? 0.0 : c->perf.Q_m;   // regions, uniform lumping: added below
    pa.n_faces = c->conv_nv ? (int64_t)fint.size() / c->conv_nv : 0;
    pa.face_nv = c->conv_nv; pa.faces = faces; pa.face_share = face_share;
    pa.conv_off = conv_off; pa.conv_face = conv_face; pa.h_film = c->conv_h;
    if (nv == 8 && c->hg_eps > 0.0 && c->hex_rule == FEDFEM_HEX_FULL)
        return fail(c, FEDFEM_E_UNSUPPORTED, "hourglass control applies to the one-point hexahedron");
    if (nv == 8 && c->hg_eps > 0.0) {   // hourglass weights, computed with the one-point matrices
        CU(dalloc(c, &c->W64, sizeof(double) * 12 * std::max<int64_t>(1, E)), "alloc");
        pa.W64 = c->W64;
        pa.hg_eps4 = 0.25 * c->hg_eps;
    }
    CU(launch_geometry(pa, st), "geometry kernel");
    if (nv == 8 && c->hex_rule == FEDFEM_HEX_FULL) {   // A_e by 2 x 2 x 2 Gauss points, exact V_e
        CU(dalloc(c, &c->A28_64, sizeof(double) * 28 * std::max<int64_t>(1, E)), "alloc");
        pa.A28 = c->A28_64;
        CU(launch_geometry_full(pa, st), "geometry kernel");
    }
    int bad_h = INT_MAX;
    CU(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
    CU(cudaStreamSynchronize(st), "geometry kernel");
    if (bad_h != INT_MAX) {
        const int in_e = L.elem_of[bad_h];
        free_device(c);
        return fail(c, FEDFEM_E_MESH, "element " + std::to_string(in_e) + " has det J <= 0 (inverted or degenerate)");
    }
    CU(launch_nodal(pa, st), "nodal kernel");
    if (!c->sched_f.empty()) {   // time-varying sources: Q = constant part, Qs = source part
        CU(dalloc(c, &c->Qs64, sizeof(double) * NF * NL), "alloc");
        PreArgs ps = pa;
        ps.Q = c->Qs64; ps.Q_m = 0.0; ps.flux_node = nullptr;
        CU(launch_nodal(ps, st), "nodal kernel");
        PreArgs pc = pa;
        pc.qr_node = nullptr; pc.n_src = 0;
        CU(launch_nodal(pc, st), "nodal kernel");
    }
    if (c->dose_on) CU(dalloc(c, &c->dose, sizeof(double) * std::max<int64_t>(1, NF * NL)), "alloc");
    double wbcb_ref = c->perf.w_b * c->perf.c_b;
    const double* beta_ref = nullptr;   // exact per-node perfusion for the Lanczos operator (uniform lumping)
    c->n_cq = c->n_reg > 0 ? c->n_reg : (uniform ? 1 : 0);
    if (c->n_cq > 0) {
        // element regions in internal order (uniform lumping: one region, the
        // material); per region: rho c expanded about the first region's T_ref
        // (u = T - T_ref), w_b c_b and Q_m; its k law
        c->emat_host.assign(E, 0);
        if (c->n_reg > 0)
            for (int64_t e = 0; e < E; ++e) c->emat_host[e] = (unsigned char)c->region[L.elem_of[e]];
        const double Tr = c->n_reg > 0 ? c->reg_mat[0].T_ref : c->mat.T_ref;
        std::vector<double> coef(5 * c->n_cq), kl(3 * c->n_cq);
        if (c->n_reg > 0) wbcb_ref = 0.0;
        for (int r = 0; r < c->n_cq; ++r) {
            const fedfem_material& m = c->n_reg > 0 ? c->reg_mat[r] : c->mat;
            const double a = m.rho0 + m.drho * (Tr - m.T_ref), b = m.drho;
            const double al = m.c0 + m.dc * (Tr - m.T_ref), be = m.dc;
            coef[5 * r + 0] = a * al;
            coef[5 * r + 1] = a * be + b * al;
            coef[5 * r + 2] = b * be;
            coef[5 * r + 3] = c->n_reg > 0 ? c->reg_perf[r].w_b * c->reg_perf[r].c_b : 0.0;   // uniform: below
            coef[5 * r + 4] = c->n_reg > 0 ? c->reg_perf[r].Q_m : 0.0;
            kl[3 * r + 0] = m.T_ref; kl[3 * r + 1] = m.k0; kl[3 * r + 2] = m.dk;
            if (c->n_reg > 0) wbcb_ref = std::max(wbcb_ref, coef[5 * r + 3]);
        }
        double* coef_d = nullptr;
        CU(dalloc(c, &c->emat, std::max<int64_t>(1, E)), "alloc");
        CU(dalloc(c, &coef_d, sizeof(double) * coef.size()), "alloc");
        CU(dalloc(c, &c->matk64, sizeof(double) * kl.size()), "alloc");
        CU(dalloc(c, &c->Cq64, sizeof(double) * 4 * std::max<int64_t>(1, NF)), "alloc");
        CU(cudaMemcpyAsync(c->emat, c->emat_host.data(), E, cudaMemcpyHostToDevice, st), "copy");
        CU(cudaMemcpyAsync(coef_d, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, st), "copy");
        CU(cudaMemcpyAsync(c->matk64, kl.data(), sizeof(double) * kl.size(), cudaMemcpyHostToDevice, st), "copy");
        CU(launch_regions(pa, c->emat, coef_d, c->Cq64, st), "region kernel");
        CU(cudaStreamSynchronize(st), "region kernel");   // coef and kl are host vectors of this frame
        release(c, coef_d, sizeof(double) * coef.size());
        if (uniform) {   // every node: beta = w_b c_b V / N, metabolic Q_m V / N (V the mesh volume, N its nodes)
            std::vector<double> vs(E), q(NF * NL), b(NF);
            CU(cudaMemcpy(vs.data(), Vshare, sizeof(double) * E, cudaMemcpyDeviceToHost), "copy");
            double V_total = 0.0;
            for (int64_t e = 0; e < E; ++e) V_total += vs[e];
            const double share = V_total * nv / (double)N;
            std::fill(b.begin(), b.end(), c->perf.w_b * c->perf.c_b * share);
            CU(cudaMemcpy(q.data(), c->Q64, sizeof(double) * NF * NL, cudaMemcpyDeviceToHost), "copy");
            for (double& x : q) x += c->perf.Q_m * share;
            CU(cudaMemcpy(c->Q64, q.data(), sizeof(double) * NF * NL, cudaMemcpyHostToDevice), "copy");
            CU(cudaMemcpy(c->Cq64 + 3 * NF, b.data(), sizeof(double) * NF, cudaMemcpyHostToDevice), "copy");
            beta_ref = c->Cq64 + 3 * NF;
        }
    }
    CU(cudaStreamSynchronize(st), "nodal kernel");
    LanczosResult lr;
    // regions: the reference operator takes the first region's k0 and rho0 c0
    // everywhere and the largest w_b c_b (property_scale bounds the rest)
    std::string lm = lanczos_lambda_max(pa, c->mat.k0, c->mat.rho0 * c->mat.c0, wbcb_ref, beta_ref,
                                        3000, 1e-14, lr, st);
    if (!lm.empty()) return fail(c, FEDFEM_E_CUDA, lm);
    c->lambda = lr.lambda;
    c->lz_iters = lr.iterations;
    c->td_scale = s;
    c->T_lo = T_lo; c->T_hi = T_hi;
    c->dt_cr = lr.lambda > 0 ? 2.0 / (s * lr.lambda) : INFINITY;
    // ---- time-loop arrays ----
    if (c->precision == FEDFEM_FP64) {
        CU(dalloc(c, (double**)&c->T, sizeof(double) * N), "alloc");
        CU(dalloc(c, (double**)&c->T2, sizeof(double) * N), "alloc");
        CU(dalloc(c, (double**)&c->slots, sizeof(double) * (E * nv + 1)), "alloc");
        CU(cudaMemsetAsync(c->slots, 0, sizeof(double) * (E * nv + 1), st), "memset");
    } else {
        CU(dalloc(c, &c->M32, sizeof(float) * 6 * E), "alloc");
        CU(dalloc(c, &c->V32, sizeof(float) * NF), "alloc");
        CU(dalloc(c, &c->Q32, sizeof(float) * NF * NL), "alloc");
        CU(dalloc(c, &c->hA32, sizeof(float) * NC), "alloc");
        CU(launch_to_f32(c->M64, c->M32, 6 * E, st), "convert");
        if (c->A28_64) {
            CU(dalloc(c, &c->A28_32, sizeof(float) * 28 * std::max<int64_t>(1, E)), "alloc");
            CU(launch_to_f32(c->A28_64, c->A28_32, 28 * E, st), "convert");
        }
        if (c->W64) {
            CU(dalloc(c, &c->W32, sizeof(float) * 12 * std::max<int64_t>(1, E)), "alloc");
            CU(launch_to_f32(c->W64, c->W32, 12 * E, st), "convert");
        }
        CU(launch_to_f32(c->V64, c->V32, NF, st), "convert");
        CU(launch_pack_lanes(c->Q64, c->Q32, NL, NF, st), "convert");
        CU(launch_to_f32(c->hA64, c->hA32, NC, st), "convert");
        if (c->Qs64) {
            CU(dalloc(c, &c->Qs32, sizeof(float) * NF * NL), "alloc");
            CU(launch_pack_lanes(c->Qs64, c->Qs32, NL, NF, st), "convert");
        }
        if (c->Cq64) {
            CU(dalloc(c, &c->Cq32, sizeof(float) * 4 * std::max<int64_t>(1, NF)), "alloc");
            CU(dalloc(c, &c->matk32, sizeof(float) * 3 * c->n_cq), "alloc");
            CU(launch_to_f32(c->Cq64, c->Cq32, 4 * NF, st), "convert");
            CU(launch_to_f32(c->matk64, c->matk32, 3 * c->n_cq, st), "convert");
        }
        CU(dalloc(c, (float**)&c->T, sizeof(float) * N * NL), "alloc");
        CU(dalloc(c, (float**)&c->T2, sizeof(float) * N * NL), "alloc");
        CU(dalloc(c, &c->Tlo, sizeof(float) * N * NL), "alloc");
        CU(dalloc(c, (float**)&c->slots, sizeof(float) * (E * nv + 1)), "alloc");
        CU(cudaMemsetAsync(c->slots, 0, sizeof(float) * (E * nv + 1), st), "memset");
    }
    CU(cudaStreamSynchronize(st), "precompute");
    // pre-computation scratch no longer needed
    release(c, x, sizeof(double) * N); release(c, y, sizeof(double) * N); release(c, z, sizeof(double) * N);
    release(c, Vshare, sizeof(double) * (E + 1)); release(c, bad, sizeof(int));
    release(c, faces, sizeof(int32_t) * fint.size());
    release(c, face_share, sizeof(double) * (fint.size() / std::max(1, c->conv_nv)));
    release(c, conv_off, sizeof(int32_t) * L.conv_off.size());
    release(c, conv_face, sizeof(int32_t) * std::max<size_t>(1, L.conv_face.size()));
    release(c, qr, sizeof(double) * NF * NL); release(c, flux, sizeof(double) * NF);
    release(c, src, sizeof(double) * std::max<size_t>(1, src_h.size()));
    release(c, node_group, sizeof(int32_t) * std::max<int64_t>(1, NF));
    if (c->precision != FEDFEM_FP64) {
        release(c, c->M64, sizeof(double) * 6 * E); c->M64 = nullptr;
        if (c->A28_64) { release(c, c->A28_64, sizeof(double) * 28 * std::max<int64_t>(1, E)); c->A28_64 = nullptr; }
        if (c->W64) { release(c, c->W64, sizeof(double) * 12 * std::max<int64_t>(1, E)); c->W64 = nullptr; }
        release(c, c->V64, sizeof(double) * NF); c->V64 = nullptr;
        release(c, c->Q64, sizeof(double) * NF * NL); c->Q64 = nullptr;
        release(c, c->hA64, sizeof(double) * NC); c->hA64 = nullptr;
        if (c->Qs64) { release(c, c->Qs64, sizeof(double) * NF * NL); c->Qs64 = nullptr; }
        if (c->Cq64) {
            release(c, c->Cq64, sizeof(double) * 4 * std::max<int64_t>(1, NF)); c->Cq64 = nullptr;
            release(c, c->matk64, sizeof(double) * 3 * c->n_cq); c->matk64 = nullptr;
        }
    }
    c->pre = true;
    c->inited = false;
    if (dt_cr_out) *dt_cr_out = c->dt_cr;
    c->err.clear();
    return FEDFEM_OK;
}

static int mirror_T(fedfem_ctx* c) {
    const size_t rs = c->precision == FEDFEM_FP64 ? sizeof(double) : sizeof(float);
    CU(cudaMemcpyAsync(c->T2, c->T, rs * c->N * c->n_lanes, cudaMemcpyDeviceToDevice, c->stream), "mirror");
    return FEDFEM_OK;
}

static int init_common(fedfem_ctx* c, bool per_lane = false) {
    for (int l = 1; l < c->n_lanes && !per_lane; ++l)   // every lane starts from the same field
        CU(cudaMemcpyAsync(c->io + l * c->N, c->io, sizeof(double) * c->N, cudaMemcpyDeviceToDevice, c->stream),
           "init copy");
    CU(launch_init_state(c->precision, c->n_lanes, c->N, c->L.N_free, c->node_of, c->io, c->T_dir, c->T, c->Tlo,
                         c->stream),
       "init kernel");
    if (int r = mirror_T(c)) return r;
    if (c->dose)
        CU(cudaMemsetAsync(c->dose, 0, sizeof(double) * std::max<int64_t>(1, c->L.N_free * c->n_lanes), c->stream),
           "dose reset");
    int r = reset_status(c);
    if (r) return r;
    c->inited = true;
    c->steps_issued = 0;
    c->sim_time = 0.0;
    c->err.clear();
    return FEDFEM_OK;
}

// any non-finite value among the n staged values sets the status word bad_input
static __global__ void k_check_finite(const double* v, int64_t n, DevStatus* st) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(v[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->bad_input, 1ULL);
}

// FEDFEM_OK when every one of the n staged initial values is finite: one pass on
// the device and an 8-byte read, instead of a host pass over the caller's array
static int check_initial_field(fedfem_ctx* c, const double* v, int64_t n) {
    CU(cudaMemsetAsync(&c->st->bad_input, 0, sizeof(unsigned long long), c->stream), "check T0");
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8LL * c->sm_count));
    k_check_finite<<<grid, 256, 0, c->stream>>>(v, n, c->st);
    CU(cudaGetLastError(), "check T0");
    unsigned long long bad = 0;
    CU(cudaMemcpyAsync(&bad, &c->st->bad_input, sizeof bad, cudaMemcpyDeviceToHost, c->stream), "check T0");
    CU(cudaStreamSynchronize(c->stream), "check T0");
    return bad ? fail(c, FEDFEM_E_ARG, "non-finite initial temperature") : FEDFEM_OK;
}

int fedfem_init(fedfem_ctx* c, const double* T0, double T0_uniform) {
    ApiRange nvtx_range("fedfem_init");
    if (!c) return FEDFEM_E_ARG;
    if (!c->pre) return fail(c, FEDFEM_E_STATE, "precompute first");
    CU(cudaSetDevice(c->device), "set device");
    if (T0) {
        CU(cudaMemcpyAsync(c->io, T0, sizeof(double) * c->N, cudaMemcpyHostToDevice, c->stream), "copy T0");
        if (int r = check_initial_field(c, c->io, c->N)) return r;
    } else {
        if (!is_finite(T0_uniform)) return fail(c, FEDFEM_E_ARG, "non-finite initial temperature");
        std::vector<double> u(c->N, T0_uniform);
        CU(cudaMemcpyAsync(c->io, u.data(), sizeof(double) * c->N, cudaMemcpyHostToDevice, c->stream), "copy T0");
        CU(cudaStreamSynchronize(c->stream), "copy T0");
    }
    return init_common(c);
}

int fedfem_init_device(fedfem_ctx* c, const double* T0_dev) {
    ApiRange nvtx_range("fedfem_init_device");
    if (!c || !T0_dev) return fail(c, FEDFEM_E_ARG, "null T0");
    if (!c->pre) return fail(c, FEDFEM_E_STATE, "precompute first");
    CU(cudaSetDevice(c->device), "set device");
    CU(cudaMemcpyAsync(c->io, T0_dev, sizeof(double) * c->N, cudaMemcpyDeviceToDevice, c->stream), "copy T0");
    if (int r = check_initial_field(c, c->io, c->N)) return r;
    return init_common(c);
}

int fedfem_init_lanes_device(fedfem_ctx* c, const double* T0_dev) {
    if (!c || !T0_dev) return fail(c, FEDFEM_E_ARG, "null T0");
    if (!c->pre) return fail(c, FEDFEM_E_STATE, "precompute first");
    CU(cudaSetDevice(c->device), "set device");
    CU(cudaMemcpyAsync(c->io, T0_dev, sizeof(double) * c->N * c->n_lanes, cudaMemcpyDeviceToDevice, c->stream),
       "copy T0");
    if (int r = check_initial_field(c, c->io, c->N * c->n_lanes)) return r;
    return init_common(c, true);
}

int fedfem_read_lanes_device(fedfem_ctx* c, double* out_dev) {
    if (!c || !out_dev) return fail(c, FEDFEM_E_ARG, "null output");
    if (!c->inited) return fail(c, FEDFEM_E_STATE, "init first");
    CU(cudaSetDevice(c->device), "set device");
    for (int l = 0; l < c->n_lanes; ++l)
        CU(launch_read_state(c->precision, c->n_lanes, l, c->N, c->node_of, c->T, c->Tlo, out_dev + l * c->N,
                             c->stream),
           "read kernel");
    CU(cudaStreamSynchronize(c->stream), "read");
    return FEDFEM_OK;
}

int fedfem_step(fedfem_ctx* c, double dt, int64_t n_steps) {
    ApiRange nvtx_range("fedfem_step");
    if (!c) return FEDFEM_E_ARG;
    if (!c->inited) return fail(c, FEDFEM_E_STATE, "init first");
    if (!(dt > 0) || !is_finite(dt) || n_steps < 0) return fail(c, FEDFEM_E_ARG, "need dt > 0 and n_steps >= 0");
    if (!(dt < c->dt_cr)) return fail(c, FEDFEM_E_UNSTABLE_DT, "dt >= critical step " + std::to_string(c->dt_cr));
    if (n_steps == 0) return FEDFEM_OK;
    CU(cudaSetDevice(c->device), "set device");
    LaunchCfg cfg;
    if (int r = prepare_launch(c, cfg)) return r;
    cudaError_t e = launch_all(c, dt, n_steps, cfg);
    if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
    c->last = cfg;
    c->steps_issued += n_steps;
    c->sim_time += dt * (double)n_steps;
    return FEDFEM_OK;
}

int fedfem_capture_graph(fedfem_ctx* c, double dt, int64_t n_steps) {
    if (!c) return FEDFEM_E_ARG;
    if (!c->inited) return fail(c, FEDFEM_E_STATE, "init first");
    if (!(dt > 0) || !is_finite(dt) || n_steps <= 0) return fail(c, FEDFEM_E_ARG, "need dt > 0 and n_steps > 0");
    if (!(dt < c->dt_cr)) return fail(c, FEDFEM_E_UNSTABLE_DT, "dt >= critical step " + std::to_string(c->dt_cr));
    if (!c->sched_f.empty())
        return fail(c, FEDFEM_E_UNSUPPORTED, "a graph fixes the start time; step a source schedule with fedfem_step");
    CU(cudaSetDevice(c->device), "set device");
    LaunchCfg cfg;
    if (int r = prepare_launch(c, cfg)) return r;   // tiles are planned outside the capture
    free_graph(c);
    CU(cudaStreamSynchronize(c->stream), "capture");
    CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = launch_all(c, dt, n_steps, cfg);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return cuda_fail(c, e != cudaSuccess ? e : e2, "graph capture");
    }
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { c->graph = nullptr; return cuda_fail(c, e, "graph instantiate"); }
    c->graph_steps = n_steps;
    c->graph_dt = dt;
    c->last = cfg;
    return FEDFEM_OK;
}

int fedfem_replay_graph(fedfem_ctx* c) {
    if (!c) return FEDFEM_E_ARG;
    if (!c->graph || !c->inited) return fail(c, FEDFEM_E_STATE, "capture a graph (after init) first");
    CU(cudaSetDevice(c->device), "set device");
    CU(cudaGraphLaunch(c->graph, c->stream), "graph launch");
    c->steps_issued += c->graph_steps;
    c->sim_time += c->graph_dt * (double)c->graph_steps;
    return FEDFEM_OK;
}

int fedfem_sync(fedfem_ctx* c, int64_t* steps_done) {
    ApiRange nvtx_range("fedfem_sync");
    if (!c) return FEDFEM_E_ARG;
    if (!c->inited) return fail(c, FEDFEM_E_STATE, "init first");
    CU(cudaSetDevice(c->device), "set device");
    CU(cudaStreamSynchronize(c->stream), "sync");
    DevStatus h{};
    CU(cudaMemcpy(&h, c->st, sizeof(h), cudaMemcpyDeviceToHost), "status read");
    int64_t done = c->steps_issued;
    int rc = FEDFEM_OK;
    if (h.flags & STATUS_TIMEOUT) {
        done = h.steps_done;
        rc = fail(c, FEDFEM_E_TIMEOUT, "a grid barrier wait gave up after its spin limit");
    } else if (h.flags & STATUS_RANGE) {
        done = h.fail_step + 1;
        const int64_t node = (h.fail_node >= 0 && h.fail_node < c->N) ? c->L.node_of[h.fail_node] : -1;
        rc = fail(c, FEDFEM_E_RANGE, "temperature left [T_lo, T_hi] or became NaN at step " +
                                         std::to_string(h.fail_step) + ", node " + std::to_string(node));
    }
    if (steps_done) *steps_done = done;
    return rc;
}

int fedfem_read_temperature_device(fedfem_ctx* c, double* out_dev) {
    ApiRange nvtx_range("fedfem_read_temperature_device");
    if (!c || !out_dev) return fail(c, FEDFEM_E_ARG, "null output");
    if (!c->inited) return fail(c, FEDFEM_E_STATE, "init first");
    CU(cudaSetDevice(c->device), "set device");
    CU(launch_read_state(c->precision, c->n_lanes, 0, c->N, c->node_of, c->T, c->Tlo, out_dev, c->stream),
       "read kernel");
    CU(cudaStreamSynchronize(c->stream), "read");
    return FEDFEM_OK;
}

int fedfem_read_temperature_lane(fedfem_ctx* c, int lane, double* out) {
    if (!c || !out) return fail(c, FEDFEM_E_ARG, "null output");
    if (!c->inited) return fail(c, FEDFEM_E_STATE, "init first");
    if (lane < 0 || lane >= c->n_lanes) return fail(c, FEDFEM_E_ARG, "lane out of range");
    CU(cudaSetDevice(c->device), "set device");
    CU(launch_read_state(c->precision, c->n_lanes, lane, c->N, c->node_of, c->T, c->Tlo, c->io, c->stream),
       "read kernel");
    CU(cudaMemcpyAsync(out, c->io, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream), "copy out");
    CU(cudaStreamSynchronize(c->stream), "read");
    return FEDFEM_OK;
}

int fedfem_read_temperature(fedfem_ctx* c, double* out) {
    ApiRange nvtx_range("fedfem_read_temperature");
    if (!c || !out) return fail(c, FEDFEM_E_ARG, "null output");
    if (!c->inited) return fail(c, FEDFEM_E_STATE, "init first");
    CU(cudaSetDevice(c->device), "set device");
    CU(launch_read_state(c->precision, c->n_lanes, 0, c->N, c->node_of, c->T, c->Tlo, c->io, c->stream),
       "read kernel");
    CU(cudaMemcpyAsync(out, c->io, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream), "copy out");
    CU(cudaStreamSynchronize(c->stream), "read");
    return FEDFEM_OK;
}

struct StateHeader {
    uint64_t magic;
    int32_t version, precision;
    int64_t N, E;
    int32_t order, nv;
    int64_t steps_done;
    double sim_time;
    uint64_t payload;
};
static const uint64_t kMagic = 0x5453464d45464546ULL;   // "FEFEMFST"

int fedfem_get_state(fedfem_ctx* c, void* buf, size_t* bytes) {
    ApiRange nvtx_range("fedfem_get_state");
    if (!c || !bytes) return fail(c, FEDFEM_E_ARG, "null size pointer");
    if (!c->inited) return fail(c, FEDFEM_E_STATE, "init first");
    const size_t tb = (c->precision == FEDFEM_FP64 ? sizeof(double) : sizeof(float)) * c->N * c->n_lanes;
    const size_t lb = (c->precision == FEDFEM_FP64 ? 0 : sizeof(float) * c->N * c->n_lanes);
    const size_t db = c->dose ? sizeof(double) * c->L.N_free * c->n_lanes : 0;
    const size_t need = sizeof(StateHeader) + tb + lb + db;
    if (!buf) { *bytes = need; return FEDFEM_OK; }
    if (*bytes < need) return fail(c, FEDFEM_E_ARG, "state buffer too small");
    int64_t done = 0;
    int rc = fedfem_sync(c, &done);
    if (rc) return rc;
    StateHeader h{kMagic, 1, c->precision, c->N, c->E, c->order, c->nv, done, c->sim_time, tb + lb + db};
    std::memcpy(buf, &h, sizeof(h));
    char* p = (char*)buf + sizeof(h);
    CU(cudaMemcpy(p, c->T, tb, cudaMemcpyDeviceToHost), "state copy");
    if (lb) CU(cudaMemcpy(p + tb, c->Tlo, lb, cudaMemcpyDeviceToHost), "state copy");
    if (db) CU(cudaMemcpy(p + tb + lb, c->dose, db, cudaMemcpyDeviceToHost), "state copy");
    *bytes = need;
    return FEDFEM_OK;
}

int fedfem_set_state(fedfem_ctx* c, const void* buf, size_t bytes) {
    ApiRange nvtx_range("fedfem_set_state");
    if (!c || !buf) return fail(c, FEDFEM_E_ARG, "null state");
    if (!c->pre) return fail(c, FEDFEM_E_STATE, "precompute first");
    if (bytes < sizeof(StateHeader)) return fail(c, FEDFEM_E_ARG, "state too short");
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    const size_t tb = (c->precision == FEDFEM_FP64 ? sizeof(double) : sizeof(float)) * c->N * c->n_lanes;
    const size_t lb = (c->precision == FEDFEM_FP64 ? 0 : sizeof(float) * c->N * c->n_lanes);
    const size_t db = c->dose ? sizeof(double) * c->L.N_free * c->n_lanes : 0;
    if (h.magic != kMagic || h.version != 1 || h.precision != c->precision || h.N != c->N || h.E != c->E ||
        h.order != c->order || h.nv != c->nv || h.payload != tb + lb + db || bytes < sizeof(h) + tb + lb + db)
        return fail(c, FEDFEM_E_ARG, "state does not match this context");
    CU(cudaSetDevice(c->device), "set device");
    const char* p = (const char*)buf + sizeof(h);
    CU(cudaMemcpy(c->T, p, tb, cudaMemcpyHostToDevice), "state copy");
    if (lb) CU(cudaMemcpy(c->Tlo, p + tb, lb, cudaMemcpyHostToDevice), "state copy");
    if (db) CU(cudaMemcpy(c->dose, p + tb + lb, db, cudaMemcpyHostToDevice), "state copy");
    if (int m = mirror_T(c)) return m;
    int r = reset_status(c);
    if (r) return r;
    c->inited = true;
    c->steps_issued = h.steps_done;
    c->sim_time = h.sim_time;
    return FEDFEM_OK;
}

int fedfem_get_info(fedfem_ctx* c, fedfem_info* info) {
    if (!c || !info) return fail(c, FEDFEM_E_ARG, "null info");
    if (!c->pre) return fail(c, FEDFEM_E_STATE, "precompute first");
    std::memset(info, 0, sizeof(*info));
    const Layout& L = c->L;
    info->n_nodes = c->N; info->n_elems = c->E; info->n_free = L.N_free;
    info->n_dirichlet = c->N - L.N_free; info->n_convective = L.N_free - L.N_plain;
    info->elem_type = c->nv; info->precision = c->precision; info->order = c->order;
    info->dt_cr = c->dt_cr; info->lambda_max_ref = c->lambda; info->td_scale = c->td_scale;
    info->lanczos_iterations = c->lz_iters;
    info->steps_done = c->steps_issued;
    info->sim_time = c->sim_time;
    info->device_bytes = c->dev_bytes;
    const int64_t R = c->precision == FEDFEM_FP64 ? 8 : 4;
    const int64_t node_state = c->precision == FEDFEM_FP32_KAHAN ? 4 * R : 2 * R;   // T (+lo) read+write
    const int64_t E = c->E, NF = L.N_free, NC = L.N_free - L.N_plain;
    const int64_t NL = c->n_lanes;   // lanes share V, hA and the element data
    const int64_t nm = (c->A28_64 || c->A28_32) ? 28 : (c->W64 || c->W32) ? 18 : 6;   // element matrix values
    info->algorithmic_bytes_per_step = E * (4 * c->nv + nm * R) + NF * (NL * (node_state + R) + R) + NC * R;
    if (c->matrix_free)   // coordinates (each node once) instead of the element matrices
        info->algorithmic_bytes_per_step += 12 * c->N - E * nm * R;
    // a source schedule reads the source part of Q too; the dose (8 bytes per node) is read and written
    const int64_t extra = (c->sched_f.empty() ? 0 : NF * NL * R) + (c->dose ? NF * 16 : 0) +
                          (c->n_cq > 0 ? NF * 4 * R + E : 0);   // regions: node coefficients, element ids
    info->algorithmic_bytes_per_step += extra;
    // two-phase / persistent model: + slot write and read, gather ids, their slice offsets, T gathered once
    info->bytes_per_step = info->algorithmic_bytes_per_step + E * c->nv * 2 * R + (int64_t)L.sell_ids.size() * 4 +
                           (int64_t)L.sell_off.size() * 4;
    if (tile_kind(c) > 0 || c->tile.kernel == FEDFEM_KERNEL_TILED) {
      if (c->tiles_ok) {
        const Tiles& t = c->tiles_host;
        // every packed block once, halo values, owned T read; then T written, lo read+write, V, Q, hA
        const int64_t node_rest = NF * (NL * (node_state - R + R) + R) + NC * R;
        info->bytes_per_step =
            c->t_block_bytes + (int64_t)t.halo.size() * R * NL + NF * R * NL + node_rest + extra;
      }
    }
    info->sm_count = c->sm_count;
    info->grid_blocks = c->last.grid_used;
    info->block_threads = tile_kind(c) > 0 ? staged_threads(c) : 256;
    info->kernel = c->tile.kernel;
    info->tile_nodes = c->tiles_ok ? c->tiles_B : 0;
    info->lanes = c->n_lanes;
    return FEDFEM_OK;
}

}  // extern "C"
