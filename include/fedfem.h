/*
 * fedfem.h -- C ABI of the GB300 FED-FEM Pennes bio-heat library.
 *
 * The library advances the Pennes bio-heat equation (Eq. 1, constant
 * properties; Eq. 2, temperature-dependent properties) on an unstructured mesh
 * of one-point hexahedra (Eq. 14) or linear tetrahedra (Eq. 15) with the fast
 * explicit dynamics scheme of Zhang & Chauhan (arXiv:1909.05098): forward Euler
 * in time (Eq. 6), element-level conduction loads F_e = k_e A_e T_e from
 * pre-computed element matrices (Eq. 12-17, k_e by Eq. 13), lumped capacitance
 * and perfusion (Section 2.3.4-2.3.5) and the nodal update of Eq. 19, below the
 * critical step of Eq. 9.  Call order follows Algorithm 1:
 *
 *   fedfem_create -> fedfem_set_* (load mesh and boundary conditions, Alg. 1
 *   pre-computation) -> fedfem_precompute (A_e, lumped C, K_b, Q_b, dt_cr)
 *   -> fedfem_init (T0, Alg. 1 initialisation) -> fedfem_step(n) (the time
 *   loop) -> fedfem_sync / fedfem_read_temperature.
 *
 * Conventions for every call:
 *  - The return value is a fedfem_status; 0 (FEDFEM_OK) is success.  On any
 *    other value fedfem_last_error() holds a one-line message and the context
 *    is unchanged unless stated.
 *  - Array inputs are host pointers and are COPIED before the call returns;
 *    the caller keeps ownership.  Output arrays are caller-allocated host
 *    buffers, except in the *_device calls, which take device pointers on the
 *    context's device.
 *  - Node and element indices at this boundary are 0-based and always refer
 *    to the caller's input order; the library's internal reordering is never
 *    visible.
 *  - Units are SI, temperatures in degrees Celsius; w_b is the perfusion rate
 *    in kg/(m^3 s) as in Eq. 1.
 *  - All device work is issued on the context's CUDA stream.  fedfem_step is
 *    asynchronous; every other call that touches the device returns after its
 *    work has completed.  Device buffers passed to the *_device calls must be
 *    ready on that stream: when they were written on another stream, the
 *    caller synchronizes first.
 *  - A context is used by one host thread at a time.
 *  - The library owns all device memory it allocates and frees it in
 *    fedfem_destroy.
 */
#ifndef FEDFEM_H
#define FEDFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fedfem_ctx fedfem_ctx;

typedef enum {
    FEDFEM_OK = 0,
    FEDFEM_E_ARG = -1,          /* invalid argument (null pointer, bad size, bad index, NaN) */
    FEDFEM_E_MESH = -2,         /* element with det J <= 0, or a node used by no element */
    FEDFEM_E_STATE = -3,        /* call out of order (e.g. step before init) */
    FEDFEM_E_UNSTABLE_DT = -4,  /* dt >= the critical step of Eq. 9 */
    FEDFEM_E_RANGE = -5,        /* T left [T_lo, T_hi] or became NaN; rho c or k not positive on the range */
    FEDFEM_E_TIMEOUT = -6,      /* a bounded device wait (grid barrier) gave up */
    FEDFEM_E_CUDA = -7,         /* CUDA runtime error */
    FEDFEM_E_OOM = -8,          /* device allocation failed */
    FEDFEM_E_UNSUPPORTED = -9   /* option not available for this element type / precision */
} fedfem_status;

enum { FEDFEM_TET4 = 4, FEDFEM_HEX8 = 8 };

/* Arithmetic of the time loop.  Pre-computation is always FP64. */
enum {
    FEDFEM_FP64 = 0,        /* FP64 state and arithmetic */
    FEDFEM_FP32_KAHAN = 1,  /* FP32 loads and arithmetic, state kept as an FP32 pair
                               (hi, lo) updated by compensated (Kahan) summation */
    FEDFEM_FP32_PLAIN = 2   /* FP32 state without compensation (a negative control) */
};

/* Internal element order; the node order follows by first touch. */
enum { FEDFEM_ORDER_INPUT = 0, FEDFEM_ORDER_MORTON = 1, FEDFEM_ORDER_RCM = 2 };

/* Time-loop kernel family.  All give bit-identical results. */
enum {
    FEDFEM_KERNEL_TWO_PHASE = 0,   /* one element launch and one node launch per step */
    FEDFEM_KERNEL_PERSISTENT = 1,  /* one cooperative launch for n steps, bounded grid barriers */
    FEDFEM_KERNEL_TILED = 2,       /* persistent, node tiles: T and element loads in shared memory, no global slots */
    FEDFEM_KERNEL_TILED_STAGED = 3,/* as TILED, each tile's constant data streamed into shared memory by bulk copies */
    FEDFEM_KERNEL_TILED_REP = 4    /* as TILED_STAGED, with the tile's owned temperatures copied into one row per
                                      rank, so that one 16-bit offset per element corner addresses both its
                                      temperature and its load slot; one lane; at most one owned node per thread */
};

/* Linear laws p(T) = p0 + dp (T - T_ref) for density rho [kg/m^3], specific
 * heat c [J/(kg K)] and conductivity k [W/(m K)] (Eq. 2; Section 3.1.6 uses
 * this linear form between two temperatures).  Constant properties: dp = 0. */
typedef struct { double T_ref, rho0, drho, c0, dc, k0, dk; } fedfem_material;

/* Perfusion rate w_b [kg/(m^3 s)], blood specific heat c_b [J/(kg K)],
 * arterial temperature T_a [degC] and metabolic heat Q_m [W/m^3] (Eq. 1). */
typedef struct { double w_b, c_b, T_a, Q_m; } fedfem_perfusion;

/* Launch knobs (chosen by the autotuner).  Results do not depend on them. */
typedef struct {
    int kernel;        /* FEDFEM_KERNEL_* */
    int block;         /* threads per block: 64..1024, multiple of 32 (0 = default); the
                          staged tiled kernel is built for 256, 512 (default) and 1024, the
                          replicated-row kernel for 128, 256 and 512 (default 512 for hex8 and
                          256 for tet4, halved in FP64) */
    int tile_nodes;    /* TILED: owned nodes per tile, multiple of 8 (0 = default: the library
                          picks a size near 512 (hex) / 256 (tet), smaller when such tiles
                          do not fit in shared memory, that gives every resident block the
                          same number of tiles) */
    int blocks_per_sm; /* PERSISTENT/TILED: resident blocks per SM (0 = occupancy maximum) */
} fedfem_tile;

/* Read-only facts about a pre-computed context. */
typedef struct {
    int64_t n_nodes, n_elems, n_free, n_dirichlet, n_convective;
    int elem_type, precision, order;
    double dt_cr;              /* critical step of Eq. 9 over [T_lo, T_hi] */
    double lambda_max_ref;     /* largest eigenvalue at reference properties */
    double td_scale;           /* factor applied for temperature-dependent laws */
    double dt_element_bound;   /* conservative step from element eigenvalue bounds */
    int lanczos_iterations;
    int64_t steps_done;        /* steps completed since fedfem_init */
    double sim_time;           /* simulated seconds since fedfem_init */
    int64_t device_bytes;      /* device memory held by the context */
    int64_t bytes_per_step;    /* bytes the chosen kernel reads and writes per time step (model) */
    int64_t algorithmic_bytes_per_step; /* minimum bytes any step must move (fused model) */
    int sm_count, grid_blocks, block_threads;
    int kernel;                /* FEDFEM_KERNEL_* in use */
    int tile_nodes;            /* owned nodes per tile of the tiled kernels (0 if none built) */
    int lanes;                 /* scenario lanes (1 or 4) */
} fedfem_info;

/* Create a context on CUDA device `device`.  `precision` is a FEDFEM_FP*
 * value.  `cuda_stream` is a cudaStream_t to issue work on, or NULL for a
 * stream owned by the context.  *out receives the context (NULL on error). */
int fedfem_create(fedfem_ctx** out, int device, int precision, void* cuda_stream);

/* Mesh (the input of Algorithm 1).  xyz: n_nodes x 3 doubles,
 * metres, row-major.  conn: n_elems x elem_type 0-based node ids, row-major.
 * hex8 (Eq. 14): corners at natural coordinates (-1,-1,-1), (1,-1,-1),
 * (1,1,-1), (-1,1,-1), then the same four at zeta = +1, det J > 0.
 * tet4 (Eq. 15): det[x1-x0, x2-x0, x3-x0] > 0.  Every node must be used by
 * an element.  Replaces any earlier mesh and clears boundary conditions,
 * sources and the pre-computation. */
int fedfem_set_mesh(fedfem_ctx* ctx, int elem_type, int64_t n_nodes, const double* xyz,
                    int64_t n_elems, const int32_t* conn);

#define FEDFEM_HEX_ONE_POINT 0
#define FEDFEM_HEX_FULL 1
/* Integration rule of hex8 elements: FEDFEM_HEX_ONE_POINT (default; Eq. 14,
 * J at the centre, V_e = 8 det J, the factored 6-value element matrix) or
 * FEDFEM_HEX_FULL (2 x 2 x 2 Gauss points: A_e = sum of det J B^T B, exact for
 * the trilinear element, no hourglass modes, V_e = sum of det J; an element
 * with det J <= 0 at any point is E_MESH).  The full rule stores the 28
 * off-diagonal entries per element (the diagonal follows from the zero row
 * sums) and runs on the two-phase and persistent kernels (the tiled kernels
 * refuse it with E_UNSUPPORTED at the next step); the critical step uses the
 * full matrices.  Ignored for tet4.  E_ARG for another rule.  Takes effect at
 * the next fedfem_precompute. */
int fedfem_set_hex_integration(fedfem_ctx* ctx, int rule);

/* Hourglass control of the one-point hexahedron (Section 2.3.3 keeps Eq. 14's
 * single point and leaves the remedy for its zero-energy modes to another
 * work).  eps > 0 adds to each one-point element matrix
 *   c sum_a gamma_a gamma_a^T,  c = eps trace(A_1pt) / 32,
 * where gamma_a = h_a - sum_i (h_a . x_i) b_i are the four hourglass patterns
 * h_a (products of the corner signs s_x s_y, s_y s_z, s_z s_x, s_x s_y s_z)
 * made blind to linear fields (x_i: the corners' i-th coordinates, b_i: the
 * i-th row of Eq. 14's B).  Linear fields keep exactly the one-point energy;
 * on a parallelepiped the added matrix carries eps times the trace of the
 * one-point one.  Each element stores 12 weights w_ad (gamma_a = h_a -
 * sum_d w_ad s_d), computed in FP64 with the geometry; the critical step
 * includes the added term.  eps = 0 (default) turns it off.  Ignored for
 * tet4; E_UNSUPPORTED at fedfem_precompute with the full rule.  Takes effect
 * at the next fedfem_precompute.  E_ARG for eps < 0 or not finite. */
int fedfem_set_hourglass_control(fedfem_ctx* ctx, double eps);

/* Matrix-free element geometry for tet4 meshes with FP32 state (the pre-
 * computation of Eq. 15-16 moved into the time loop; the paper pre-computes
 * A_e once, its aim (v) in the introduction).  on = 1: the tiled kernels
 * (FEDFEM_KERNEL_TILED, FEDFEM_KERNEL_TILED_STAGED) read each tile's node
 * coordinates (FP32, relative to the centre of the mesh's bounding box,
 * rounded once from the FP64 input) instead of the 6 matrix values of every
 * element, and
 * recompute M_e = V_tet E^-1 E^-T from the corners of each element in FP32
 * every step: 24 bytes fewer per element and step, about 60 more arithmetic
 * operations.  Results agree with the stored-matrix kernels to rounding (not
 * bit for bit) and are the same bits for both kernels and every tile size;
 * the critical step is unchanged (pre-computed in FP64).  Other
 * kernels, FP64 state and hex8 meshes give E_UNSUPPORTED (at the next step
 * for kernels and precision; at once for a hex8 mesh already set).  on = 0
 * (default): stored matrices. */
int fedfem_set_matrix_free(fedfem_ctx* ctx, int on);

/* Element order used internally (FEDFEM_ORDER_*; default MORTON). */
int fedfem_set_order(fedfem_ctx* ctx, int order);

/* Homogeneous tissue laws (Eq. 2), linear in T.  Clears any table set by
 * fedfem_set_material_table. */
int fedfem_set_material(fedfem_ctx* ctx, const fedfem_material* m);

/* Tabulated laws: Section 3.1.6 gives rho, c and k at two temperatures (a
 * two-point table, the linear laws above); n points give piecewise-linear
 * laws.  T: n strictly increasing temperatures (degC); rho, c, k: the values
 * at each (kg/m^3, J/(kg K), W/(m K)), n in 2..8.  Inside [T[0], T[n-1]]
 * each property is linear on the interval that holds T; below and above the
 * table the first and last intervals extend linearly.  The first point is
 * the reference state of the critical step (k0 = k[0], rho0 c0 = rho[0]
 * c[0]), which fedfem_precompute bounds over [T_lo, T_hi] as for linear
 * laws; E_RANGE there if rho c or k is not positive on that range.
 * Replaces the material and any regions (a later fedfem_set_material or
 * fedfem_set_regions replaces the table).
 * Host arrays, copied; E_ARG for non-finite values, T not increasing, or
 * rho[0], c[0], k[0] not positive.  Steps of a context with a table run the
 * kernel builds that hold the source-schedule and dose paths.
 * (fedfem_step_static, which has no context, takes linear laws only.) */
int fedfem_set_material_table(fedfem_ctx* ctx, int n, const double* T, const double* rho, const double* c,
                              const double* k);

/* Heterogeneous tissue (the finite element form lets properties vary from
 * element to element, Section 1): element e (input order) belongs to region
 * region[e] in 0..n-1, n in 1..16, with region r's linear laws mats[r] (as in
 * fedfem_set_material) and perfusion perf[r] (w_b, c_b and Q_m; T_a stays
 * that of fedfem_set_perfusion).  k_e (Eq. 13) averages the element's own k
 * law over its nodes; the lumped C_i, the perfusion beta_i and the metabolic
 * heat of node i sum the shares V_e / nv of its elements times their
 * region's rho(T_i) c(T_i), w_b c_b and Q_m.  The critical step
 * (fedfem_precompute) is computed for the first region's k0 and rho0 c0
 * everywhere with the largest w_b c_b of any region, then scaled by
 * max(1, max k / k0) * max(1, rho0 c0 / min rho c) over every region and
 * [T_lo, T_hi]: an upper bound of every region's eigenvalue, so the step is
 * safe but may be smaller than that of the exact heterogeneous operator.
 * Requires a mesh (E_STATE); E_ARG for n out of range, a region id out of
 * range, or a material or perfusion value fedfem_set_material /
 * fedfem_set_perfusion would refuse.  Replaces the material and any table;
 * a later fedfem_set_material, fedfem_set_material_table or fedfem_set_mesh
 * removes the regions.  Host arrays, copied.  Steps of a context with regions
 * run the kernel builds that hold the source-schedule and dose paths.
 * (fedfem_step_static takes one material.) */
int fedfem_set_regions(fedfem_ctx* ctx, int n, const fedfem_material* mats, const fedfem_perfusion* perf,
                       const int32_t* region);

#define FEDFEM_LUMP_ELEMENT 0
#define FEDFEM_LUMP_UNIFORM 1
/* How perfusion and metabolic heat reach the nodes: FEDFEM_LUMP_ELEMENT
 * (default) lumps them like C, beta_i = w_b c_b V_i and Q_m V_i with V_i the
 * sum of the element shares V_e / nv (Section 2.3.5); FEDFEM_LUMP_UNIFORM
 * gives every node the same share V / N of the mesh volume V over its N nodes
 * (the form of the paper's verification runs, Sections 3.1.3-3.1.4: a film
 * w_b c_b V / N and a heat flow Q_m V / N per node).  C stays lumped by
 * element shares.  The uniform form runs on the kernel builds that hold the
 * source-schedule and dose paths; the critical step takes its exact per-node
 * perfusion.  With element groups (several meshes in one context) V and N
 * are those of the whole context, not of each group.  E_ARG for another
 * mode; E_UNSUPPORTED at fedfem_precompute with regions or a property table.
 * Takes effect at the next fedfem_precompute. */
int fedfem_set_lumping(fedfem_ctx* ctx, int mode);

/* Perfusion and metabolism (Eq. 1); K_b and Q_b are lumped (Section 2.3.5). */
int fedfem_set_perfusion(fedfem_ctx* ctx, const fedfem_perfusion* p);

/* Regional source density Q_r at every node [W/m^3] (Eq. 1), n_nodes values,
 * or NULL to clear.  Adds to any Gaussian sources. */
int fedfem_set_source(fedfem_ctx* ctx, const double* q_r);

/* Add Q_r(x) = peak exp(-|x - x0|^2 / (2 sigma^2)) [W/m^3]. */
int fedfem_add_gaussian_source(fedfem_ctx* ctx, const double x0[3], double sigma, double peak);

/* Remove all Gaussian sources. */
int fedfem_clear_sources(fedfem_ctx* ctx);

/* Essential boundary (Eq. 3): n nodes held at T (degC) from fedfem_init on.
 * A node listed twice takes its last value.  Dirichlet wins over every other
 * condition on the same node. */
int fedfem_set_dirichlet(fedfem_ctx* ctx, int64_t n, const int32_t* nodes, const double* T);

/* Film condition on boundary faces: q = h (T_inf - T), lumped to nodes with
 * each face's area split equally over its nverts (3 or 4) nodes, explicit at
 * the current T.  faces: n_faces x nverts node ids. */
int fedfem_set_convective(fedfem_ctx* ctx, int64_t n_faces, int nverts, const int32_t* faces,
                          double h, double T_inf);

/* Concentrated nodal heat flows q [W] (heat-flux boundary of Eq. 4 as the
 * paper applies it).  Repeated nodes add. */
int fedfem_set_nodal_flux(fedfem_ctx* ctx, int64_t n, const int32_t* nodes, const double* q_W);

/* Time-varying regional sources: Algorithm 1 updates the loads after every
 * step; Section 3.1.5 heats for 3 s and then relaxes with the sources
 * removed.  The regional source part of each node's load (Gaussian sources
 * and fedfem_set_source densities, every lane) is multiplied by factor[k]
 * for steps whose start time t lies in [t_end[k-1], t_end[k]) (t_end[-1] =
 * -inf); after t_end[n-1] the last factor holds.  Metabolic heat and nodal
 * flows stay constant.  t is the simulated time since fedfem_init.  n = 0
 * removes the schedule.  At most 8 segments; t_end strictly increasing
 * (E_ARG otherwise).  Host arrays, copied.  Takes effect at the next
 * fedfem_precompute (call order: set_* -> precompute).  A context with a
 * schedule cannot capture a CUDA graph (E_UNSUPPORTED): the start time of
 * each call is a launch argument. */
int fedfem_set_source_schedule(fedfem_ctx* ctx, int n, const double* t_end, const double* factor);

/* Thermal dose (the treatment-planning use Section 5 names; the paper gives
 * no formula): cumulative equivalent minutes at 43 degC of Sapareto and
 * Dewey, CEM43 += (dt / 60) R^(43 - T) with R = 1/2 at or above 43 degC and
 * 1/4 below, T the node's temperature at the start of each step (the hi part
 * in FP32+Kahan), accumulated inside the node update of every kernel (every
 * scenario lane separately): in FP64 with FP64 state, as a compensated FP32
 * pair (about 2^-48 relative) with FP32 state; the power is evaluated in the
 * state's precision.  on != 0 enables it from the next fedfem_precompute;
 * fedfem_init resets it to 0; checkpoints carry it. */
int fedfem_enable_dose(fedfem_ctx* ctx, int on);

#define FEDFEM_DOSE_CEM43 0
#define FEDFEM_DOSE_ARRHENIUS 1
/* The dose model (default CEM43).  FEDFEM_DOSE_ARRHENIUS: the thermal damage
 * integral of Henriques and Moritz, Omega += dt A exp(-Ea / (R T_K)), A the
 * frequency factor (1/s), Ea the activation energy (J/mol), R = 8.314462618
 * J/(mol K), T_K = T + 273.15, at each step's start temperature, summed as
 * the CEM43 dose is (the exponential in the state's precision); fedfem_read_dose then
 * returns Omega (dimensionless; 1 is the usual coagulation threshold).
 * FEDFEM_DOSE_CEM43 ignores A and Ea.  E_ARG for another model or A, Ea not
 * finite and positive.  Takes effect at the next fedfem_step; fedfem_init
 * resets the accumulated value, so set it before fedfem_init.  A graph
 * captured before the change keeps the model it was captured with: capture
 * again after changing it. */
int fedfem_set_dose_model(fedfem_ctx* ctx, int model, double A, double Ea);
/* CEM43 in minutes (or Omega, see fedfem_set_dose_model), n_nodes doubles in
 * input node order (caller-owned host buffer).  Dirichlet nodes report their fixed temperature held for the
 * elapsed simulated time.  Waits for the context's stream.  E_STATE if the
 * dose is not enabled or before fedfem_init. */
int fedfem_read_dose(fedfem_ctx* ctx, double* out);
/* The same for one scenario lane (0 .. lanes-1; E_ARG otherwise). */
int fedfem_read_dose_lane(fedfem_ctx* ctx, int lane, double* out);

/* Pre-computation (the first stage of Algorithm 1) in FP64 on the GPU: element
 * geometry and A_e (Eq. 16), lumped volumes, perfusion and source loads, face
 * areas, and the critical step of Eq. 9 for properties anywhere in
 * [T_lo, T_hi].  Writes dt_cr to *dt_cr_out (may be NULL).  Returns
 * FEDFEM_E_MESH on an element with det J <= 0, FEDFEM_E_RANGE if rho c or k
 * is not positive on the range. */
int fedfem_precompute(fedfem_ctx* ctx, double T_lo, double T_hi, double* dt_cr_out);

/* Initial field (the initialisation of Algorithm 1): T0 has n_nodes values in input order,
 * or is NULL for T0_uniform everywhere.  Dirichlet nodes take their values.
 * Clears the device status and the step counter.  A non-finite value gives
 * FEDFEM_E_ARG and leaves the state as it was (the values are checked on the
 * device after the copy; the call returns once the check is read back). */
int fedfem_init(fedfem_ctx* ctx, const double* T0, double T0_uniform);

/* As fedfem_init, T0 a device pointer to n_nodes doubles (input order); the
 * same check. */
int fedfem_init_device(fedfem_ctx* ctx, const double* T0_dev);

/* Advance n_steps explicit steps of size dt (Algorithm 1's time loop),
 * asynchronously.  FEDFEM_E_UNSTABLE_DT if dt >= dt_cr.  A range violation
 * or barrier timeout stops the loop on the device and is reported by
 * fedfem_sync. */
int fedfem_step(fedfem_ctx* ctx, double dt, int64_t n_steps);

/* Wait for the context's stream; *steps_done (may be NULL) receives the steps
 * completed since init.  Returns FEDFEM_E_RANGE or FEDFEM_E_TIMEOUT if the
 * device recorded one (sticky until the next init or set_state). */
int fedfem_sync(fedfem_ctx* ctx, int64_t* steps_done);

/* Nodal temperatures (n_nodes doubles, input order).  FP32 states return
 * (double)hi + (double)lo. */
int fedfem_read_temperature(fedfem_ctx* ctx, double* out);

/* As fedfem_read_temperature into a device buffer of n_nodes doubles. */
int fedfem_read_temperature_device(fedfem_ctx* ctx, double* out_dev);

/* Checkpoint: with buf == NULL, *bytes receives the size needed.  Otherwise
 * the state (temperature pair, step counter, simulated time) is written to
 * buf (capacity *bytes).  Restoring it with fedfem_set_state into a context
 * with the same mesh, options and precision resumes bit-identically. */
int fedfem_get_state(fedfem_ctx* ctx, void* buf, size_t* bytes);
int fedfem_set_state(fedfem_ctx* ctx, const void* buf, size_t bytes);

/* ---- Batched planning: many independent problems in one launch ----------
 * The paper's future work (Section 5) is treatment planning, i.e. many runs of
 * the same method.  Two mechanisms let one context step many runs at once:
 *
 * Scenario lanes: up to 4 problems that share the mesh, materials, perfusion
 * and boundary conditions but differ in their regional sources.  Their
 * temperatures are stored interleaved (4 floats per node), so each element
 * matrix and connectivity entry is read once for all lanes.  Each lane's
 * arithmetic is exactly that of a single run (bit-identical results).  FP32
 * precisions and the tiled kernels only; all lanes start from the same T0.
 * Sources added with fedfem_add_gaussian_source / fedfem_set_source apply to
 * every lane; the *_lane calls add to one lane.  Call before precompute. */
int fedfem_set_lanes(fedfem_ctx* ctx, int n_lanes);   /* 1 (default) or 4 */
/* group >= 0 restricts the source to the nodes of that element group (see
 * fedfem_set_element_groups); -1: every node. */
int fedfem_add_gaussian_source_lane(fedfem_ctx* ctx, int lane, int group, const double x0[3], double sigma,
                                    double peak);
int fedfem_set_source_lane(fedfem_ctx* ctx, int lane, const double* q_r);
/* Temperatures of one lane (n_nodes doubles, input order). */
int fedfem_read_temperature_lane(fedfem_ctx* ctx, int lane, double* out);
/* Initial field per lane from device memory: n_lanes x n_nodes doubles
 * (lane-major, input order); Dirichlet nodes take their values.  As
 * fedfem_init otherwise. */
int fedfem_init_lanes_device(fedfem_ctx* ctx, const double* T0_dev);
/* All lanes' temperatures into device memory, n_lanes x n_nodes doubles. */
int fedfem_read_lanes_device(fedfem_ctx* ctx, double* out_dev);

/* Element groups: several independent meshes given as one mesh (their node
 * sets disjoint); group[e] (n_elems values) keeps each mesh's elements
 * together in the internal order, so tiles never mix meshes.  NULL clears.
 * The critical step is then the smallest over the meshes. */
int fedfem_set_element_groups(fedfem_ctx* ctx, const int32_t* group);

/* Record one fedfem_step(dt, n_steps) as a CUDA graph on the context's
 * stream, then launch it with fedfem_replay_graph (asynchronous, as
 * fedfem_step).  Tiles are planned before the capture.  Step indices in range
 * errors count from the capture.  A new capture replaces the old graph; any
 * set_* call drops it. */
int fedfem_capture_graph(fedfem_ctx* ctx, double dt, int64_t n_steps);
int fedfem_replay_graph(fedfem_ctx* ctx);

/* Launch knobs; see fedfem_tile.  May be called after precompute. */
int fedfem_set_tile(fedfem_ctx* ctx, const fedfem_tile* tile);

/* Facts about the context (after precompute). */
int fedfem_get_info(fedfem_ctx* ctx, fedfem_info* info);

/* Last error message of this context ("" if none).  Valid until the next call. */
const char* fedfem_last_error(const fedfem_ctx* ctx);

/* Free everything the context holds.  NULL is allowed. */
void fedfem_destroy(fedfem_ctx* ctx);

/* Library version string. */
const char* fedfem_version(void);

/* Measurement helper (the paper has no counterpart): launches `blocks` x
 * `threads` threads that each run `iterations` rounds of eight independent
 * FP64 fused multiply-adds, 16 * iterations * blocks * threads FLOPs in all,
 * asynchronously on `stream`; timing it with CUDA events gives the FP64 rate
 * the FP64 time-loop kernels are bound by.  sink_dev: device array of at
 * least `blocks` doubles (written only in a case that never occurs).
 * FEDFEM_E_ARG for a bad size, FEDFEM_E_CUDA when the launch fails. */
int fedfem_fp64_fma_loop(long long iterations, int blocks, int threads, double* sink_dev, void* stream);

/* Sizes of the layout fedfem_plan_layout returns. */
typedef struct {
    int64_t n_nodes, n_elems;
    int64_t n_plain, n_free;      /* node ranges: [0,n_plain) plain free, [n_plain,n_free) film, rest Dirichlet */
    int64_t n_slices, n_gather;   /* sliced-ELL gather over the free nodes */
    int max_degree;
    int tile_nodes;               /* owned nodes per tile (0: no tiles requested) */
    int64_t n_tiles, n_tile_elems, n_halo;
    int max_tile_local, max_tile_elems;
    int max_tile_degree;          /* most elements at one owned node of a tile */
    int tile_rank_shift;          /* tile_lconn entry = local id | rank << tile_rank_shift */
} fedfem_layout_info;

/* Host-only planning (no device work): the internal order and the gather
 * structures that fedfem_precompute and the tiled kernel build for this mesh.
 * For inspection and tests.  Call once with every array NULL to get the sizes
 * in *info, then again with caller-allocated arrays:
 *   node_of[n_nodes]       internal node -> input node
 *   elem_of[n_elems]       internal element -> input element
 *   slice_off[n_slices+1], gather[n_gather]: node i (internal, free) receives
 *       the element loads gather[slice_off[i/32] + 32k + i%32], k = 0.., each
 *       entry internal_element * elem_type + corner, pads = n_elems * elem_type,
 *       in input element order (the summation order of every kernel)
 *   tile_elem_off[n_tiles+1], tile_elems[n_tile_elems] (internal elements,
 *       ascending), tile_lconn[n_tile_elems * elem_type]: the local id of each
 *       corner (owned nodes first, then tile_halo) in the low tile_rank_shift
 *       bits and, for an owned corner, above them the element's rank in that
 *       node's gather list (its position in the node's fixed-order sum),
 *   tile_halo_off[n_tiles+1], tile_halo[n_halo] (internal node ids),
 *   tile_degree[n_tiles] (most elements at one owned node of the tile).
 * tile_nodes <= 0 requests no tiles.  groups: element groups as in
 * fedfem_set_element_groups, or NULL.  Mesh / Dirichlet / face arguments as in
 * the set_* calls.  Returns FEDFEM_E_MESH / FEDFEM_E_ARG on bad input. */
int fedfem_plan_layout(int elem_type, int64_t n_nodes, const double* xyz, int64_t n_elems, const int32_t* conn,
                       const int32_t* groups, int order, int64_t n_dirichlet, const int32_t* dirichlet_nodes,
                       int64_t n_faces, int nverts, const int32_t* faces, int tile_nodes,
                       fedfem_layout_info* info, int32_t* node_of,
                       int32_t* elem_of, int32_t* slice_off, int32_t* gather, int32_t* tile_elem_off,
                       int32_t* tile_elems, uint16_t* tile_lconn, int32_t* tile_halo_off, int32_t* tile_halo,
                       int32_t* tile_degree);

/* Explicit steps that allocate nothing (the paper has no counterpart).
 *
 * For callers that may not allocate device memory themselves or through this
 * library -- code running inside another framework's memory pool, a
 * real-time loop that forbids allocation after start-up, or a plug-in that
 * must not call cudaMalloc/cudaFree.  There is no context: the caller passes
 * the mesh, the gather structure and the temperature as its own device
 * buffers, and every temporary (element loads, element matrices, lumped
 * volumes and loads) lives in one fixed device array inside the library
 * (about 18.3 MB, held by every GPU that loads the library until the process
 * exits).  Nothing is allocated or freed by the call.
 *
 * What it computes: n_steps explicit steps in FP64 of the same element loads
 * and nodal update as fedfem_step, restricted to one material with linear
 * laws (mat), uniform perfusion and metabolism (perf), hex8 with the one-point
 * rule only, and the element-share lumped volume (V_i = sum of V_e / nv over
 * the node's elements).  No film condition, nodal flux, tables, regions,
 * uniform V/N lumping, source schedule or dose; no temperature range check.
 * It runs on the CURRENT CUDA device, on `cuda_stream` (NULL = legacy default
 * stream), and returns after its work has completed.  Each call looks up the
 * array's device address on the current device and recomputes the element
 * matrices and lumped volumes.
 *   xyz_dev     n_nodes x 3 coordinates (m), row-major
 *   conn_dev    n_elems x elem_type node ids, as in fedfem_set_mesh
 *   row_ptr_dev n_nodes + 1 offsets into slot_dev: row_ptr[0] = 0,
 *               non-decreasing, row_ptr[n_nodes] = n_elems * elem_type
 *   slot_dev    n_elems * elem_type entries; for node i, entries
 *               row_ptr[i] .. row_ptr[i+1]-1 are e * elem_type + corner for
 *               every (element e, corner) that is node i, in increasing order
 *               (this fixes the summation order)
 *   q_r_dev     n_nodes source densities (W/m^3) or NULL; loads are
 *               V_i (Q_m + q_r[i]) with V_i the lumped volume
 *   held_dev    n_nodes bytes, 1 = Dirichlet node kept at its value in T, or NULL
 *   T_dev       n_nodes temperatures, updated in place
 * Limits: n_elems <= 131072 and n_nodes <= 160000; larger meshes get
 * FEDFEM_E_ARG ("beyond the fixed scratch") without touching the device.
 * FEDFEM_E_MESH: a corner or slot index out of range, a gather row that is
 * not the node's corners in increasing order, a node with no element that is
 * not held, or an element with det J <= 0.  The indices are checked on the
 * device before anything is read through them, and T_dev is then left
 * unchanged.
 * All calls share the one array and it keeps the last call's contents (each
 * call clears its own flag word first); two calls whose work overlaps on the
 * GPU (other streams or other host threads) race. */
int fedfem_step_static(int elem_type, int64_t n_nodes, int64_t n_elems, const double* xyz_dev,
                       const int32_t* conn_dev, const int32_t* row_ptr_dev, const int32_t* slot_dev,
                       const fedfem_material* mat, const fedfem_perfusion* perf, const double* q_r_dev,
                       const unsigned char* held_dev, double dt, int64_t n_steps, double* T_dev,
                       void* cuda_stream);

/* ---- Learned surrogate building block ------------------------------------
 * BF16 GEMM on the tensor cores (the paper has no counterpart; it only points
 * to neural networks as future work, Section 4):
 *   Z = A B^T + bias,  out = act(Z)  (act 0: identity, 1: SiLU)
 * A: M x K bf16 (device, row-major, leading dimension lda), B: N x K bf16
 * (ldb); lda, ldb multiples of 8; K a multiple of 64; N a multiple of 16, at
 * most 256.  FP32 accumulation.  Outputs (any may be NULL): Z (fp32, ldz),
 * Cf (fp32 out, ldc), Cb (bf16 out, ldc).  k_chunk < K splits K over blocks
 * (multiples of 64); then `partial` must hold ceil(K/k_chunk) * M * N floats
 * and the splits are summed in a fixed order.  `status` (device int): bit 0
 * is set if a bounded wait gave up.  Asynchronous on `stream`. */
int fedfem_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K, int k_chunk,
                     const float* bias, int act, float* Z, int64_t ldz, float* Cf, void* Cb, int64_t ldc,
                     float* partial, int* status, void* stream);

/* Message-passing surrogate (the paper has no counterpart beyond pointing to
 * neural networks as future work, Section 4).  An encode-process-decode graph
 * network over the conduction sparsity graph (hidden 64, `layers` message-
 * passing layers) that maps node inputs [(T-37)/10, q/1e7, k(T)/k0, c(T)/c0,
 * Dirichlet flag] to y, the temperature change over a fixed number of
 * explicit steps in degC.  GEMMs run on the tensor cores in BF16 with FP32
 * accumulation; all sums have a fixed order (deterministic).  Flat parameter
 * layout: W_ne[64][5] b_ne[64] W_ee[64][4] b_ee[64], per layer W_e[64][192]
 * b_e[64] W_n[64][128] b_n[64], then w_d[64] b_d[1].  Batches of up to
 * max_batch graphs share the graph; device arrays are batch-major.
 *   src/dst: n_edges directed edges (host), sorted by dst then src;
 *   xyz: n_nodes x 3 coordinates (host, m); edge inputs are
 *   [(x_dst - x_src) / length_scale, |x_dst - x_src| / length_scale]. */
typedef struct fedfem_mpnn fedfem_mpnn;
int fedfem_mpnn_create(fedfem_mpnn** out, int device, int64_t n_nodes, int64_t n_edges, const int32_t* src,
                       const int32_t* dst, const double* xyz, double length_scale, int layers, int max_batch,
                       void* cuda_stream);
void fedfem_mpnn_destroy(fedfem_mpnn* m);
int64_t fedfem_mpnn_n_params(const fedfem_mpnn* m);
const char* fedfem_mpnn_last_error(const fedfem_mpnn* m);
/* Parameters as host floats (n_params); set_params also resets the optimiser. */
int fedfem_mpnn_set_params(fedfem_mpnn* m, const float* params);
int fedfem_mpnn_get_params(fedfem_mpnn* m, float* params);
/* Node inputs (device): T and q are batch x n_nodes floats, dirichlet n_nodes
 * bytes or NULL; x_out batch x n_nodes x 5. */
int fedfem_mpnn_features(fedfem_mpnn* m, int batch, const float* T_dev, const float* q_dev,
                         const unsigned char* dirichlet_dev, const fedfem_material* mat, float* x_out_dev);
/* y_dev (batch x n_nodes) = network(x_dev); keeps what fedfem_mpnn_loss_grad
 * needs (the training path). */
int fedfem_mpnn_forward(fedfem_mpnn* m, int batch, const float* x_dev, float* y_dev);
/* y_dev (batch x n_nodes) = network(x_dev) by the fused inference kernels:
 * per layer one edge kernel (gather, tensor-core product, message, edge
 * update and per-node message sums in its epilogue) and one node kernel; no
 * training caches.  Same numbers as fedfem_mpnn_forward.  Asynchronous on the
 * network's stream; fedfem_mpnn_sync reports a tensor-core wait that gave up
 * (FEDFEM_E_TIMEOUT).  Needs every node's in-degree <= 128
 * (FEDFEM_E_UNSUPPORTED at create otherwise). */
int fedfem_mpnn_infer(fedfem_mpnn* m, int batch, const float* x_dev, float* y_dev);
/* Wait for the network's stream; FEDFEM_E_TIMEOUT if a bounded wait gave up. */
int fedfem_mpnn_sync(fedfem_mpnn* m);
/* Mean squared error over nodes with mask 1 (mask_dev: n_nodes floats) and
 * its gradient; *loss and grad (n_params host floats) may be NULL.  Keeps the
 * gradient for fedfem_mpnn_adam. */
int fedfem_mpnn_loss_grad(fedfem_mpnn* m, int batch, const float* x_dev, const float* target_dev,
                          const float* mask_dev, float* loss, float* grad);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with the last gradient. */
int fedfem_mpnn_adam(fedfem_mpnn* m, float lr);

/* Testing hooks (the paper has no counterpart).  key 1: barrier spin limit in
 * clock64 ticks for later fedfem_step calls (default 4e9, or the environment
 * variable FEDFEM_BARRIER_SPIN_LIMIT).  key 2: index of a block that never
 * arrives at the grid barrier from the next fedfem_init on (-1: none); the
 * other blocks then give up after the spin limit and fedfem_sync returns
 * FEDFEM_E_TIMEOUT.  Used to test the bounded waits without faulting. */
int fedfem_debug_set(fedfem_ctx* ctx, int key, int64_t value);

#ifdef __cplusplus
}
#endif
#endif /* FEDFEM_H */
