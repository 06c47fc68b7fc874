/*
 * ram.h -- C ABI of the GB300 (sm_103a) RAM library.
 *
 * RAM (Rapid Advection Algorithm on Arbitrary Meshes, Benitez-Llambay, Krapp,
 * Ramos & Kratter, arXiv 2305.05362) solves  dQ/dt + d(Q v)/dx = 0  with
 * v = v0 + dv (Eq. 1, Eq. 4) by operator splitting (Eqs. 5-6): every row of cells
 * is first shifted by the bulk displacement s = v0 dt with a conservative remap
 * (Sec. 3: reconstruction, Eqs. 15-18, Eq. 26), then advanced with the residual
 * velocity dv by an upwind step.
 *
 * Conventions used by every entry point
 *  - A plan describes n_rows independent periodic rows (rings of a disk,
 *    problems of a batch; dimensional splitting, Sec. 3.5).  Row r owns the
 *    cells [row_offset[r], row_offset[r+1]) of every packed cell array.
 *  - Row r has N_r cells and N_r+1 strictly increasing nodes
 *    x_{-1/2} < x_{1/2} < ... < x_{N-1/2} (Sec. 2); its period is
 *    L_r = x_{N-1/2} - x_{-1/2}.
 *  - Cell values Q are cell averages (Eq. 2-3), packed, FP32 or FP64 (ram_dtype).
 *  - The residual velocity dv is given at interfaces: element row_offset[r]+j is
 *    dv at node x_{j-1/2} of row r, same dtype as Q, j = 0..N_r-1 (node N is node 0).
 *  - The content of a row moves by +s: output cell i receives the mass of the
 *    source interval [x_{i-1/2} - s, x_{i+1/2} - s] (Sec. 3.2).  Any real s is
 *    accepted; it is reduced modulo L_r.
 *  - Device pointers are device memory of the plan's device.  The caller owns
 *    every cell, velocity, shift, phase and gradient buffer; the plan owns its
 *    copy of the mesh, its tile lists and its device error word.
 *  - The step entry points (ram_shift, ram_residual_upwind, ram_step,
 *    ram_step_adjoint, ram_row_mass) only enqueue kernels on `stream`: they
 *    never allocate and never synchronise, so they may be captured in a CUDA
 *    graph.  They validate host-visible arguments synchronously and return an
 *    error without launching anything.  Conditions found on the device (CFL
 *    above 1 in the residual step, a non-finite shift, an out-of-range sub-step
 *    count, a wait that timed out) set bits in the plan's error word, which
 *    ram_plan_check_errors reads and clears.
 *  - Input and output cell arrays must not overlap (RAM_ERR_ARG).
 */
#ifndef RAM_H
#define RAM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RAM_OK = 0,
    RAM_ERR_ARG = 1,          /* bad pointer, size, enum, aliasing or alignment */
    RAM_ERR_MESH = 2,         /* nodes not strictly increasing, N < 1, bad period */
    RAM_ERR_CFL = 3,          /* |dv| dt / (nsub dx) > 1 somewhere (residual step) */
    RAM_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    RAM_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    RAM_ERR_NOMEM = 6,        /* allocation during planning failed */
    RAM_ERR_UNSUPPORTED = 7,  /* valid request outside what the plan/kernels support */
    RAM_ERR_NONFINITE = 8     /* a non-finite shift was found on the device */
} ram_status;

typedef enum { RAM_F32 = 0, RAM_F64 = 1 } ram_dtype;
typedef enum { RAM_DONOR = 0, RAM_VANLEER = 1 } ram_scheme;

/* plan flags */
#define RAM_LIMITER_OFF 1u  /* unlimited reconstruction (PLM centred slope, PPM
                               without App. A.2); makes the shift linear in Q */
#define RAM_SHARED_MESH 2u  /* every row uses row 0's nodes (all rows equal N) */
#define RAM_ADJOINT 4u      /* reserve the device scratch that ram_step_adjoint needs on
                               rows with their own mesh when a residual step is
                               present (2 x n_cells values of the plan's widest dtype) */
#define RAM_A4 8u           /* the fourth-order cell-average correction of Sec. 3.1: the
                               cell arrays hold point values; ram_shift and ram_step remap
                               <Q>_i = Q_i + (Q_{i+1} - 2Q_i + Q_{i-1}) / 24 with PPM and
                               return the point values whose corrected averages are the
                               remapped ones (the periodic tridiagonal inverse), then the
                               residual step acts on the point values.  Every row must be
                               uniform and of order 3 (else RAM_ERR_UNSUPPORTED); reserves
                               2 x n_cells values of scratch; no adjoint. */

/* largest residual sub-step count a row may ask for */
#define RAM_MAX_NSUB 8

typedef struct ram_plan_s *ram_plan;

typedef struct {
    int32_t n_rows;            /* >= 1 */
    const int64_t *row_offset; /* host, n_rows+1 entries, row_offset[0] = 0, increasing */
    const double *nodes;       /* host, FP64.  Per-row meshes: row r's N_r+1 nodes are
                                  nodes[row_offset[r] + r .. row_offset[r+1] + r].
                                  RAM_SHARED_MESH: nodes[0 .. N] only. */
    const int8_t *order;       /* host, per-row reconstruction order p in {2,3,4}
                                  (2 = PLM, 3 = PPM, 4 = quartic cumulative, with the
                                  limiter on scaled toward the cell mean within the
                                  range of the cell and its neighbours); NULL ->
                                  default_order for every row */
    int8_t default_order;
    uint32_t flags;            /* RAM_LIMITER_OFF | RAM_SHARED_MESH | RAM_ADJOINT | RAM_A4 */
} ram_mesh_desc;

/* Build a plan for the rows in `desc` on CUDA device `device` (Sec. 2 mesh,
 * Sec. 3.2 index search).  Validates the mesh, copies it to the device in the
 * plan's own layout, classifies rows (uniform rows take the O(1) index of
 * Sec. 3.2.1), builds the tile lists and allocates the error word.  Host
 * synchronous; the only entry point besides ram_plan_autotune that allocates.
 * On failure *out is NULL and nothing is leaked. */
ram_status ram_plan_mesh(const ram_mesh_desc *desc, int device, ram_plan *out);

/* A row generated by a mesh-density function: the periodic bump of App. B.1,
 * density 1 + c for |x| <= a, 1 + c cos^2(pi/2 (|x| - a)/(b - a)) for a < |x| < b,
 * 1 beyond, on the row's domain [x_min, x_max] (which holds the bump: x_min <= -b,
 * b <= x_max), normalised by I = (x_max - x_min) + c (a + b) (Eq. 24). */
typedef struct {
    double x_min, x_max;
    double a, b, c;
} ram_density;

/* Mark rows as generated by their mesh-density function, so that the kernels
 * locate shifted edges with the index function of Sec. 3.2.1, p = floor(N u(x~))
 * with u the normalised cumulative of the density in closed form (App. B.1),
 * corrected against the row's exact nodes, instead of the plan's bucket table.
 * dens: host, one entry per row (with RAM_SHARED_MESH: one entry), or NULL to go
 * back to the bucket tables.  Each row's nodes must be the density's: x_0 = x_min,
 * x_N = x_max and |N u(x_j) - j| <= 1/4 at every node (RAM_ERR_MESH otherwise, the
 * plan unchanged).  Uniform rows ignore it.  Host synchronous, allocates. */
ram_status ram_plan_set_density(ram_plan plan, const ram_density *dens);

/* Free every device and host resource of the plan (the device copy of the
 * Sec. 2 mesh, the Sec. 3.2.1 index tables and the tile lists built by
 * ram_plan_mesh).  Host synchronous; NULL is accepted.  The caller's current
 * device is restored before returning. */
ram_status ram_plan_destroy(ram_plan plan);

/* The shift step alone (Sec. 3, steps 1-3; Eqs. 15-18 and 26): for every row r,
 * q_out = remap of q_in by +shift[r].  shift: device, FP64, one per row, any
 * real value (reduced modulo the period). */
ram_status ram_shift(ram_plan plan, ram_dtype dtype, const void *q_in, void *q_out,
                     const double *shift, void *stream);

/* The residual step alone (Eq. 6): nsub[r] flux-form upwind sub-steps of length
 * dt/nsub[r] with the interface velocity dv.  scheme: RAM_DONOR (upwind cell
 * value) or RAM_VANLEER (van Leer PLM slope of the upwind cell, evaluated at the
 * midpoint of the swept region).  nsub: device int32 per row in
 * [1, RAM_MAX_NSUB], or NULL for 1. */
ram_status ram_residual_upwind(ram_plan plan, ram_dtype dtype, const void *q_in,
                               void *q_out, const void *dv_iface, double dt,
                               ram_scheme scheme, const int32_t *nsub, void *stream);

/* One full RAM step (Eqs. 5-6 with Sec. 3): shift by s_r = v0[r] * dt, then the
 * residual step with dv_iface (NULL -> dv = 0, no residual).  v0: device FP64
 * per row.  phase: device FP64 per row, or NULL; when given, phase[r] is
 * replaced by (phase[r] + s_r) reduced to [0, L_r), the accumulated offset
 * v0 t mod L of the row (always in FP64).  The cell shift s_r N_r / L_r is
 * formed in FP64, except on FP32 rows of the shared-memory ring form of the
 * warp-segment kernel, which form it in two-float arithmetic (about 2^-46
 * relative) and treat a shift of 2^40 cells or more as non-finite. */
ram_status ram_step(ram_plan plan, ram_dtype dtype, const void *q_in, void *q_out,
                    double *phase, const double *v0, double dt, const void *dv_iface,
                    ram_scheme scheme, const int32_t *nsub, void *stream);

/* Transpose of one linear RAM step (Eqs. 5-6 with the remap of Sec. 3,
 * Eqs. 15-18 and 26).  With the limiter off the reconstruction of Sec. 3.1 /
 * App. A is linear in Q, so the remap is a fixed matrix A(s) for a given shift
 * and the donor-cell residual step (Eq. 6) is linear in Q too; this entry point
 * applies the transpose of their product.  The plan must have RAM_LIMITER_OFF
 * and the residual scheme is donor cell.  Given the step input q_in (the same arguments
 * as the forward ram_step) and the cotangent g_out of the step output, writes
 * g_in = J^T g_out and, when g_dv is not NULL, ADDS d<g_out, out>/d dv into g_dv
 * (device, same packing and dtype as dv).  At dv_j == 0 the upwind side of the
 * flux derivative is the left cell.  dv_iface NULL -> no residual step. */
ram_status ram_step_adjoint(ram_plan plan, ram_dtype dtype, const void *q_in,
                            const void *g_out, void *g_in, const double *v0, double dt,
                            const void *dv_iface, void *g_dv, const int32_t *nsub,
                            void *stream);

/* The radial sweep of a polar disk, for dimensional splitting in two dimensions
 * (Sec. 3.5: RAM along the azimuth, a standard upwind step along the radius).  The
 * plan must have RAM_SHARED_MESH (RAM_ERR_UNSUPPORTED otherwise): its rows are the
 * rings j = 0 .. n_rows-1 of N azimuthal cells on one mesh, ring j between the
 * radii rf[j] < rf[j+1] (rf: device, FP64, n_rows + 1 values, increasing).
 * vr: device, the plan's dtype, (n_rows + 1) x N values, element j N + i is the
 * radial velocity on face j (radius rf[j], between rings j-1 and j) at azimuthal
 * cell i; faces 0 and n_rows are closed walls and are not read.  One flux-form
 * upwind step of length dt in cylindrical geometry:
 *   q'_j = q_j - dt (rf[j+1] F_{j+1} - rf[j] F_j) / A_j,  A_j = (rf[j+1]^2 - rf[j]^2) / 2,
 * F = vr q_up (RAM_DONOR) or vr times the upwind ring's van Leer profile (Sec. 3.1,
 * centre spacings; flat in the rings next to the walls) at the midpoint of the
 * swept interval (RAM_VANLEER).  Conserves sum_j A_j q_j over every column.
 * |vr| dt above the upwind ring's width sets RAM_ERR_CFL in the error word.
 * Enqueues one kernel; no allocation or synchronisation. */
ram_status ram_radial_upwind(ram_plan plan, ram_dtype dtype, const void *q_in, void *q_out,
                             const double *rf, const void *vr, double dt, ram_scheme scheme,
                             void *stream);

/* Mass of every row, sum_i Q_i dx_i (Eq. 10), written as FP64 to mass_out
 * (device, one per row).  FP32 cells are summed exactly as products and
 * accumulated with a compensated (two-float) scan. */
ram_status ram_row_mass(ram_plan plan, ram_dtype dtype, const void *q, double *mass_out,
                        void *stream);

/* Synchronise the plan's device, then return (and clear) the first condition
 * recorded in the device error word since the last call: RAM_OK, RAM_ERR_CFL,
 * RAM_ERR_NONFINITE, RAM_ERR_ARG (sub-step count out of range) or
 * RAM_ERR_TIMEOUT. */
ram_status ram_plan_check_errors(ram_plan plan);

/* Failure-detection test hook.  Every device-side wait of the step kernels (the
 * persistent whole-row kernel's waits for its staged rows and for free stages)
 * is bounded: after `limit` tries (default 2^20) it gives up, records
 * RAM_ERR_TIMEOUT in the error word and the CTA returns once its own copies in
 * flight have landed, so a stalled pipeline ends the launch instead of hanging
 * the GPU.  `limit` = 0 makes every such wait give up at once, which exercises
 * that path deterministically: the next ram_plan_check_errors returns
 * RAM_ERR_TIMEOUT and the step's output is undefined.  Other kernels have no
 * waits and are unaffected.  Host only; applies to later launches of this plan.
 * Returns RAM_ERR_ARG for a NULL plan. */
ram_status ram_plan_set_wait_limit(ram_plan plan, uint32_t limit);

typedef struct {
    int32_t n_rows;
    int64_t n_cells;
    int32_t n_uniform_rows;   /* rows on the O(1)-index path */
    int32_t n_tiles_uniform;
    int32_t n_tiles_general;
    int32_t tile_cells;       /* output cells per tile */
    int32_t threads;          /* threads per CTA */
    int32_t device;
    int32_t n_nseg_rows;      /* rows with their own mesh that FP32 steps run on the
                                 warp-segment kernel (the others take the tiled one) */
    int32_t n_density_rows;   /* rows located by their mesh-density function */
} ram_plan_info;

ram_status ram_plan_query(ram_plan plan, ram_plan_info *info);

/* Tuning: output cells per tile (64..8192) and threads per CTA (64..1024,
 * multiple of 32) of the tiled kernels.  Rebuilds the tile lists; host
 * synchronous. */
ram_status ram_plan_set_tiling(ram_plan plan, int32_t tile_cells, int32_t threads);

/* Launch shapes of a plan's kernels. */
typedef struct {
    int32_t rows_cells_per_thread_f32;  /* whole-row kernel, FP32: 5, 7, 9, 11 or 15 */
    int32_t rows_cells_per_thread_f64;  /* whole-row kernel, FP64 */
    int32_t tile_cells;                 /* tiled kernels: output cells per tile */
    int32_t threads;                    /* tiled kernels: threads per CTA */
    int32_t uniform_kernel_f32;         /* uniform rows, FP32: 0 = persistent whole-row
                                           kernel (TMA-staged rows), 1 = warp segments,
                                           2 = streaming warps (TMA-staged segments) */
    int32_t uniform_kernel_f64;         /* uniform rows, FP64: 0 or 1 */
    int32_t rows_ctas_per_sm_f32;       /* whole-row kernel, FP32: CTAs per SM, 1..4 */
    int32_t rows_ctas_per_sm_f64;       /* whole-row kernel, FP64: 1 */
    int32_t stream_cells_per_lane_f32;  /* streaming-warp kernel, FP32: 4 or 8 cells per
                                           lane and segment (8 needs rows >= 520 cells) */
    int32_t seg_variant_f32;            /* warp-segment kernel, FP32: 0 = one segment in
                                           flight per warp, 1 = the loads of a warp's next
                                           segment in flight while it computes, 2 = a ring
                                           of 2 shared-memory stages per warp, the row's
                                           segments handed out by a counter as the warps
                                           issue their copies, its shift parameters
                                           formed in the kernel (no parameter kernel
                                           when every row takes it; the default) */
    int32_t seg_warps;                  /* warp-segment kernel: warps per row CTA, 3..8
                                           (default 3) */
    int32_t nonuniform_kernel_f32;      /* FP32 rows with their own mesh: 0 = the
                                           per-order kernels (shared-memory-free without
                                           a residual, tiled with one; the default),
                                           1 = the warp-segment kernel (one launch for
                                           every order, shift and residual together) */
} ram_tuning;

ram_status ram_plan_get_tuning(ram_plan plan, ram_tuning *out);
/* Host synchronous (rebuilds the tile lists when the tile shape changes). */
ram_status ram_plan_set_tuning(ram_plan plan, const ram_tuning *tuning);

/* Autotuner: times every candidate launch shape of the kernels this plan uses
 * on the caller's buffers -- the arguments of ram_step, without the phase --
 * with CUDA events on `stream` (`reps` timed steps per candidate) and keeps the
 * fastest in the plan.  Candidates: for uniform rows the warp-segment kernel
 * (3, 4, 6 or 8 warps per row CTA; FP32: with and without prefetch),
 * for FP32 the streaming-warp kernel with 4 or 8 cells per lane, and the
 * persistent whole-row kernel with (cells per thread, CTAs per SM) in
 * {5,7,9,11,15} x {2,3,4} as the register budget allows; tile cells
 * {256,512,1024,2048} x threads {128,256,512} of the tiled kernels; for FP32
 * rows with their own mesh, the warp-segment kernel against the per-order
 * kernels.  Host synchronous; overwrites q_out. */
ram_status ram_plan_autotune(ram_plan plan, ram_dtype dtype, const void *q_in, void *q_out,
                             const double *v0, double dt, const void *dv_iface,
                             ram_scheme scheme, const int32_t *nsub, int32_t reps,
                             void *stream);

/* Largest number of rows ram_step_uniform_noalloc accepts. */
#define RAM_STATIC_MAX_ROWS 4096

/* One RAM step that allocates no device memory, for callers that cannot call
 * cudaMalloc (code running inside an allocator or memory-pool callback, or
 * next to a fixed device-memory budget that must not move).  The paper has no
 * counterpart: it is a plan-free variant of ram_step for n_rows rows of
 * n_cells_per_row cells each, packed back to back, all on one uniform periodic
 * mesh of period `period` (the rings of a disk), with reconstruction `order`
 * (2, 3, 4; order 4 only with RAM_LIMITER_OFF, else RAM_ERR_UNSUPPORTED) and
 * flags 0 or RAM_LIMITER_OFF.  The other arguments are those of
 * ram_step (no phase).  Its row table, row list and per-row shift parameters
 * live in one static device array of about 0.6 MiB that every GPU loading the
 * library keeps until the process exits; rows beyond RAM_STATIC_MAX_ROWS are
 * refused with RAM_ERR_ARG.  Rows must have at least 512 cells and a multiple
 * of 16 bytes per row, and q_in, q_out and dv_iface must be 16-byte aligned
 * (RAM_ERR_UNSUPPORTED / RAM_ERR_ARG otherwise).
 * flags other than RAM_LIMITER_OFF are refused with RAM_ERR_ARG.
 * Device-side conditions (CFL, non-finite shift, sub-step count) are ORed into
 * *device_errors (device int32, bits as in the plan error word: 1 CFL,
 * 2 non-finite, 4 sub-step count) when it is not NULL; the caller clears it.
 * With device_errors NULL those conditions are not reported to the caller.
 * `stream` must belong to the current device: the call uses the current
 * device's copy of the array.  The first call on a device looks up the array's
 * device address (once per device, with that device current) and caches it for
 * the life of the process: make that first call before any stream capture, and
 * do not reset the device (cudaDeviceReset) after it.  Every call overwrites
 * the array, so calls whose kernels overlap on the GPU (other streams, other
 * threads) race; order them on one stream. */
ram_status ram_step_uniform_noalloc(ram_dtype dtype, int32_t n_rows, int32_t n_cells_per_row,
                                    double period, int32_t order, uint32_t flags,
                                    const void *q_in, void *q_out, const double *v0,
                                    double dt, const void *dv_iface, ram_scheme scheme,
                                    const int32_t *nsub, int32_t *device_errors,
                                    void *stream);

const char *ram_status_string(ram_status status);

/* Library version, major * 10000 + minor * 100 + patch. */
int32_t ram_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RAM_H */
