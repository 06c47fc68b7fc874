// Internal declarations of the GB300 RAM library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ram.h"

namespace ram {

// bits of the plan's device error word
enum ErrBits : int {
    ERR_CFL = 1,        // |dv| dt / (nsub dx) > 1
    ERR_NONFINITE = 2,  // non-finite shift
    ERR_NSUB = 4,       // sub-step count outside [1, RAM_MAX_NSUB]
    ERR_TIMEOUT = 8,    // a bounded wait gave up
    ERR_WINDOW = 16,    // a source window exceeded its planned bound
};

enum Mode : int { MODE_SHIFT = 0, MODE_RESIDUAL = 1, MODE_STEP = 2 };

// Per-row data on the device.
struct RowInfo {
    int64_t cell_off;     // first cell of the row in packed Q / dv arrays
    int64_t mesh_off;     // first cell of the row's mesh in the plan's mesh arrays
    int64_t bucket_off;   // first entry of the row's bucket table
    int32_t n;            // cells
    int32_t order;        // 2, 3, 4
    int32_t uniform;      // 1: equal widths, O(1) edge index
    int32_t bucket_bits;  // log2 of the row's bucket count
    int32_t qshift;       // FP32 warp-segment kernel: window-relative fixed-point
                          // positions are kept as 32-bit values in units of 2^qshift
    int32_t density;      // index of the row's mesh-density function, -1: none
    double period;        // L
    double cells_per_length;  // N / L
    double dx;            // L / N (uniform rows)
    double inv_period;    // 1 / L
};

// A row's mesh-density function (App. B.1, the periodic bump centred at 0 on
// [x_min, x_min + L]), for the index function of Sec. 3.2.1.
struct Density {
    float x_min, L, a, b, c, inv_norm;  // inv_norm = 1 / (L + c (a + b))
    float prim_min;                       // the bump's primitive at x_min
    float pad;
};

// Position of a row in the packed arrays, for kernels that stage whole rows.
struct RowPos {
    int64_t cell_off;
    int32_t row;
    int32_t n;
};

// One unit of work: output cells [start, start + count) of one row.
struct Tile {
    int32_t row;
    int32_t start;
    int32_t count;
    int32_t window;       // bound on the source-window cells (non-uniform tiles)
};

// Non-uniform tiles: residual halo (cells per side, the most sub-steps) and
// reconstruction halo (cells per side) of the general kernel.
constexpr int kGenHalo = 2 * RAM_MAX_NSUB;
constexpr int kGenHR = 2;

// FP32 rows with their own mesh: the warp-segment kernel (ram_nseg.cu).  A lane
// forms the reconstructions of kNsegV consecutive window cells; a segment has
// at most kNseg output cells; a CTA of kNsegWarps warps takes a tile of up to
// kNsegWarps * kNsegPerWarp segments.
constexpr int kNsegV = 4;
constexpr int kNseg = 96;
constexpr int kNsegHR = 2;          // reconstruction halo, cells per side
constexpr int kNsegWarps = 8;
constexpr int kNsegPerWarp = 4;
// shortest row it takes (a segment and its residual halo span less than a period)
constexpr int kNsegMinCells = 2 * kGenHalo + 2;

// Tries of a bounded device-side wait before it gives up and records a timeout.
constexpr uint32_t kWaitLimit = 1u << 20;

// Arguments shared by the step kernels (passed by value).

struct StepArgs {
    const RowInfo *rows;
    const Tile *tiles;
    int32_t n_tiles;
    int32_t mode;         // Mode
    const void *q_in;
    void *q_out;
    const double *shift;  // MODE_SHIFT
    const double *v0;     // MODE_STEP
    double dt;            // MODE_STEP / MODE_RESIDUAL
    double *phase;        // MODE_STEP, may be null
    const void *dv;       // null -> no residual
    const int32_t *nsub;  // null -> 1
    int32_t scheme;       // RAM_DONOR / RAM_VANLEER
    int32_t limiter;      // 1 = limiters on
    int *err;             // device error word
    // mesh of non-uniform rows
    const uint64_t *xfix;   // fixed-point nodes: (x_j - x_0) / L * 2^64, j = 0..N-1
    const float *dx32;      // widths, FP32
    const double *dx64;     // widths, FP64
    const int32_t *buckets; // per-row bucket table: cell holding each bucket start
    const Density *density; // mesh-density functions of rows that have one
    uint32_t wait_limit = kWaitLimit;  // tries of every bounded mbarrier wait
    int32_t row_phase = 0;  // no parameter kernel ran: the row kernels advance the phase
};

// Shift parameters of one uniform row for one launch (S0), written by the
// parameter kernel and read by the uniform-row kernels.
template <typename T> struct RowParams {
    int64_t cell_off;  // first cell of the row in the packed arrays
    int32_t n;         // cells
    int32_t K;         // whole cells of the shift, in [0, n)
    int32_t whole;     // the shift is a whole number of cells
    int32_t nsub;      // residual sub-steps (0: no residual in this launch)
    T c[5];            // partial-integral coefficients at the edge offset
    T cf;              // uniform rows: Courant number per unit dv of one sub-step;
                       // other rows: the sub-step length dt / nsub
    uint64_t sfix;     // the shift as a fraction of the period in units of 2^-64
};

// the plan
struct Plan {
    int device = 0;
    int32_t n_rows = 0;
    int64_t n_cells = 0;
    uint32_t flags = 0;
    int limiter = 1;
    int32_t tile_cells = 1024;
    int32_t threads = 256;
    int32_t rows_v[2] = {7, 7};    // cells per thread of the whole-row kernel (FP32, FP64)
    int32_t rows_cps[2] = {2, 1};  // CTAs per SM of the whole-row kernel (FP32, FP64)
    std::vector<int64_t> row_offset;
    std::vector<RowInfo> rows_h;
    std::vector<double> nodes_h;   // host copy of the FP64 nodes (per row or shared)
    std::vector<Tile> tiles_uniform_h[5];  // by order (index 2..4): every uniform row
    std::vector<Tile> tiles_general_h[5];  // whole-row tiles first, then windowed ones
    // per order: whole-row tiles, and for (whole-row, windowed) tiles the largest
    // source window and output extent (cells) the general kernel stages
    int32_t gen_whole[5] = {0};
    int32_t gen_wcap[5][2] = {{0}};  // [order][class]
    int32_t gen_qcap[5][2] = {{0}};
    // FP32: the tiles of the rows the warp-segment kernel does not take (the same
    // layout as above), and the warp-segment kernel's tiles (window = cells per
    // segment of the row) with the largest source window of any of its segments
    std::vector<Tile> tiles_general32_h[5];
    int32_t gen32_whole[5] = {0};
    int32_t gen32_wcap[5][2] = {{0}};
    int32_t gen32_qcap[5][2] = {{0}};
    // adjoint of rows with their own mesh: tiles of at most adj_nu_tcap cells per
    // order, and (flag RAM_ADJOINT) scratch for the shifted field and the residual's
    // cotangent, n_cells values each of the plan's widest dtype
    std::vector<Tile> tiles_adj_nu_h[5];
    Tile *tiles_adj_nu[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int32_t adj_nu_tcap = 512;
    void *adj_scratch = nullptr;
    // RAM_ADJOINT with the limiter on: every row (uniform ones too) has the
    // fixed-point mesh and takes the gather adjoint, linearised at the step input
    int32_t adj_all = 0;
    // the fourth-order cell-average correction (flag RAM_A4): scratch for the
    // corrected averages and the remapped ones, n_cells values each (FP64 size)
    int32_t a4 = 0;
    void *a4_scratch = nullptr;
    std::vector<Tile> tiles_nseg_h;
    int32_t nseg_rows = 0;
    int32_t nu_kernel = 0;         // FP32 rows with their own mesh: 1 = warp-segment kernel
    // uniform rows taken by the persistent whole-row kernel, per dtype and order, and
    // the tiles of the remaining uniform rows
    std::vector<int32_t> rows_fit_h[2][5];
    std::vector<RowPos> rows_fit_pos_h[2][5];
    std::vector<Tile> tiles_rest_h[2][5];
    int32_t ncap_fit[2][5] = {{0}};
    // uniform rows taken by the warp-segment kernel, and the tiles of the others
    std::vector<int32_t> rows_seg_h[2][5];
    std::vector<Tile> tiles_rest_seg_h[2][5];
    // longest and shortest FP32 warp-segment row, by order (the streaming kernel
    // takes the same rows)
    int32_t stream_nmax[5] = {0};
    int32_t stream_nmin[5] = {0};
    int32_t stream_v = 8;          // cells per lane of the streaming kernel
    int32_t seg_variant = 0;       // warp-segment kernel (FP32): 1 = the next segment's
                                   // loads in flight
    int32_t seg_warps = 8;         // warp-segment kernel: warps per row CTA (3..8)
    // 0: persistent whole-row, 1: warp segments, 2: streaming warps (FP32 only)
    int32_t uniform_kernel[2] = {1, 1};
    int32_t n_uniform_rows = 0;
    int32_t window_max = 0;        // max planned source window (non-uniform tiles)
    uint32_t wait_limit = kWaitLimit;  // tries of the bounded waits (0: give up at once)
    // device
    RowInfo *rows = nullptr;
    Tile *tiles_uniform[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    Tile *tiles_general[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    Tile *tiles_general32[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    Tile *tiles_nseg = nullptr;
    int32_t *rows_fit[2][5] = {{nullptr}};
    RowPos *rows_fit_pos[2][5] = {{nullptr}};
    Tile *tiles_rest[2][5] = {{nullptr}};
    int32_t *rows_seg[2][5] = {{nullptr}};
    Tile *tiles_rest_seg[2][5] = {{nullptr}};
    void *row_par = nullptr;        // RowParams<double> per row (FP32 launches use the first
                                    // half of each slot as RowParams<float>)
    uint64_t *xfix = nullptr;
    float *dx32 = nullptr;
    double *dx64 = nullptr;
    int32_t *buckets = nullptr;
    Density *density = nullptr;
    int *err = nullptr;
};

// per-row shift parameters of the uniform rows (ram_params.cu)
cudaError_t launch_params(const Plan &p, ram_dtype dt, const StepArgs &a, cudaStream_t s);
// launch with programmatic stream serialization (the kernel may start before
// the previous kernel in the stream finishes; it calls griddepcontrol.wait
// before touching that kernel's results)
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// launchers (ram_uniform.cu, ram_general.cu)
cudaError_t launch_uniform(const Plan &p, ram_dtype dt, const StepArgs &a, cudaStream_t s);
cudaError_t launch_general(const Plan &p, ram_dtype dt, const StepArgs &a, cudaStream_t s);
// FP32 rows with their own mesh, warp-segment kernel (ram_nseg.cu)
cudaError_t launch_nseg(const Plan &p, const StepArgs &a, cudaStream_t s);
size_t nseg_smem_bytes(bool resid);
// largest source window (cells) a warp of it stages; rows above it take the tiled
// kernels
int nseg_window_cap();
cudaError_t launch_row_mass(const Plan &p, ram_dtype dt, const void *q, double *out,
                            cudaStream_t s);
cudaError_t launch_adjoint(const Plan &p, ram_dtype dt, const StepArgs &a, const void *g_out,
                           void *g_in, void *g_dv, cudaStream_t s);
// the fourth-order cell-average correction (ram_a4.cu): to_avg: point values to
// corrected averages, else the inverse
cudaError_t launch_a4(const Plan &p, ram_dtype dt, const void *in, void *out, cudaStream_t s,
                      bool to_avg);
// the radial sweep of a polar disk (ram_radial.cu)
cudaError_t launch_radial(const Plan &p, ram_dtype dt, const void *q_in, void *q_out,
                          const double *rf, const void *vr, double step, int scheme,
                          cudaStream_t s);
// rows with their own mesh (ram_adjoint_nu.cu)
cudaError_t launch_adjoint_nu(const Plan &p, ram_dtype dt, const StepArgs &a, const void *g_out,
                              void *g_in, void *g_dv, cudaStream_t s);

cudaError_t launch_rows(const Plan &p, ram_dtype dt, const StepArgs &a, cudaStream_t s,
                        int order, const RowPos *rows, int n_rows, int ncap);
cudaError_t launch_useg(const Plan &p, ram_dtype dt, const StepArgs &a, cudaStream_t s,
                        int order, const int32_t *row_ids, int n_rows);

// streaming kernel for the FP32 warp-segment rows of one order (ram_stream.cu)
cudaError_t launch_stream(const Plan &p, const StepArgs &a, cudaStream_t s, int order);
// the smallest row the streaming kernel takes with v cells per lane
int stream_min_cells(int v);
extern const int kStreamVCandidates[];
extern const int kStreamVCount;

// tiling (ram_plan.cu)
ram_status build_tiles(Plan &p);

// Largest row length (cells) the persistent whole-row kernel stages in shared memory.
int rows_kernel_max_cells(ram_dtype dt);

// Cells-per-thread values the whole-row kernel is built for (autotuner candidates).
extern const int kRowsVCandidates[];
extern const int kRowsVCount;

}  // namespace ram
