// A RAM step that allocates no device memory, for callers that cannot call
// cudaMalloc: code running inside an allocator or memory-pool callback, code
// that must not disturb a fixed device-memory budget, or hosts where device
// allocation is reserved to another component.  It covers rows of equal length
// on one uniform periodic mesh (the rings of a disk) and runs the same kernels
// as ram_step's warp-segment path; the per-row table, the row list and the
// per-row shift parameters that those kernels keep in plan-owned memory live
// here in one fixed-size static device array instead.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "ram_internal.h"

namespace ram {
namespace {

constexpr int kStaticRows = RAM_STATIC_MAX_ROWS;
constexpr size_t kErrBytes = 256;
constexpr size_t kRowInfoBytes = ((sizeof(RowInfo) * kStaticRows + 255) / 256) * 256;
constexpr size_t kParamBytes = ((sizeof(RowParams<double>) * kStaticRows + 255) / 256) * 256;
constexpr size_t kIdsBytes = ((sizeof(int32_t) * kStaticRows + 255) / 256) * 256;
constexpr size_t kScratchBytes = kErrBytes + kRowInfoBytes + kParamBytes + kIdsBytes;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the array, looked up once per device with that device current.
constexpr int kMaxDevices = 64;
unsigned char *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

cudaError_t scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned char *>(ptr);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// Row table and row list of the call (every row: n cells, period L, packed back
// to back).
__global__ void k_static_rows(RowInfo *rows, int32_t *ids, int n_rows, int n, double period,
                              int order)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    RowInfo ri;
    ri.cell_off = (int64_t)r * n;
    ri.mesh_off = 0;
    ri.bucket_off = 0;
    ri.n = n;
    ri.order = order;
    ri.uniform = 1;
    ri.bucket_bits = 0;
    ri.qshift = 0;
    ri.density = -1;
    ri.period = period;
    ri.cells_per_length = (double)n / period;
    ri.dx = period / n;
    ri.inv_period = 1.0 / period;
    rows[r] = ri;
    ids[r] = r;
}

bool aligned16(const void *p) { return ((uintptr_t)p % 16) == 0; }

}  // namespace
}  // namespace ram

using namespace ram;

extern "C" ram_status ram_step_uniform_noalloc(ram_dtype dtype, int32_t n_rows,
                                               int32_t n_cells_per_row, double period,
                                               int32_t order, uint32_t flags,
                                               const void *q_in, void *q_out,
                                               const double *v0, double dt,
                                               const void *dv_iface, ram_scheme scheme,
                                               const int32_t *nsub, int32_t *device_errors,
                                               void *stream)
{
    if (dtype != RAM_F32 && dtype != RAM_F64) return RAM_ERR_ARG;
    if (n_rows < 1 || n_rows > kStaticRows) return RAM_ERR_ARG;
    const size_t es = dtype == RAM_F32 ? 4 : 8;
    const int n = n_cells_per_row;
    if (n < 512 || (n * es) % 16 != 0) return RAM_ERR_UNSUPPORTED;
    if (!(period > 0.0) || period > 1e300) return RAM_ERR_MESH;
    if (order < 2 || order > 4) return RAM_ERR_ARG;
    if (flags & ~RAM_LIMITER_OFF) return RAM_ERR_ARG;
    // the limited order 4 needs per-cell work the uniform-row kernels do not do
    if (order == 4 && !(flags & RAM_LIMITER_OFF)) return RAM_ERR_UNSUPPORTED;
    if (scheme != RAM_DONOR && scheme != RAM_VANLEER) return RAM_ERR_ARG;
    if (!(dt >= 0.0) || dt > 1e300) return RAM_ERR_ARG;
    if (!q_in || !q_out || !v0) return RAM_ERR_ARG;
    if (!aligned16(q_in) || !aligned16(q_out) || (dv_iface && !aligned16(dv_iface)))
        return RAM_ERR_ARG;
    const size_t bytes = (size_t)n_rows * n * es;
    const char *a0 = static_cast<const char *>(q_in);
    const char *b0 = static_cast<const char *>(q_out);
    if (a0 < b0 + bytes && b0 < a0 + bytes) return RAM_ERR_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RAM_ERR_CUDA;
    unsigned char *base = nullptr;
    if (scratch_address(dev, &base) != cudaSuccess) return RAM_ERR_CUDA;
    int *err = reinterpret_cast<int *>(base);
    RowInfo *rows = reinterpret_cast<RowInfo *>(base + kErrBytes);
    void *par = base + kErrBytes + kRowInfoBytes;
    int32_t *ids = reinterpret_cast<int32_t *>(base + kErrBytes + kRowInfoBytes + kParamBytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // the error word of the previous call is cleared; the row table is rewritten
    if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return RAM_ERR_CUDA;
    k_static_rows<<<(n_rows + 127) / 128, 128, 0, s>>>(rows, ids, n_rows, n, period, order);
    if (cudaGetLastError() != cudaSuccess) return RAM_ERR_CUDA;

    // the same kernels as the plan path, pointed at the static tables
    Plan p;
    p.device = dev;
    p.n_rows = n_rows;
    p.n_cells = (int64_t)n_rows * n;
    p.n_uniform_rows = n_rows;
    p.row_par = par;
    StepArgs a{};
    a.rows = rows;
    a.q_in = q_in;
    a.q_out = q_out;
    a.mode = MODE_STEP;
    a.v0 = v0;
    a.dt = dt;
    a.phase = nullptr;
    a.dv = dv_iface;
    a.nsub = nsub;
    a.scheme = scheme;
    a.limiter = (flags & RAM_LIMITER_OFF) ? 0 : 1;
    a.err = device_errors ? reinterpret_cast<int *>(device_errors) : err;
    cudaError_t e = launch_params(p, dtype, a, s);
    if (e == cudaSuccess) e = launch_useg(p, dtype, a, s, order, ids, n_rows);
    return e == cudaSuccess ? RAM_OK : RAM_ERR_CUDA;
}
