// C ABI entry points of the step family: argument checks on the host, then the
// kernels are enqueued on the caller's stream (no allocation, no sync).
#include <cuda_runtime.h>

#include <cstdint>

#include "ram_internal.h"

using namespace ram;

namespace {

// Switches to the plan's device for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t dtype_size(ram_dtype d) { return d == RAM_F64 ? 8 : 4; }

bool overlaps(const void *a, const void *b, size_t bytes)
{
    const char *x = static_cast<const char *>(a);
    const char *y = static_cast<const char *>(b);
    return x < y + bytes && y < x + bytes;
}

ram_status check_common(const Plan *p, ram_dtype dt, const void *q_in, const void *q_out)
{
    if (!p) return RAM_ERR_ARG;
    if (dt != RAM_F32 && dt != RAM_F64) return RAM_ERR_ARG;
    if (!q_in || !q_out) return RAM_ERR_ARG;
    const size_t es = dtype_size(dt);
    if (((uintptr_t)q_in % es) || ((uintptr_t)q_out % es)) return RAM_ERR_ARG;
    if (overlaps(q_in, q_out, (size_t)p->n_cells * es)) return RAM_ERR_ARG;
    return RAM_OK;
}

StepArgs base_args(const Plan *p, const void *q_in, void *q_out)
{
    StepArgs a{};
    a.rows = p->rows;
    a.q_in = q_in;
    a.q_out = q_out;
    a.limiter = p->limiter;
    a.err = p->err;
    a.scheme = RAM_VANLEER;
    a.xfix = p->xfix;
    a.dx32 = p->dx32;
    a.dx64 = p->dx64;
    a.buckets = p->buckets;
    a.density = p->density;
    a.wait_limit = p->wait_limit;
    return a;
}

// Every row of this FP32 launch forms its own shift parameters, so no parameter
// kernel is needed: uniform rows on the shared-memory ring form of the
// warp-segment kernel (which needs 16-byte aligned arrays), rows with their own
// mesh on the non-uniform warp-segment kernel.
bool rows_form_params(const Plan &p, ram_dtype dt, const StepArgs &a)
{
    if (dt != RAM_F32) return false;
    size_t seg = 0;
    if (p.n_uniform_rows > 0) {
        if (p.uniform_kernel[0] != 1 || p.seg_variant != 2) return false;
        for (const void *ptr : {a.q_in, static_cast<const void *>(a.q_out), a.dv})
            if ((uintptr_t)ptr % 16) return false;
        for (int o = 2; o <= 4; ++o) seg += p.rows_seg_h[0][o].size();
    }
    return seg + (size_t)(p.nu_kernel == 1 ? p.nseg_rows : 0) == (size_t)p.n_rows;
}

ram_status run(const Plan *p, ram_dtype dt, const StepArgs &a0, void *stream)
{
    DeviceGuard g(p->device);
    if (!g.ok) return RAM_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StepArgs a = a0;
    cudaError_t e = cudaSuccess;
    if (rows_form_params(*p, dt, a))
        a.row_phase = 1;
    else
        e = launch_params(*p, dt, a, s);
    if (e == cudaSuccess) e = launch_uniform(*p, dt, a, s);
    if (e == cudaSuccess) e = launch_general(*p, dt, a, s);
    if (e == cudaErrorNotSupported) return RAM_ERR_UNSUPPORTED;
    return e == cudaSuccess ? RAM_OK : RAM_ERR_CUDA;
}

// A step of an A4 plan: corrected averages of the input, the shift of them,
// point values back, then the residual step (if any) on the point values.
ram_status run_a4(const Plan *p, ram_dtype dt, const StepArgs &a0, void *stream)
{
    DeviceGuard g(p->device);
    if (!g.ok) return RAM_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *s1 = static_cast<char *>(p->a4_scratch);
    char *s2 = s1 + (size_t)p->n_cells * sizeof(double);
    const bool resid = a0.mode == MODE_STEP && a0.dv != nullptr;
    if (launch_a4(*p, dt, a0.q_in, s1, s, true) != cudaSuccess) return RAM_ERR_CUDA;
    StepArgs a1 = a0;
    a1.q_in = s1;
    a1.q_out = s2;
    a1.dv = nullptr;
    ram_status st = run(p, dt, a1, stream);
    if (st != RAM_OK) return st;
    if (launch_a4(*p, dt, s2, resid ? static_cast<void *>(s1) : a0.q_out, s, false) != cudaSuccess)
        return RAM_ERR_CUDA;
    if (!resid) return RAM_OK;
    StepArgs a2 = a0;
    a2.mode = MODE_RESIDUAL;
    a2.q_in = s1;
    a2.phase = nullptr;
    return run(p, dt, a2, stream);
}

}  // namespace

extern "C" ram_status ram_shift(ram_plan plan, ram_dtype dtype, const void *q_in, void *q_out,
                                const double *shift, void *stream)
{
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    ram_status st = check_common(p, dtype, q_in, q_out);
    if (st != RAM_OK) return st;
    if (!shift) return RAM_ERR_ARG;
    StepArgs a = base_args(p, q_in, q_out);
    a.mode = MODE_SHIFT;
    a.shift = shift;
    return p->a4 ? run_a4(p, dtype, a, stream) : run(p, dtype, a, stream);
}

extern "C" ram_status ram_residual_upwind(ram_plan plan, ram_dtype dtype, const void *q_in,
                                          void *q_out, const void *dv_iface, double dt,
                                          ram_scheme scheme, const int32_t *nsub,
                                          void *stream)
{
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    ram_status st = check_common(p, dtype, q_in, q_out);
    if (st != RAM_OK) return st;
    if (!dv_iface || (scheme != RAM_DONOR && scheme != RAM_VANLEER)) return RAM_ERR_ARG;
    if (!(dt >= 0.0) || dt != dt || dt > 1e300) return RAM_ERR_ARG;
    StepArgs a = base_args(p, q_in, q_out);
    a.mode = MODE_RESIDUAL;
    a.dt = dt;
    a.dv = dv_iface;
    a.nsub = nsub;
    a.scheme = scheme;
    return run(p, dtype, a, stream);
}

extern "C" ram_status ram_step(ram_plan plan, ram_dtype dtype, const void *q_in, void *q_out,
                               double *phase, const double *v0, double dt,
                               const void *dv_iface, ram_scheme scheme, const int32_t *nsub,
                               void *stream)
{
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    ram_status st = check_common(p, dtype, q_in, q_out);
    if (st != RAM_OK) return st;
    if (!v0) return RAM_ERR_ARG;
    if (scheme != RAM_DONOR && scheme != RAM_VANLEER) return RAM_ERR_ARG;
    if (!(dt >= 0.0) || dt > 1e300) return RAM_ERR_ARG;
    StepArgs a = base_args(p, q_in, q_out);
    a.mode = MODE_STEP;
    a.v0 = v0;
    a.dt = dt;
    a.phase = phase;
    a.dv = dv_iface;
    a.nsub = nsub;
    a.scheme = scheme;
    return p->a4 ? run_a4(p, dtype, a, stream) : run(p, dtype, a, stream);
}

extern "C" ram_status ram_step_adjoint(ram_plan plan, ram_dtype dtype, const void *q_in,
                                       const void *g_out, void *g_in, const double *v0,
                                       double dt, const void *dv_iface, void *g_dv,
                                       const int32_t *nsub, void *stream)
{
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    ram_status st = check_common(p, dtype, g_out, g_in);
    if (st != RAM_OK) return st;
    if (!q_in || !v0) return RAM_ERR_ARG;
    // the transpose of a linear step, or of a limited PLM / PPM step linearised at
    // q_in (RAM_ADJOINT plans); no A4
    if (p->a4 || (p->limiter && !p->adj_all)) return RAM_ERR_UNSUPPORTED;
    if (p->limiter)
        for (const RowInfo &ri : p->rows_h)
            if (ri.order == 4) return RAM_ERR_UNSUPPORTED;
    if (!(dt >= 0.0) || dt > 1e300) return RAM_ERR_ARG;
    const size_t bytes = (size_t)p->n_cells * dtype_size(dtype);
    if (overlaps(q_in, g_in, bytes)) return RAM_ERR_ARG;
    if (g_dv && (overlaps(g_dv, g_in, bytes) || overlaps(g_dv, g_out, bytes)))
        return RAM_ERR_ARG;
    StepArgs a = base_args(p, q_in, nullptr);
    a.mode = MODE_STEP;
    a.v0 = v0;
    a.dt = dt;
    a.dv = dv_iface;
    a.nsub = nsub;
    a.scheme = RAM_DONOR;
    DeviceGuard g(p->device);
    if (!g.ok) return RAM_ERR_CUDA;
    cudaError_t e = launch_adjoint(*p, dtype, a, g_out, g_in, g_dv,
                                   static_cast<cudaStream_t>(stream));
    if (e == cudaErrorNotSupported) return RAM_ERR_UNSUPPORTED;
    return e == cudaSuccess ? RAM_OK : RAM_ERR_CUDA;
}

extern "C" ram_status ram_row_mass(ram_plan plan, ram_dtype dtype, const void *q,
                                   double *mass_out, void *stream)
{
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p || !q || !mass_out || (dtype != RAM_F32 && dtype != RAM_F64)) return RAM_ERR_ARG;
    DeviceGuard g(p->device);
    if (!g.ok) return RAM_ERR_CUDA;
    cudaError_t e = launch_row_mass(*p, dtype, q, mass_out, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RAM_OK : RAM_ERR_CUDA;
}

extern "C" ram_status ram_radial_upwind(ram_plan plan, ram_dtype dtype, const void *q_in,
                                        void *q_out, const double *rf, const void *vr,
                                        double dt, ram_scheme scheme, void *stream)
{
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    ram_status st = check_common(p, dtype, q_in, q_out);
    if (st != RAM_OK) return st;
    if (!rf || !vr || (scheme != RAM_DONOR && scheme != RAM_VANLEER)) return RAM_ERR_ARG;
    if (!(dt >= 0.0) || dt > 1e300) return RAM_ERR_ARG;
    if (!(p->flags & RAM_SHARED_MESH)) return RAM_ERR_UNSUPPORTED;  // rings of one mesh
    DeviceGuard g(p->device);
    if (!g.ok) return RAM_ERR_CUDA;
    cudaError_t e = launch_radial(*p, dtype, q_in, q_out, rf, vr, dt, scheme,
                                  static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? RAM_OK : RAM_ERR_CUDA;
}
