// S0 of the hot path: the shift parameters of every row for one launch
// (shift_params: K whole cells, the fraction's partial-integral coefficients,
// the residual Courant factor, the phase update), computed in FP64 by one thread
// per row, for the kernels that read them from plan memory.
#include <cuda_runtime.h>

#include "ram_device.cuh"

namespace ram {
namespace {

template <typename T>
__global__ void __launch_bounds__(32) k_params(StepArgs a, int n_rows, RowParams<T> *out)
{
    // the row kernels that follow may start now; they wait for these results
    pdl_trigger();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    RowParams<T> P;
    shift_params<T>(a, a.rows[r], r, true, P);
    out[r] = P;
}

}  // namespace

cudaError_t launch_params(const Plan &p, ram_dtype dt, const StepArgs &a, cudaStream_t s)
{
    // one warp per CTA: the FP64 work of the rows spreads over many SMs
    const int threads = 32;
    const int blocks = (p.n_rows + threads - 1) / threads;
    if (dt == RAM_F32)
        k_params<float><<<blocks, threads, 0, s>>>(a, p.n_rows,
                                                   static_cast<RowParams<float> *>(p.row_par));
    else
        k_params<double><<<blocks, threads, 0, s>>>(a, p.n_rows,
                                                    static_cast<RowParams<double> *>(p.row_par));
    return cudaGetLastError();
}

}  // namespace ram
