// S0 of the hot path for uniform rows: the bulk displacement of one launch and
// everything the uniform-row kernels derive from it, computed once per row in
// FP64 (one thread per row, all rows in parallel).
//
//   s    = v0 dt (ram_step), the given shift (ram_shift) or 0 (residual only);
//          the accumulated phase v0 t mod L is advanced by s (ram_step).
//   sig  = (s mod L) N / L in [0, N): the shift in cells, K = floor(sig) whole
//          cells and the fraction f = sig - K (Sec. 3.2.1 on a uniform mesh:
//          every shifted edge sits at offset xi = 1 - f inside its source cell).
//   c[]  = coefficients of the left partial integral at xi for the row's order:
//          PLM  G/dx = Q xi + slope (xi^2 - xi)/2,
//          PPM  G/dx = QL (xi - xi^2/2) + QR xi^2/2 + Q6 (xi^2/2 - xi^3/3), folded
//               with Q6 = 6Q - 3(QL + QR) into coefficients of QL, QR and Q,
//          order 4: Lagrange weights of the two quartics of the cumulative mass.
//   cf   = dt / (nsub dx): Courant number per unit dv of one residual sub-step.
#include <cuda_runtime.h>

#include "ram_device.cuh"

namespace ram {
namespace {

template <typename T>
__global__ void __launch_bounds__(128) k_params(StepArgs a, int n_rows, RowParams<T> *out)
{
    // the row kernels that follow may start now; they wait for these results
    pdl_trigger();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    const RowInfo row = a.rows[r];
    const int N = row.n;
    RowParams<T> P;
    P.cell_off = row.cell_off;
    P.n = N;
    const double sft = row_shift(a, r);
    if (a.mode == MODE_STEP && a.phase != nullptr)
        a.phase[r] = reduce_mod_rcp(a.phase[r] + sft, row.period, row.inv_period);
    const double sred = reduce_mod_rcp(sft, row.period, row.inv_period);
    // fixed-point shift for rows with their own mesh: nodes are stored as fractions
    // of the period in units of 2^-64, so x - s and the periodic wrap are exact
    // integer arithmetic
    {
        const double t = sred * row.inv_period;  // in [0, 1]
        P.sfix = (t >= 1.0) ? 0ull : __double2ull_rn(t * 18446744073709551616.0);
    }
    double sig = sred * row.cells_per_length;
    if (sig >= (double)N) sig -= (double)N;
    const double Kd = floor(sig);
    const double f = sig - Kd;
    P.K = (int)Kd;
    P.whole = (f == 0.0);
    const double xi = 1.0 - f;
    for (int j = 0; j < 5; ++j) P.c[j] = T(0);
    if (row.order == 2) {
        P.c[0] = (T)xi;
        P.c[1] = (T)(0.5 * (xi * xi - xi));
    } else if (row.order == 3) {
        const double c0 = xi - 0.5 * xi * xi, c1 = 0.5 * xi * xi;
        const double c6 = 0.5 * xi * xi - xi * xi * xi * (1.0 / 3.0);
        P.c[0] = (T)(c0 - 3.0 * c6);
        P.c[1] = (T)(c1 - 3.0 * c6);
        P.c[2] = (T)(6.0 * c6);
    } else {
        double c[5];
        quartic_coeffs_u(xi, c);
        for (int j = 0; j < 5; ++j) P.c[j] = (T)c[j];
    }
    const bool has_dv = (a.mode != MODE_SHIFT) && (a.dv != nullptr);
    int nsub = 0;
    P.cf = T(0);
    if (has_dv) {
        nsub = a.nsub ? a.nsub[r] : 1;
        if (nsub < 1 || nsub > RAM_MAX_NSUB) {
            atomicOr(a.err, ERR_NSUB);
            nsub = nsub < 1 ? 1 : RAM_MAX_NSUB;
        }
        P.cf = row.uniform ? (T)(a.dt * row.cells_per_length * inv_small(nsub))
                           : (T)(a.dt * inv_small(nsub));
    }
    P.nsub = nsub;
    out[r] = P;
}

}  // namespace

cudaError_t launch_params(const Plan &p, ram_dtype dt, const StepArgs &a, cudaStream_t s)
{
    const int threads = 128;
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
