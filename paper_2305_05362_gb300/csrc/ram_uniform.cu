// Fused RAM step on rows with equal widths (the phi rings of a disk, uniform
// lines).  On such a row the shifted edges all sit at the same offset inside
// their source cells (Sec. 3.2.1 with u(x) affine), so the edge index is O(1)
// per row and every output cell takes the right part of one source cell and the
// left part of the next (Eq. 18 with p(i+1) = p(i) + 1): the prefix sum of the
// masses telescopes to the single whole mass M_{p(i)}.
//
// One CTA per tile of output cells.  The source window (tile + residual halo +
// reconstruction halo, cyclic) is staged in shared memory; the shifted field Q'
// and the residual sub-steps (Eq. 6) stay on chip; the tile is written once.
#include <cuda_runtime.h>

#include "ram_device.cuh"

namespace ram {
namespace {

constexpr int kMaxHalo = 2 * RAM_MAX_NSUB;  // residual halo (cells per side)

template <typename T, int ORDER>
__global__ void __launch_bounds__(1024) k_uniform(StepArgs a, int tile_cap)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int HR = (ORDER == 2) ? 1 : 2;  // reconstruction halo
    const int wcap = tile_cap + 2 * kMaxHalo + 1 + 2 * HR;
    const int qcap = tile_cap + 2 * kMaxHalo + 1;
    T *sQ = reinterpret_cast<T *>(smem_raw);  // source window
    T *sA = sQ + wcap;                        // left partial of every source cell
    T *sP = sA + wcap;                        // Q' (ping)
    T *sP2 = sP + qcap;                       // pong
    T *sV = sP2 + qcap;                       // dv at interfaces
    T *sF = sV + qcap;                        // fluxes

    __shared__ long long s_K;
    __shared__ double s_f;
    __shared__ T s_c[5];

    const Tile tile = a.tiles[blockIdx.x];
    const RowInfo row = a.rows[tile.row];
    const int N = row.n;
    const int tid = threadIdx.x, nth = blockDim.x;

    if (tid == 0) {
        const double s = row_shift(a, tile.row);
        if (a.mode == MODE_STEP && a.phase != nullptr && tile.start == 0)
            a.phase[tile.row] = reduce_mod(a.phase[tile.row] + s, row.period);
        // reduce the shift modulo the period first (a whole number of periods is
        // then exactly no shift), then express it in cells: K whole cells plus a
        // fraction f in [0, 1)
        double sig = __dmul_rn(reduce_mod(s, row.period), row.cells_per_length);
        if (sig >= (double)N) sig -= (double)N;
        const double Kd = floor(sig);
        s_K = (long long)Kd;
        s_f = sig - Kd;
        // source offset of every shifted edge inside its cell, in widths
        const double xi = 1.0 - s_f;
        if (ORDER == 2) {
            s_c[0] = (T)xi;
            s_c[1] = (T)(0.5 * (xi * xi - xi));
        } else if (ORDER == 3) {
            // g(xi) = QL (xi - xi^2/2) + QR xi^2/2 + Q6 (xi^2/2 - xi^3/3)
            s_c[0] = (T)(xi - 0.5 * xi * xi);
            s_c[1] = (T)(0.5 * xi * xi);
            s_c[2] = (T)(0.5 * xi * xi - xi * xi * xi / 3.0);
        } else {
            double c[5];
            quartic_coeffs_u(xi, c);
            for (int k = 0; k < 5; ++k) s_c[k] = (T)c[k];
        }
    }
    __syncthreads();

    const bool residual = (a.mode != MODE_SHIFT) && (a.dv != nullptr);
    int nsub = 0;
    if (residual) {
        nsub = a.nsub ? a.nsub[tile.row] : 1;
        if (nsub < 1 || nsub > RAM_MAX_NSUB) {
            if (tid == 0) atomicOr(a.err, ERR_NSUB);
            nsub = nsub < 1 ? 1 : RAM_MAX_NSUB;
        }
    }
    const int R = (a.scheme == RAM_VANLEER) ? 2 : 1;
    const int H = nsub * R;
    const int T_out = tile.count;
    const int nq = T_out + 2 * H;       // cells of Q' on chip
    const int Wn = nq + 1 + 2 * HR;     // source cells on chip
    const long long K = s_K;
    const bool whole = (s_f == 0.0);    // whole-cell shift: a cyclic permutation
    const T *qin = static_cast<const T *>(a.q_in) + row.cell_off;
    T *qout = static_cast<T *>(a.q_out) + row.cell_off;

    // stage the source window: cells start - H - K - 1 - HR + w (cyclic)
    const int w0 = wrap_index((int64_t)tile.start - H - K - 1 - HR, N);
    if (Wn <= N) {
        for (int w = tid; w < Wn; w += nth) {
            int c = w0 + w;
            if (c >= N) c -= N;
            sQ[w] = qin[c];
        }
    } else {
        for (int w = tid; w < Wn; w += nth) sQ[w] = qin[(w0 + w) % N];
    }
    __syncthreads();

    // left partial g_p(xi) of every source cell that an output cell touches
    if (!whole) {
        const bool lim = a.limiter != 0;
        for (int w = HR + tid; w < Wn - HR; w += nth) {
            T g;
            if (ORDER == 2) {
                const T q0 = sQ[w];
                T sl;
                if (lim)
                    sl = vl_slope_u(sQ[w - 1], q0, sQ[w + 1]);
                else
                    sl = T(0.5) * (sQ[w + 1] - sQ[w - 1]);
                g = q0 * s_c[0] + sl * s_c[1];
            } else if (ORDER == 3) {
                T QL, QR, Q6;
                ppm_u(sQ[w - 2], sQ[w - 1], sQ[w], sQ[w + 1], sQ[w + 2], lim, QL, QR, Q6);
                g = QL * s_c[0] + QR * s_c[1] + Q6 * s_c[2];
            } else {
                g = s_c[0] * sQ[w - 2] + s_c[1] * sQ[w - 1] + s_c[2] * sQ[w] +
                    s_c[3] * sQ[w + 1] + s_c[4] * sQ[w + 2];
            }
            sA[w] = g;
        }
        __syncthreads();
    }

    // Q'_m = right part of cell m-K-1 + left part of cell m-K (Eqs. 18, 26)
    for (int j = tid; j < nq; j += nth) {
        const int w = j + HR;
        sP[j] = whole ? sQ[w + 1] : (sQ[w] - sA[w]) + sA[w + 1];
    }

    T *cur = sP, *nxt = sP2;
    if (residual) {
        const T *dv = static_cast<const T *>(a.dv) + row.cell_off;
        const int v0i = wrap_index((int64_t)tile.start - H, N);
        for (int j = tid; j <= nq; j += nth) sV[j] = dv[(v0i + j) % N];
        const T cf = (T)(a.dt / nsub / row.dx);  // Courant number per unit dv
        const bool vl = (a.scheme == RAM_VANLEER);
        __syncthreads();
        for (int k = 0; k < nsub; ++k) {
            const int lo = k * R + R, hi = nq - k * R - R;  // interfaces lo..hi
            bool cfl_bad = false;
            for (int j = lo + tid; j <= hi; j += nth) {
                const T c = sV[j] * cf;
                T flux = T(0);
                if (c > T(0)) {
                    T qh = cur[j - 1];
                    if (vl) qh += T(0.5) * vl_slope_u(cur[j - 2], cur[j - 1], cur[j]) * (T(1) - c);
                    flux = c * qh;
                } else if (c < T(0)) {
                    T qh = cur[j];
                    if (vl) qh -= T(0.5) * vl_slope_u(cur[j - 1], cur[j], cur[j + 1]) * (T(1) + c);
                    flux = c * qh;
                }
                if (fabs(c) > T(1)) cfl_bad = true;
                sF[j] = flux;
            }
            if (cfl_bad) atomicOr(a.err, ERR_CFL);
            __syncthreads();
            for (int j = lo + tid; j < hi; j += nth) nxt[j] = cur[j] - (sF[j + 1] - sF[j]);
            __syncthreads();
            T *t = cur;
            cur = nxt;
            nxt = t;
        }
    } else {
        __syncthreads();
    }

    for (int i = tid; i < T_out; i += nth) qout[tile.start + i] = cur[H + i];
}

template <typename T, int ORDER>
cudaError_t launch_order(const Plan &p, const StepArgs &a0, cudaStream_t s)
{
    const int n = (int)p.tiles_uniform_h[ORDER].size();
    if (n == 0) return cudaSuccess;
    StepArgs a = a0;
    a.tiles = p.tiles_uniform[ORDER];
    a.n_tiles = n;
    int cap = 0;
    for (const Tile &t : p.tiles_uniform_h[ORDER]) cap = cap > t.count ? cap : t.count;
    constexpr int HR = (ORDER == 2) ? 1 : 2;
    const size_t wcap = cap + 2 * kMaxHalo + 1 + 2 * HR;
    const size_t qcap = cap + 2 * kMaxHalo + 1;
    const size_t smem = sizeof(T) * (2 * wcap + 4 * qcap);
    cudaError_t e = cudaFuncSetAttribute(k_uniform<T, ORDER>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_uniform<T, ORDER><<<n, p.threads, smem, s>>>(a, cap);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_uniform(const Plan &p, ram_dtype dt, const StepArgs &a, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (dt == RAM_F32) {
        if ((e = launch_order<float, 2>(p, a, s)) != cudaSuccess) return e;
        if ((e = launch_order<float, 3>(p, a, s)) != cudaSuccess) return e;
        if ((e = launch_order<float, 4>(p, a, s)) != cudaSuccess) return e;
    } else {
        if ((e = launch_order<double, 2>(p, a, s)) != cudaSuccess) return e;
        if ((e = launch_order<double, 3>(p, a, s)) != cudaSuccess) return e;
        if ((e = launch_order<double, 4>(p, a, s)) != cudaSuccess) return e;
    }
    return e;
}

}  // namespace ram
