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

#include <cstdint>
#include <vector>

#include "ram_device.cuh"

namespace ram {
namespace {

constexpr int kMaxHalo = 2 * RAM_MAX_NSUB;  // residual halo (cells per side)

template <typename T, int ORDER>
__global__ void __launch_bounds__(1024)
    k_uniform(StepArgs a, int tile_cap, const RowParams<T> *pars)
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

    const Tile tile = a.tiles[blockIdx.x];
    const RowInfo row = a.rows[tile.row];
    const int N = row.n;
    const int tid = threadIdx.x, nth = blockDim.x;
    // the row's shift parameters come from the parameter kernel launched just before
    pdl_wait();
    const RowParams<T> P = pars[tile.row];

    const bool residual = P.nsub > 0;
    const int nsub = P.nsub;
    const int R = (a.scheme == RAM_VANLEER) ? 2 : 1;
    const int H = nsub * R;
    const int T_out = tile.count;
    const int nq = T_out + 2 * H;       // cells of Q' on chip
    const int Wn = nq + 1 + 2 * HR;     // source cells on chip
    const long long K = P.K;
    const bool whole = P.whole != 0;    // whole-cell shift: a cyclic permutation
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
        for (int w = tid; w < Wn; w += nth) sQ[w] = qin[wrap_pos(w0 + w, N)];
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
                g = q0 * P.c[0] + sl * P.c[1];
            } else if (ORDER == 3) {
                T QL, QR, Q6;
                ppm_u(sQ[w - 2], sQ[w - 1], sQ[w], sQ[w + 1], sQ[w + 2], lim, QL, QR, Q6);
                (void)Q6;  // folded: Q6 = 6Q - 3(QL + QR)
                g = QL * P.c[0] + QR * P.c[1] + sQ[w] * P.c[2];
            } else {
                g = P.c[0] * sQ[w - 2] + P.c[1] * sQ[w - 1] + P.c[2] * sQ[w] +
                    P.c[3] * sQ[w + 1] + P.c[4] * sQ[w + 2];
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
        if (nq < N) {
            for (int j = tid; j <= nq; j += nth) {
                int c = v0i + j;
                if (c >= N) c -= N;
                sV[j] = dv[c];
            }
        } else {
            for (int j = tid; j <= nq; j += nth) sV[j] = dv[wrap_pos(v0i + j, N)];
        }
        const T cf = P.cf;  // Courant number per unit dv
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
cudaError_t launch_tiles(const Plan &p, const StepArgs &a0, cudaStream_t s, const Tile *tiles,
                         const std::vector<Tile> &tiles_h)
{
    const int n = (int)tiles_h.size();
    if (n == 0) return cudaSuccess;
    StepArgs a = a0;
    a.tiles = tiles;
    a.n_tiles = n;
    int cap = 0;
    for (const Tile &t : tiles_h) cap = cap > t.count ? cap : t.count;
    constexpr int HR = (ORDER == 2) ? 1 : 2;
    const size_t wcap = cap + 2 * kMaxHalo + 1 + 2 * HR;
    const size_t qcap = cap + 2 * kMaxHalo + 1;
    const size_t smem = sizeof(T) * (2 * wcap + 4 * qcap);
    // raise the dynamic shared-memory limit once per device and size
    static size_t configured[64] = {0};
    const int dev = p.device < 64 ? p.device : 63;
    if (smem > configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_uniform<T, ORDER>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured[dev] = smem;
    }
    return launch_pdl(k_uniform<T, ORDER>, n, p.threads, smem, s, a, cap,
                      static_cast<const RowParams<T> *>(p.row_par));
}

bool aligned16(const void *ptr) { return ptr == nullptr || ((uintptr_t)ptr % 16) == 0; }

template <typename T, int ORDER>
cudaError_t launch_order(const Plan &p, const StepArgs &a, cudaStream_t s)
{
    const int d = sizeof(T) == 4 ? 0 : 1;
    const ram_dtype dt = sizeof(T) == 4 ? RAM_F32 : RAM_F64;
    // both row kernels read 16-byte vectors (or TMA bulk copies)
    const bool vec_ok = aligned16(a.q_in) && aligned16(a.dv) && aligned16(a.q_out);
    if (!vec_ok)
        return launch_tiles<T, ORDER>(p, a, s, p.tiles_uniform[ORDER], p.tiles_uniform_h[ORDER]);
    if (d == 0 && p.uniform_kernel[0] == 2 && !p.rows_seg_h[0][ORDER].empty()) {
        // streaming warps: the same rows as the warp-segment kernel (16-byte aligned,
        // at least 512 cells: no shorter than the staged window of 4 cells per lane)
        cudaError_t e = launch_stream(p, a, s, ORDER);
        if (e != cudaSuccess) return e;
        return launch_tiles<T, ORDER>(p, a, s, p.tiles_rest_seg[d][ORDER],
                                      p.tiles_rest_seg_h[d][ORDER]);
    }
    if (p.uniform_kernel[d] == 1 && !p.rows_seg_h[d][ORDER].empty()) {
        cudaError_t e = launch_useg(p, dt, a, s, ORDER, p.rows_seg[d][ORDER],
                                    (int)p.rows_seg_h[d][ORDER].size());
        if (e != cudaSuccess) return e;
        return launch_tiles<T, ORDER>(p, a, s, p.tiles_rest_seg[d][ORDER],
                                      p.tiles_rest_seg_h[d][ORDER]);
    }
    if (p.rows_fit_h[d][ORDER].empty())
        return launch_tiles<T, ORDER>(p, a, s, p.tiles_uniform[ORDER], p.tiles_uniform_h[ORDER]);
    cudaError_t e = launch_rows(p, dt, a, s, ORDER, p.rows_fit_pos[d][ORDER],
                                (int)p.rows_fit_h[d][ORDER].size(), p.ncap_fit[d][ORDER]);
    if (e != cudaSuccess) return e;
    return launch_tiles<T, ORDER>(p, a, s, p.tiles_rest[d][ORDER], p.tiles_rest_h[d][ORDER]);
}

}  // namespace

int rows_kernel_max_cells(ram_dtype dt) { return dt == RAM_F32 ? 12288 : 6144; }

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
