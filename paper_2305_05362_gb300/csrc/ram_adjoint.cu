// Transpose of one linear RAM step (limiter off, donor residual) on uniform rows
// (rows with their own mesh: ram_adjoint_nu.cu).
//
// With the limiters off the shift of a uniform row is a fixed stencil: output
// cell m takes the right part of source cell p = m-K-1 and the left part of p+1
// (Eq. 18), and the left partial A_p of the reconstruction is linear in
// Q_{p-2..p+2}, so Q'_m = sum_u beta_u Q_{m-K-1+u} (u = -2..3) with
// beta_u = [u == 0] - alpha_u + alpha_{u-1}.  Its transpose gathers
// g_in[j] = sum_u beta_u g'[j+K+1-u].  The donor residual sub-step
// Q_i <- Q_i - (F_{i+1} - F_i), F_j = c_j Q_up(j), has the transpose
// g_k <- g_k + [c_{k+1} >= 0] c_{k+1} h_{k+1} + [c_k < 0] c_k h_k with
// h_j = g_j - g_{j-1}, and dL/d dv_j = sum over sub-steps of cf Q_up(j) h_j, where
// the forward sub-step states are recomputed from the step input.  The upwind
// side at c_j = 0 is the left cell.
//
// Launch: blockIdx.y = 0 computes g_in for a tile of source cells, blockIdx.y = 1
// adds dL/d dv for the tile's interfaces (each interface in exactly one tile, so
// there are no atomics).
#include <cuda_runtime.h>

#include <vector>

#include "ram_device.cuh"

namespace ram {
namespace {

constexpr int kMaxSub = RAM_MAX_NSUB;

// alpha_{-2..2}: coefficients of Q_{p-2..p+2} in the left partial A_p (limiter off)
template <typename T, int ORDER>
__device__ __forceinline__ void alpha_coeffs(const RowParams<T> &P, T al[5])
{
    for (int s = 0; s < 5; ++s) al[s] = T(0);
    if (ORDER == 2) {
        // A = Q c0 + (Q_{p+1} - Q_{p-1})/2 c1
        al[1] = -T(0.5) * P.c[1];
        al[2] = P.c[0];
        al[3] = T(0.5) * P.c[1];
    } else if (ORDER == 3) {
        // A = QL c0 + QR c1 + Q c2 with QL = 7/12(Q_{p-1}+Q_p) - 1/12(Q_{p-2}+Q_{p+1})
        // and QR = 7/12(Q_p+Q_{p+1}) - 1/12(Q_{p-1}+Q_{p+2})
        const T a = T(7) / T(12), b = T(1) / T(12);
        al[0] = -b * P.c[0];
        al[1] = a * P.c[0] - b * P.c[1];
        al[2] = a * P.c[0] + a * P.c[1] + P.c[2];
        al[3] = -b * P.c[0] + a * P.c[1];
        al[4] = -b * P.c[1];
    } else {
        for (int s = 0; s < 5; ++s) al[s] = P.c[s];
    }
}

template <typename T, int ORDER>
__global__ void __launch_bounds__(256)
    k_adj_uniform(StepArgs a, const RowParams<T> *pars, const T *g_out, T *g_in, T *g_dv,
                  int tcap)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wcap = tcap + 2 * kMaxSub + 16;
    T *s0 = reinterpret_cast<T *>(smem_raw);  // wcap
    T *s1 = s0 + wcap;                        // wcap
    T *sv = s1 + wcap;                        // wcap + 1 (Courant numbers)
    T *st = sv + wcap + 1;                    // forward states: kMaxSub x wcap

    const Tile tile = a.tiles[blockIdx.x];
    const RowInfo row = a.rows[tile.row];
    const int N = row.n;
    const int tid = threadIdx.x, nth = blockDim.x;
    pdl_wait();
    const RowParams<T> P = pars[tile.row];
    const int nsub = P.nsub;
    const int K = P.K;
    const int A0 = tile.start, TN = tile.count;
    const T *g = g_out + row.cell_off;
    const T *dv = nsub > 0 ? static_cast<const T *>(a.dv) + row.cell_off : nullptr;
    T al[5];
    alpha_coeffs<T, ORDER>(P, al);
    T beta[6];  // beta_u for u = -2..3
    for (int u = -2; u <= 3; ++u) {
        const T am = (u - 1 >= -2 && u - 1 <= 2) ? al[u - 1 + 2] : T(0);
        const T a0 = (u >= -2 && u <= 2) ? al[u + 2] : T(0);
        beta[u + 2] = (u == 0 ? T(1) : T(0)) - a0 + am;
    }

    if (blockIdx.y == 0) {
        // ---- g_in on source cells [A0, A0+TN): g' on [A0+K-2, A0+K+TN+3) ----
        const int m0 = A0 + K - 2 - nsub;  // first cell of g_out needed
        const int nm = TN + 5 + 2 * nsub;
        for (int i = tid; i < nm; i += nth) s0[i] = g[wrap_index((int64_t)m0 + i, N)];
        if (nsub > 0)
            for (int i = tid; i <= nm; i += nth) sv[i] = dv[wrap_index((int64_t)m0 + i, N)] * P.cf;
        __syncthreads();
        T *cur = s0, *nxt = s1;
        for (int k = 0; k < nsub; ++k) {
            // valid input [k, nm-k) -> output [k+1, nm-k-1)
            for (int i = k + 1 + tid; i < nm - k - 1; i += nth) {
                const T hL = cur[i] - cur[i - 1];      // h at interface i
                const T hR = cur[i + 1] - cur[i];      // h at interface i+1
                const T cL = sv[i], cR = sv[i + 1];
                T v = cur[i];
                if (cR >= T(0)) v += cR * hR;
                if (cL < T(0)) v += cL * hL;
                nxt[i] = v;
            }
            __syncthreads();
            T *t = cur;
            cur = nxt;
            nxt = t;
        }
        // gather: g_in[j] = sum_u beta_u g'[j+K+1-u]; g'[m] sits at cur[m - m0]
        T *gi = g_in + row.cell_off;
        for (int j = tid; j < TN; j += nth) {
            const int base = (A0 + j) + K + 1 - m0;  // index of g'[j+K+1]
            T acc;
            if (P.whole) {
                acc = cur[base - 1];  // Q'_m = Q_{m-K}: g_in[j] = g'[j+K]
            } else {
                acc = T(0);
#pragma unroll
                for (int u = -2; u <= 3; ++u) acc += beta[u + 2] * cur[base - u];
            }
            gi[A0 + j] = acc;
        }
        return;
    }

    // ---- dL/d dv on interfaces [A0, A0+TN) ----
    if (nsub == 0 || g_dv == nullptr) return;
    // forward states on cells [A0-nsub, A0+TN+nsub): Q' from the step input
    const int c0 = A0 - nsub;
    const int nc = TN + 2 * nsub;
    const T *qin = static_cast<const T *>(a.q_in) + row.cell_off;
    // Q'_m = sum_u beta_u Q_{m-K-1+u}
    for (int i = tid; i < nc; i += nth) {
        const int m = c0 + i;
        T v;
        if (P.whole) {
            v = qin[wrap_index((int64_t)m - K, N)];
        } else {
            v = T(0);
#pragma unroll
            for (int u = -2; u <= 3; ++u) v += beta[u + 2] * qin[wrap_index((int64_t)m - K - 1 + u, N)];
        }
        st[i] = v;
    }
    for (int i = tid; i <= nc; i += nth) sv[i] = dv[wrap_index((int64_t)c0 + i, N)] * P.cf;
    __syncthreads();
    // forward donor sub-steps: state k+1 from state k, valid range shrinking by one
    for (int k = 0; k + 1 < nsub; ++k) {
        const T *q = st + (size_t)k * wcap;
        T *qn = st + (size_t)(k + 1) * wcap;
        for (int i = k + 1 + tid; i < nc - k - 1; i += nth) {
            const T cL = sv[i], cR = sv[i + 1];
            const T FL = cL * (cL > T(0) ? q[i - 1] : q[i]);
            const T FR = cR * (cR > T(0) ? q[i] : q[i + 1]);
            qn[i] = q[i] - (FR - FL);
        }
        __syncthreads();
    }
    // backward sweep: g^(nsub) = g_out on the same cells
    for (int i = tid; i < nc; i += nth) s0[i] = g[wrap_index((int64_t)c0 + i, N)];
    __syncthreads();
    T *cur = s0, *nxt = s1;
    T *gd = g_dv + row.cell_off;
    T acc_local[8];
    const int per = (TN + nth - 1) / nth;  // interfaces per thread (<= 8 by the launcher)
    for (int r = 0; r < 8; ++r) acc_local[r] = T(0);
    for (int k = nsub - 1; k >= 0; --k) {
        const T *q = st + (size_t)k * wcap;
        // interfaces j in [A0, A0+TN): cell index i = j - c0 (interface i, between i-1 and i)
        for (int r = 0; r < per; ++r) {
            const int jj = tid * per + r;
            if (jj < TN) {
                const int i = jj + nsub;
                const T c = sv[i];
                const T qup = (c >= T(0)) ? q[i - 1] : q[i];
                acc_local[r] += P.cf * qup * (cur[i] - cur[i - 1]);
            }
        }
        // g^(k) from g^(k+1) on the shrinking range
        const int lo = (nsub - k), hi = nc - (nsub - k);
        for (int i = lo + tid; i < hi; i += nth) {
            const T hL = cur[i] - cur[i - 1];
            const T hR = cur[i + 1] - cur[i];
            const T cL = sv[i], cR = sv[i + 1];
            T v = cur[i];
            if (cR >= T(0)) v += cR * hR;
            if (cL < T(0)) v += cL * hL;
            nxt[i] = v;
        }
        __syncthreads();
        T *t = cur;
        cur = nxt;
        nxt = t;
    }
    for (int r = 0; r < per; ++r) {
        const int jj = tid * per + r;
        if (jj < TN) gd[A0 + jj] += acc_local[r];
    }
}

template <typename T, int ORDER>
cudaError_t launch_adj_t(const Plan &p, const StepArgs &a, const void *g_out, void *g_in,
                         void *g_dv, cudaStream_t s)
{
    const std::vector<Tile> &th = p.tiles_uniform_h[ORDER];
    if (th.empty()) return cudaSuccess;
    int cap = 0;
    for (const Tile &t : th) cap = cap > t.count ? cap : t.count;
    if (cap > 256 * 8) return cudaErrorNotSupported;
    const int wcap = cap + 2 * kMaxSub + 16;
    const size_t smem = sizeof(T) * ((size_t)3 * wcap + 1 + (size_t)kMaxSub * wcap);
    if (smem > 227 * 1024) return cudaErrorNotSupported;
    static size_t configured[64] = {0};
    const int dev = p.device < 64 ? p.device : 63;
    if (smem > configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_adj_uniform<T, ORDER>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured[dev] = smem;
    }
    StepArgs b = a;
    b.tiles = p.tiles_uniform[ORDER];
    b.n_tiles = (int)th.size();
    return launch_pdl(k_adj_uniform<T, ORDER>, dim3((int)th.size(), 2), 256, smem, s, b,
                      static_cast<const RowParams<T> *>(p.row_par), static_cast<const T *>(g_out),
                      static_cast<T *>(g_in), static_cast<T *>(g_dv), cap);
}

}  // namespace

cudaError_t launch_adjoint(const Plan &p, ram_dtype dt, const StepArgs &a, const void *g_out,
                           void *g_in, void *g_dv, cudaStream_t s)
{
    // rows with their own mesh and a residual step need the plan's scratch
    const bool nonuni = p.n_uniform_rows < p.n_rows;
    if (nonuni && a.dv != nullptr && p.adj_scratch == nullptr) return cudaErrorNotSupported;
    // a limited plan: every row on the gather adjoint, linearised at the step input
    if (p.adj_all) return launch_adjoint_nu(p, dt, a, g_out, g_in, g_dv, s);
    cudaError_t e = launch_params(p, dt, a, s);
    if (e != cudaSuccess) return e;
    if (dt == RAM_F32) {
        if ((e = launch_adj_t<float, 2>(p, a, g_out, g_in, g_dv, s)) != cudaSuccess) return e;
        if ((e = launch_adj_t<float, 3>(p, a, g_out, g_in, g_dv, s)) != cudaSuccess) return e;
        if ((e = launch_adj_t<float, 4>(p, a, g_out, g_in, g_dv, s)) != cudaSuccess) return e;
    } else {
        if ((e = launch_adj_t<double, 2>(p, a, g_out, g_in, g_dv, s)) != cudaSuccess) return e;
        if ((e = launch_adj_t<double, 3>(p, a, g_out, g_in, g_dv, s)) != cudaSuccess) return e;
        if ((e = launch_adj_t<double, 4>(p, a, g_out, g_in, g_dv, s)) != cudaSuccess) return e;
    }
    return nonuni ? launch_adjoint_nu(p, dt, a, g_out, g_in, g_dv, s) : cudaSuccess;
}

}  // namespace ram
