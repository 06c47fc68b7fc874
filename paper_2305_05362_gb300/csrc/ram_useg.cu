// RAM step on uniform rows with warp-independent segments (no staging, no
// per-phase barriers).
//
// One CTA per row.  The row's shift parameters (K whole cells and the
// partial-integral coefficients at the single edge offset, Sec. 3.2.1 on a
// uniform mesh) come ready from the parameter kernel, so every warp works alone
// from the start, with no FP64 and no barrier.  A warp covers 32 x V
// consecutive cells: each lane loads the cyclic source window of its V output
// cells straight from global memory (16-byte loads), rebuilds the PPM / PLM /
// order-4 partials (App. A, Eq. 18) and forms Q' (Eq. 26) in registers; the
// residual sub-steps (Eq. 6) exchange the two-cell halos between lanes with
// warp shuffles.  The outermost H4 cells at each end of a warp's range are halo
// (they go stale by two cells per van Leer sub-step), so consecutive warps
// overlap by 2*H4 cells and each stores only its interior.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "ram_device.cuh"

namespace ram {
namespace {

template <typename T>
__device__ __forceinline__ T half_vl2(T dl, T dr)
{
    const T p = dl * dr;
    return p > T(0) ? Num<T>::div(p, dl + dr) : T(0);
}

template <typename T>
__device__ __forceinline__ T lim_dq2(T dn, T up, bool lim)
{
    const T d = T(0.5) * (dn + up);
    if (!lim) return d;
    const T mm = fmin(fabs(dn), fabs(up));
    const T m = fmin(fabs(d), mm + mm);
    return (dn * up > T(0)) ? copysign(m, d) : T(0);
}

// Q' of V output cells from q[0..V+4] = source cells p0-2..p0+V+2 (same algebra as
// the whole-row kernel: right part of p plus left part of p+1).
template <typename T, int ORDER, int V>
__device__ __forceinline__ void remap_v(const T (&q)[V + 5], const RowParams<T> &P, bool lim,
                                        T (&out)[V])
{
    if (P.whole) {
#pragma unroll
        for (int k = 0; k < V; ++k) out[k] = q[k + 3];
        return;
    }
    T A[V + 1];
    if (ORDER == 3) {
        T dif[V + 4];
#pragma unroll
        for (int k = 0; k < V + 4; ++k) dif[k] = q[k + 1] - q[k];
        T dq[V + 3];
#pragma unroll
        for (int c = 1; c <= V + 3; ++c) dq[c - 1] = lim_dq2(dif[c - 1], dif[c], lim);
        const T sixth = T(1) / T(6);
#pragma unroll
        for (int j = 0; j <= V; ++j) {
            const T Q = q[j + 2];
            T L = fma(T(0.5), dif[j + 1], q[j + 1]) - (dq[j + 1] - dq[j]) * sixth;
            T R = fma(T(0.5), dif[j + 2], q[j + 2]) - (dq[j + 2] - dq[j + 1]) * sixth;
            if (lim) {
                const T a = R - Q, b = Q - L;
                const bool flat = a * b <= T(0);
                const bool left = fabs(b) > T(2) * fabs(a);
                const bool right = fabs(a) > T(2) * fabs(b);
                const T L2 = left ? fma(T(-2), a, Q) : L;
                const T R2 = right ? fma(T(2), b, Q) : R;
                L = flat ? Q : L2;
                R = flat ? Q : R2;
            }
            A[j] = fma(L, P.c[0], fma(R, P.c[1], Q * P.c[2]));
        }
    } else if (ORDER == 2) {
#pragma unroll
        for (int j = 0; j <= V; ++j) {
            const T dn = q[j + 2] - q[j + 1], up = q[j + 3] - q[j + 2];
            const T sl = lim ? T(2) * half_vl2(dn, up) : T(0.5) * (dn + up);
            A[j] = fma(q[j + 2], P.c[0], sl * P.c[1]);
        }
    } else {
#pragma unroll
        for (int j = 0; j <= V; ++j)
            A[j] = P.c[0] * q[j] + P.c[1] * q[j + 1] + P.c[2] * q[j + 2] + P.c[3] * q[j + 3] +
                   P.c[4] * q[j + 4];
    }
#pragma unroll
    for (int k = 0; k < V; ++k) out[k] = (q[k + 2] - A[k]) + A[k + 1];
}

__device__ __forceinline__ int wrap2(int c, int N)
{
    // c within (-2N, 2N)
    if (c < 0) c += N;
    if (c < 0) c += N;
    if (c >= N) c -= N;
    if (c >= N) c -= N;
    return c;
}

template <typename T, int ORDER, int V>
__global__ void __launch_bounds__(256, 3)
    k_useg(StepArgs a, const int32_t *row_ids, const RowParams<T> *pars)
{
    static_assert(V % (16 / sizeof(T)) == 0, "V must be a whole number of 16-byte vectors");
    constexpr int VEC = 16 / sizeof(T);
    using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const bool has_dv = (a.mode != MODE_SHIFT) && (a.dv != nullptr);
    const int r = row_ids[blockIdx.x];
    // the row's shift parameters come from the parameter kernel just before
    pdl_wait();
    const RowParams<T> P = pars[r];
    const int N = P.n;
    const int nsub = P.nsub;
    const bool lim = a.limiter != 0;
    const bool vl = a.scheme == RAM_VANLEER;
    const int R = vl ? 2 : 1;
    // halo cells per warp end, rounded to whole vectors so that lanes stay aligned
    const int H4 = ((nsub * R + VEC - 1) / VEC) * VEC;
    const int stride = 32 * V - 2 * H4;  // output cells per warp segment
    const int nseg = (N + stride - 1) / stride;
    const T *qin = static_cast<const T *>(a.q_in) + P.cell_off;
    const T *dvp = has_dv ? static_cast<const T *>(a.dv) + P.cell_off : nullptr;
    T *qout = static_cast<T *>(a.q_out) + P.cell_off;
    // source window offset inside a 16-byte vector (the same for every lane)
    const int off = ((-P.K - 1) % VEC + VEC) % VEC;
    bool cfl_bad = false;

    for (int seg = warp; seg < nseg; seg += nwarps) {
        const int out0 = seg * stride;               // first output cell of the segment
        const int m0 = out0 - H4 + lane * V;         // this lane's first cell (may wrap)
        // ---- source window: cells p0-2 .. p0+V+2, p0 = m0 - K - 1 ----
        const int p0 = m0 - P.K - 1;
        const int base = p0 - off - VEC;             // vector aligned, <= p0 - 2
        constexpr int NW = V + 3 * VEC;              // loaded cells base .. base+NW-1
        T w[NW];
#pragma unroll
        for (int c = 0; c < NW / VEC; ++c) {
            const int idx = wrap2(base + c * VEC, N);
            const Vec v = *reinterpret_cast<const Vec *>(qin + idx);
            if (sizeof(T) == 4) {
                const float4 f4 = *reinterpret_cast<const float4 *>(&v);
                w[c * VEC + 0] = (T)f4.x;
                w[c * VEC + 1] = (T)f4.y;
                w[c * VEC + 2] = (T)f4.z;
                w[c * VEC + 3] = (T)f4.w;
            } else {
                const double2 d2 = *reinterpret_cast<const double2 *>(&v);
                w[c * VEC + 0] = (T)d2.x;
                w[c * VEC + 1] = (T)d2.y;
            }
        }
        // q[j] = w[off + VEC - 2 + j]: a warp-uniform shift
        T q[V + 5];
        if (sizeof(T) == 4) {
            switch (off) {
            case 0:
#pragma unroll
                for (int j = 0; j < V + 5; ++j) q[j] = w[j + VEC - 2];
                break;
            case 1:
#pragma unroll
                for (int j = 0; j < V + 5; ++j) q[j] = w[j + VEC - 1];
                break;
            case 2:
#pragma unroll
                for (int j = 0; j < V + 5; ++j) q[j] = w[j + VEC];
                break;
            default:
#pragma unroll
                for (int j = 0; j < V + 5; ++j) q[j] = w[j + VEC + 1];
                break;
            }
        } else {
            if (off == 0) {
#pragma unroll
                for (int j = 0; j < V + 5; ++j) q[j] = w[j + VEC - 2];
            } else {
#pragma unroll
                for (int j = 0; j < V + 5; ++j) q[j] = w[j + VEC - 1];
            }
        }
        T cur[V];
        remap_v<T, ORDER, V>(q, P, lim, cur);

        // ---- residual sub-steps with shuffled two-cell halos ----
        if (nsub > 0) {
            T v[V + 1];
            const int vi = wrap2(m0, N);
#pragma unroll
            for (int c = 0; c < V / VEC; ++c) {
                const Vec vv = *reinterpret_cast<const Vec *>(dvp + wrap2(vi + c * VEC, N));
                if (sizeof(T) == 4) {
                    const float4 f4 = *reinterpret_cast<const float4 *>(&vv);
                    v[c * VEC + 0] = (T)f4.x;
                    v[c * VEC + 1] = (T)f4.y;
                    v[c * VEC + 2] = (T)f4.z;
                    v[c * VEC + 3] = (T)f4.w;
                } else {
                    const double2 d2 = *reinterpret_cast<const double2 *>(&vv);
                    v[c * VEC + 0] = (T)d2.x;
                    v[c * VEC + 1] = (T)d2.y;
                }
            }
            v[V] = __shfl_down_sync(0xffffffffu, v[0], 1);
            const T cf = P.cf;
            for (int sub = 0; sub < nsub; ++sub) {
                T z[V + 4];
                z[0] = __shfl_up_sync(0xffffffffu, cur[V - 2], 1);
                z[1] = __shfl_up_sync(0xffffffffu, cur[V - 1], 1);
#pragma unroll
                for (int k = 0; k < V; ++k) z[k + 2] = cur[k];
                z[V + 2] = __shfl_down_sync(0xffffffffu, cur[0], 1);
                z[V + 3] = __shfl_down_sync(0xffffffffu, cur[1], 1);
                T hs[V + 2];
                if (vl) {
#pragma unroll
                    for (int c = 0; c < V + 2; ++c)
                        hs[c] = half_vl2(z[c + 1] - z[c], z[c + 2] - z[c + 1]);
                }
                T F[V + 1];
#pragma unroll
                for (int k = 0; k <= V; ++k) {
                    const T c = v[k] * cf;
                    const bool pos = c > T(0);
                    const T Qu = pos ? z[k + 1] : z[k + 2];
                    T qh = Qu;
                    if (vl) {
                        const T h = pos ? hs[k] : hs[k + 1];
                        qh = Qu + h * ((pos ? T(1) : T(-1)) - c);
                    }
                    F[k] = c * qh;
                    cfl_bad |= fabs(c) > T(1);
                }
#pragma unroll
                for (int k = 0; k < V; ++k) cur[k] = z[k + 2] - (F[k + 1] - F[k]);
            }
        }

        // ---- store the interior [H4, H4 + stride) of the segment, cells < N ----
        const int li0 = lane * V;                    // local index of cur[0]
        const bool full = li0 >= H4 && li0 + V <= H4 + stride && out0 - H4 + li0 + V <= N;
        if (full) {
#pragma unroll
            for (int c = 0; c < V / VEC; ++c) {
                Vec vv;
                if (sizeof(T) == 4) {
                    float4 f4 = make_float4((float)cur[c * VEC], (float)cur[c * VEC + 1],
                                            (float)cur[c * VEC + 2], (float)cur[c * VEC + 3]);
                    vv = *reinterpret_cast<Vec *>(&f4);
                } else {
                    double2 d2 = make_double2((double)cur[c * VEC], (double)cur[c * VEC + 1]);
                    vv = *reinterpret_cast<Vec *>(&d2);
                }
                *reinterpret_cast<Vec *>(qout + m0 + c * VEC) = vv;
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const int li = li0 + k;
                const int g = out0 - H4 + li;
                if (li >= H4 && li < H4 + stride && g < N) qout[g] = cur[k];
            }
        }
    }
    if (cfl_bad) atomicOr(a.err, ERR_CFL);
}

}  // namespace

// Rows for this kernel: the plan's whole-row list (16-byte aligned rows) whose
// length is at least two warp segments; V = 8 (FP32) / 4 (FP64) cells per lane.
cudaError_t launch_useg(const Plan &p, ram_dtype dt, const StepArgs &a, cudaStream_t s,
                        int order, const int32_t *row_ids, int n_rows)
{
    if (n_rows == 0) return cudaSuccess;
    const int threads = 256;
    const RowParams<float> *pf = static_cast<const RowParams<float> *>(p.row_par);
    const RowParams<double> *pd = static_cast<const RowParams<double> *>(p.row_par);
    if (dt == RAM_F32) {
        if (order == 2) return launch_pdl(k_useg<float, 2, 8>, n_rows, threads, 0, s, a, row_ids, pf);
        if (order == 3) return launch_pdl(k_useg<float, 3, 8>, n_rows, threads, 0, s, a, row_ids, pf);
        return launch_pdl(k_useg<float, 4, 8>, n_rows, threads, 0, s, a, row_ids, pf);
    }
    if (order == 2) return launch_pdl(k_useg<double, 2, 4>, n_rows, threads, 0, s, a, row_ids, pd);
    if (order == 3) return launch_pdl(k_useg<double, 3, 4>, n_rows, threads, 0, s, a, row_ids, pd);
    return launch_pdl(k_useg<double, 4, 4>, n_rows, threads, 0, s, a, row_ids, pd);
}

}  // namespace ram
