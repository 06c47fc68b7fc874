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

#include "ram_lane.cuh"
#include "ram_tma.cuh"

namespace ram {
namespace {

__device__ __forceinline__ int wrap2(int c, int N)
{
    // c within (-2N, 2N)
    if (c < 0) c += N;
    if (c < 0) c += N;
    if (c >= N) c -= N;
    if (c >= N) c -= N;
    return c;
}

// Index i in [0, 2N) brought into [0, N): one compare for the vectors of a
// lane's window once its start is in [0, N).
__device__ __forceinline__ int wrap1(int i, int N) { return i >= N ? i - N : i; }

// One row's state for the warp-segment kernels.
template <typename T>
struct SegRow {
    int N, nsub, H4, stride, nseg, off;
    const T *qin, *dvp;
    T *qout;
};

template <typename T, int V, bool VL>
__device__ __forceinline__ void seg_row(const StepArgs &a, const RowParams<T> &P, SegRow<T> &S)
{
    constexpr int VEC = 16 / sizeof(T);
    const bool has_dv = (a.mode != MODE_SHIFT) && (a.dv != nullptr);
    S.N = P.n;
    S.nsub = P.nsub;
    // halo cells per warp end, rounded to whole vectors so that lanes stay aligned
    S.H4 = ((P.nsub * (VL ? 2 : 1) + VEC - 1) / VEC) * VEC;
    S.stride = 32 * V - 2 * S.H4;  // output cells per warp segment
    S.nseg = (S.N + S.stride - 1) / S.stride;
    S.qin = static_cast<const T *>(a.q_in) + P.cell_off;
    S.dvp = has_dv ? static_cast<const T *>(a.dv) + P.cell_off : nullptr;
    S.qout = static_cast<T *>(a.q_out) + P.cell_off;
    // source window offset inside a 16-byte vector (the same for every lane)
    S.off = ((-P.K - 1) % VEC + VEC) % VEC;
}

// Segment seg of a row: this lane's V cells.
template <typename T, int ORDER, int V, bool LIM, bool VL>
__device__ __forceinline__ void seg_step(const RowParams<T> &P, const SegRow<T> &S, int seg,
                                         int lane, T &cmax)
{
    static_assert(V % (16 / sizeof(T)) == 0, "V must be a whole number of 16-byte vectors");
    constexpr int VEC = 16 / sizeof(T);
    using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    const int N = S.N, nsub = S.nsub, H4 = S.H4, stride = S.stride, off = S.off;
    const T *qin = S.qin;
    const T *dvp = S.dvp;
    T *qout = S.qout;
    constexpr bool lim = LIM;
    constexpr bool vl = VL;
    const int out0 = seg * stride;               // first output cell of the segment
    const int m0 = out0 - H4 + lane * V;         // this lane's first cell (may wrap)
    // ---- source window: cells p0-2 .. p0+V+2, p0 = m0 - K - 1 ----
    const int p0 = m0 - P.K - 1;
    const int base = p0 - off - VEC;             // vector aligned, <= p0 - 2
    constexpr int NW = V + 3 * VEC;              // loaded cells base .. base+NW-1
    T w[NW];
    Vec raw[NW / VEC];
    // warp-uniform: when the warp's whole window lies inside the row (all but
    // the segments at the row's ends), no lane's window wraps
    const int wb = wrap2(out0 - H4 - P.K - 1 - off - VEC, N);
    if (wb + 32 * V + NW <= N) {
        const T *src = qin + wb + lane * V;
#pragma unroll
        for (int c = 0; c < NW / VEC; ++c) raw[c] = *reinterpret_cast<const Vec *>(src + c * VEC);
    } else {
        const int b0 = wrap2(base, N);
#pragma unroll
        for (int c = 0; c < NW / VEC; ++c)
            raw[c] = *reinterpret_cast<const Vec *>(qin + wrap1(b0 + c * VEC, N));
    }
#pragma unroll
    for (int c = 0; c < NW / VEC; ++c) {
        const Vec v = raw[c];
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
    if (sizeof(T) == 4)
        remap_group<T, ORDER, V>(q, P, lim, cur);
    else
        remap_group_cs<T, ORDER, V>(q, P, lim, cur);

    // ---- residual sub-steps with shuffled two-cell halos ----
    if (nsub > 0) {
        T v[V + 1];
        Vec vraw[V / VEC];
        const int wv = wrap2(out0 - H4, N);
        if (wv + 32 * V <= N) {
            const T *src = dvp + wv + lane * V;
#pragma unroll
            for (int c = 0; c < V / VEC; ++c)
                vraw[c] = *reinterpret_cast<const Vec *>(src + c * VEC);
        } else {
            const int vi = wrap2(m0, N);
#pragma unroll
            for (int c = 0; c < V / VEC; ++c)
                vraw[c] = *reinterpret_cast<const Vec *>(dvp + wrap1(vi + c * VEC, N));
        }
#pragma unroll
        for (int c = 0; c < V / VEC; ++c) {
            const Vec vv = vraw[c];
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
        const T cf = P.cf;
        if constexpr (sizeof(T) == 4) {
            // the Courant numbers of the lane's faces are the same in every
            // sub-step: formed (and checked against 1) once per segment
            float c[V];
            float cm = 0.0f;
#pragma unroll
            for (int k = 0; k < V; ++k) {
                c[k] = v[k] * cf;
                cm = fmaxf(cm, fabsf(c[k]));
            }
            cmax = fmaxf(cmax, cm);
            for (int sub = 0; sub < nsub; ++sub) residual_warp<V, VL>(cur, c);
        } else {
            v[V] = __shfl_down_sync(0xffffffffu, v[0], 1);
            for (int sub = 0; sub < nsub; ++sub) {
                T z[V + 4];
                z[0] = __shfl_up_sync(0xffffffffu, cur[V - 2], 1);
                z[1] = __shfl_up_sync(0xffffffffu, cur[V - 1], 1);
#pragma unroll
                for (int k = 0; k < V; ++k) z[k + 2] = cur[k];
                z[V + 2] = __shfl_down_sync(0xffffffffu, cur[0], 1);
                z[V + 3] = __shfl_down_sync(0xffffffffu, cur[1], 1);
                bool bad = false;
                residual_group_cs<T, V>(z, v, cf, vl, bad, cur);
                if (bad) cmax = T(2);
            }
        }
    }

    // ---- store the interior [H4, H4 + stride) of the segment, cells < N ----
    // H4, stride, out0 and N are whole vectors, so every vector of the lane is
    // either wholly stored or wholly halo: no scalar tail
    const int li0 = lane * V;                    // local index of cur[0]
#pragma unroll
    for (int c = 0; c < V / VEC; ++c) {
        const int li = li0 + c * VEC;
        if (li >= H4 && li < H4 + stride && m0 + c * VEC < N) {
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
    }
}

// LIM: limiters on; VL: van Leer residual (else donor) -- compile-time so that
// the per-cell code carries no flag tests.  One CTA per row.
template <typename T, int ORDER, int V, bool LIM, bool VL>
__global__ void __launch_bounds__(256, V * sizeof(T) <= 32 ? 3 : 2)
    k_useg(StepArgs a, const int32_t *row_ids, const RowParams<T> *pars)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const int r = row_ids[blockIdx.x];
    // the row's shift parameters come from the parameter kernel just before
    pdl_wait();
    const RowParams<T> P = pars[r];
    SegRow<T> S;
    seg_row<T, V, VL>(a, P, S);
    T cmax = T(0);
    for (int seg = warp; seg < S.nseg; seg += nwarps)
        seg_step<T, ORDER, V, LIM, VL>(P, S, seg, lane, cmax);
    if (cmax > T(1)) atomicOr(a.err, ERR_CFL);
}

// One FP32 warp segment from its raw window and dv vectors (in registers): the
// remap of the lane's V cells (its source cells start at w[off + 2]), the
// residual sub-steps with shuffled neighbours, and the store of the segment's
// interior [H4, H4 + stride) (whole vectors; the cells past N belong to no
// segment).  Shared by the register-prefetch and shared-memory-ring kernels.
template <int ORDER, int V, bool LIM, bool VL>
__device__ __forceinline__ void seg_compute_f32(const RowParams<float> &P, int N, int nsub,
                                                int H4, int stride, int off, bool use_dv,
                                                int seg, int lane,
                                                const float4 (&xw)[(V + 12) / 4],
                                                const float4 (&xv)[V / 4], float *qout,
                                                float &cmax)
{
    constexpr int VEC = 4, NW = V + 12;
    const int out0 = seg * stride;
    const int m0 = out0 - H4 + lane * V;
    float w[NW];
#pragma unroll
    for (int c = 0; c < NW / VEC; ++c) {
        w[4 * c] = xw[c].x;
        w[4 * c + 1] = xw[c].y;
        w[4 * c + 2] = xw[c].z;
        w[4 * c + 3] = xw[c].w;
    }
    float q[V + 5];
    switch (off) {
    case 0:
#pragma unroll
        for (int j = 0; j < V + 5; ++j) q[j] = w[j + 2];
        break;
    case 1:
#pragma unroll
        for (int j = 0; j < V + 5; ++j) q[j] = w[j + 3];
        break;
    case 2:
#pragma unroll
        for (int j = 0; j < V + 5; ++j) q[j] = w[j + 4];
        break;
    default:
#pragma unroll
        for (int j = 0; j < V + 5; ++j) q[j] = w[j + 5];
        break;
    }
    float cur[V];
    if constexpr (ORDER == 3)
        remap_warp3<V>(q, P, LIM, cur);
    else
        remap_group<float, ORDER, V>(q, P, LIM, cur);
    if (use_dv) {
        float v[V];
#pragma unroll
        for (int c = 0; c < V / VEC; ++c) {
            v[4 * c] = xv[c].x;
            v[4 * c + 1] = xv[c].y;
            v[4 * c + 2] = xv[c].z;
            v[4 * c + 3] = xv[c].w;
        }
        float cm = 0.0f;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            v[k] *= P.cf;  // the faces' Courant numbers, the same in every sub-step
            cm = fmaxf(cm, fabsf(v[k]));
        }
        cmax = fmaxf(cmax, cm);
        for (int sub = 0; sub < nsub; ++sub) residual_warp<V, VL>(cur, v);
    }
    const int li0 = lane * V;
#pragma unroll
    for (int c = 0; c < V / VEC; ++c) {
        const int li = li0 + c * VEC;
        if (li >= H4 && li < H4 + stride && m0 + c * VEC < N)
            *reinterpret_cast<float4 *>(qout + m0 + c * VEC) =
                make_float4(cur[4 * c], cur[4 * c + 1], cur[4 * c + 2], cur[4 * c + 3]);
    }
}

// The same step with the loads of a warp's next segment in flight while it
// computes the current one (two register sets, the loop unrolled by two so the
// sets swap roles without copies).  FP32 rows, 8 cells per lane.
template <int ORDER, bool LIM, bool VL>
__global__ void __launch_bounds__(256, 2)
    k_useg_pf(StepArgs a, const int32_t *row_ids, const RowParams<float> *pars)
{
    constexpr int V = 8, VEC = 4, NW = V + 12;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const bool has_dv = (a.mode != MODE_SHIFT) && (a.dv != nullptr);
    const int r = row_ids[blockIdx.x];
    pdl_wait();
    const RowParams<float> P = pars[r];
    const int N = P.n;
    const int nsub = P.nsub;
    // halo at the ends of a warp's 32 V cells, whole vectors: the residual
    // sub-steps spoil nsub (donor) or 2 nsub (van Leer) cells at each end, and
    // the PPM remap with shared neighbours (remap_warp3) 1 more on the left and 2
    // on the right; H4 cells on the left, HR on the right are not stored
    const int spoil = nsub * (VL ? 2 : 1);
    const int H4 = ((spoil + (ORDER == 3 ? 1 : 0) + VEC - 1) / VEC) * VEC;
    const int HR = ((spoil + (ORDER == 3 ? 2 : 0) + VEC - 1) / VEC) * VEC;
    const int stride = 32 * V - H4 - HR;
    const int nseg = (N + stride - 1) / stride;
    const float *qin = static_cast<const float *>(a.q_in) + P.cell_off;
    const float *dvp = has_dv ? static_cast<const float *>(a.dv) + P.cell_off : nullptr;
    float *qout = static_cast<float *>(a.q_out) + P.cell_off;
    const int off = ((-P.K - 1) % VEC + VEC) % VEC;
    const bool use_dv = has_dv && nsub > 0;
    float cmax = 0.0f;

    struct Raw {
        float4 w[NW / VEC];
        float4 v[V / VEC];
    };
    auto load = [&](int seg, Raw &x) {
        const int w0 = seg * stride - H4;  // the warp's first cell
        const int m0 = w0 + lane * V;
        // warp-uniform: no lane's window wraps unless the segment is at a row end
        const int wb = wrap2(w0 - P.K - 1 - off - VEC, N);
        if (wb + 32 * V + NW <= N) {
            const float *src = qin + wb + lane * V;
#pragma unroll
            for (int c = 0; c < NW / VEC; ++c)
                x.w[c] = *reinterpret_cast<const float4 *>(src + c * VEC);
        } else {
            const int b0 = wrap2(m0 - P.K - 1 - off - VEC, N);
#pragma unroll
            for (int c = 0; c < NW / VEC; ++c)
                x.w[c] = *reinterpret_cast<const float4 *>(qin + wrap1(b0 + c * VEC, N));
        }
        if (use_dv) {
            const int wv = wrap2(w0, N);
            if (wv + 32 * V <= N) {
                const float *src = dvp + wv + lane * V;
#pragma unroll
                for (int c = 0; c < V / VEC; ++c)
                    x.v[c] = *reinterpret_cast<const float4 *>(src + c * VEC);
            } else {
                const int vi = wrap2(m0, N);
#pragma unroll
                for (int c = 0; c < V / VEC; ++c)
                    x.v[c] = *reinterpret_cast<const float4 *>(dvp + wrap1(vi + c * VEC, N));
            }
        }
    };
    auto compute = [&](int seg, const Raw &x) {
        seg_compute_f32<ORDER, V, LIM, VL>(P, N, nsub, H4, stride, off, use_dv, seg, lane, x.w,
                                           x.v, qout, cmax);
    };

    Raw ra, rb;
    int seg = warp;
    if (seg < nseg) load(seg, ra);
    for (; seg < nseg; seg += 2 * nwarps) {
        const int s1 = seg + nwarps, s2 = seg + 2 * nwarps;
        if (s1 < nseg) load(s1, rb);
        compute(seg, ra);
        if (s2 < nseg) load(s2, ra);
        if (s1 < nseg) compute(s1, rb);
    }
    if (cmax > 1.0f) atomicOr(a.err, ERR_CFL);
}

// Shared-memory layout of the ring kernel, per warp: S stages, each the warp
// segment's source window (32 V + 12 cells from a 16-byte aligned start)
// followed by its dv (32 V cells).  One stage: the warp reads it into registers
// before computing, so the copies of its next segment already overlap the
// computation of the current one; more stages in flight made the step slower
// (the segments a warp claims ahead are no longer handed out to the warps that
// finish first: 15.4, 15.9, 17.0 and 18.1 µs per step for 1-4 stages on the
// 1024 x 4096 disk).
template <int V>
struct RingLayout {
    static constexpr int WQ = 32 * V + 12;
    static constexpr int WV = 32 * V;
    static constexpr int S = 1;
    static constexpr int stage_floats = WQ + WV;
    static constexpr int warp_bytes = S * stage_floats * 4;
    static_assert((stage_floats * 4) % 16 == 0, "16-byte aligned stages");
};

// The same step with each warp's segments staged through a ring of S shared-memory
// stages filled by asynchronous 16-byte copies (the data does not pass through
// registers until the segment is computed), so that S segments per warp are in
// flight.  A warp reads a stage into registers, refills it at once with the
// copies of its next segment and computes.  The warps of a row take its segments
// from a counter in shared memory as they issue the copies, so a warp on a
// crowded scheduler takes fewer of them and the row's CTA finishes with its
// warps.  The row's shift parameters are formed in the kernel
// (shift_params_two_float), so no parameter kernel runs before it when every row
// of the step takes this kernel; the phase is then advanced here too
// (a.row_phase).  FP32 rows of at least 32 V + 12 cells.
template <int ORDER, int V, bool LIM, bool VL>
__global__ void __launch_bounds__(256, 3)
    k_useg_ring(StepArgs a, const int32_t *row_ids)
{
    using L = RingLayout<V>;
    constexpr int VEC = 4, NW = V + 12;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int seg_next;                // the row's next segment to hand out
    __shared__ int seg_slot[8][L::S];       // segment held by each warp's stages
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *ring = reinterpret_cast<float *>(smem_raw + (size_t)warp * L::warp_bytes);
    int *slot = seg_slot[warp];

    const bool has_dv = (a.mode != MODE_SHIFT) && (a.dv != nullptr);
    const int r = row_ids[blockIdx.x];
    const RowInfo row = a.rows[r];  // plan data: readable before the previous kernel ends
    if (threadIdx.x == 0) seg_next = 0;
    pdl_wait();
    // every warp forms the row's shift parameters itself, in two-float arithmetic
    // (no FP64 instruction, no parameter kernel before this one)
    RowParams<float> P;
    shift_params_two_float(a, row, r, threadIdx.x == 0, P);
    if (a.row_phase && threadIdx.x == 0) advance_phase(a, row, r);
    const int N = P.n;
    const int nsub = P.nsub;
    // halo at the ends of a warp's 32 V cells, whole vectors: the residual
    // sub-steps spoil nsub (donor) or 2 nsub (van Leer) cells at each end, and
    // the PPM remap with shared neighbours (remap_warp3) 1 more on the left and 2
    // on the right; H4 cells on the left, HR on the right are not stored
    const int spoil = nsub * (VL ? 2 : 1);
    const int H4 = ((spoil + (ORDER == 3 ? 1 : 0) + VEC - 1) / VEC) * VEC;
    const int HR = ((spoil + (ORDER == 3 ? 2 : 0) + VEC - 1) / VEC) * VEC;
    const int stride = 32 * V - H4 - HR;
    const int nseg = (N + stride - 1) / stride;
    const float *qin = static_cast<const float *>(a.q_in) + P.cell_off;
    const float *dvp = has_dv ? static_cast<const float *>(a.dv) + P.cell_off : nullptr;
    float *qout = static_cast<float *>(a.q_out) + P.cell_off;
    const int off = ((-P.K - 1) % VEC + VEC) % VEC;
    const bool use_dv = has_dv && nsub > 0;
    __syncthreads();  // seg_next is set

    // copies of the segment this warp takes next into stage i % S, one commit
    // group per stage use (empty once the row's segments are all handed out, so
    // that group i is always the (i+1)-th).  The window starts at the 16-byte
    // aligned cell wb in [0, N); a vector past the row's end comes from its
    // start.  Lane l copies the 16-byte chunks l, l + 32, ... of the window and
    // of the dv range.
    const uint32_t ring_s = smem_u32(ring) + 16u * lane;
    constexpr uint32_t kStageBytes = L::stage_floats * 4;
    const int wshift = P.K + 1 + off + VEC;  // window start = w0 - wshift
    const float *const qlane = qin + 4 * lane;
    const float *const dlane = use_dv ? dvp + 4 * lane : nullptr;
    auto issue = [&](int i) {
        int seg = 0;
        if (lane == 0) seg = atomicAdd(&seg_next, 1);
        seg = __shfl_sync(0xffffffffu, seg, 0);
        slot[i % L::S] = seg;  // every lane writes the same value
        if (seg < nseg) {
            const int w0 = seg * stride - H4;
            const uint32_t sq = ring_s + (uint32_t)(i % L::S) * kStageBytes;
            const int wb = wrap2(w0 - wshift, N);
            if (wb + L::WQ <= N) {
                const float *src = qlane + wb;
#pragma unroll
                for (int j = 0; j < (L::WQ / 4 + 31) / 32; ++j)
                    if (lane + 32 * j < L::WQ / 4) cp_async16_s(sq + 512u * j, src + 128 * j);
            } else {
#pragma unroll
                for (int j = 0; j < (L::WQ / 4 + 31) / 32; ++j) {
                    const int c = lane + 32 * j;
                    if (c < L::WQ / 4) cp_async16_s(sq + 512u * j, qin + wrap1(wb + 4 * c, N));
                }
            }
            if (use_dv) {
                const int wv = wrap2(w0, N);
                const uint32_t sv = sq + L::WQ * 4;
                if (wv + L::WV <= N) {
                    const float *src = dlane + wv;
#pragma unroll
                    for (int j = 0; j < L::WV / 128; ++j) cp_async16_s(sv + 512u * j, src + 128 * j);
                } else {
#pragma unroll
                    for (int j = 0; j < L::WV / 128; ++j)
                        cp_async16_s(sv + 512u * j, dvp + wrap1(wv + 4 * (lane + 32 * j), N));
                }
            }
        }
        cp_async_commit();
    };

#pragma unroll
    for (int i = 0; i < L::S; ++i) issue(i);
    float cmax = 0.0f;
    // this lane's cells in a stage: window floats lane V .., dv floats WQ + lane V ..
    const uint32_t lds0 = smem_u32(ring) + 4u * V * lane;
    for (int i = 0;; ++i) {
        // the stages are used in the order they were filled: once a stage holds no
        // segment, no later one does
        const int seg = slot[i % L::S];
        if (seg >= nseg) break;
        // S + i groups committed; segment i's is complete once at most S - 1 remain
        cp_async_wait<L::S - 1>();
        __syncwarp();
        const uint32_t sq = lds0 + (uint32_t)(i % L::S) * kStageBytes;
        float4 xw[NW / VEC], xv[V / VEC];
#pragma unroll
        for (int c = 0; c < NW / VEC; ++c) xw[c] = lds128(sq + 16u * c);
        if (use_dv) {
#pragma unroll
            for (int c = 0; c < V / VEC; ++c) xv[c] = lds128(sq + L::WQ * 4 + 16u * c);
        }
        // every lane has read the stage: refill it with the warp's next segment
        __syncwarp();
        issue(i + L::S);
        seg_compute_f32<ORDER, V, LIM, VL>(P, N, nsub, H4, stride, off, use_dv, seg, lane, xw,
                                           xv, qout, cmax);
    }
    cp_async_wait<0>();
    if (cmax > 1.0f) atomicOr(a.err, ERR_CFL);
}

template <typename T, int ORDER, int V>
cudaError_t launch_useg_v(const StepArgs &a, cudaStream_t s, int threads, const int32_t *row_ids,
                          int n_rows,
                          const RowParams<T> *par)
{
    const bool lim = a.limiter != 0, vl = a.scheme == RAM_VANLEER;
    if (lim && vl)
        return launch_pdl(k_useg<T, ORDER, V, true, true>, n_rows, threads, 0, s, a, row_ids, par);
    if (lim)
        return launch_pdl(k_useg<T, ORDER, V, true, false>, n_rows, threads, 0, s, a, row_ids, par);
    if (vl)
        return launch_pdl(k_useg<T, ORDER, V, false, true>, n_rows, threads, 0, s, a, row_ids, par);
    return launch_pdl(k_useg<T, ORDER, V, false, false>, n_rows, threads, 0, s, a, row_ids, par);
}

template <int ORDER>
cudaError_t launch_useg_pf(const StepArgs &a, cudaStream_t s, int threads, const int32_t *row_ids,
                           int n_rows,
                           const RowParams<float> *par)
{
    const bool lim = a.limiter != 0, vl = a.scheme == RAM_VANLEER;
    if (lim && vl)
        return launch_pdl(k_useg_pf<ORDER, true, true>, n_rows, threads, 0, s, a, row_ids, par);
    if (lim)
        return launch_pdl(k_useg_pf<ORDER, true, false>, n_rows, threads, 0, s, a, row_ids, par);
    if (vl)
        return launch_pdl(k_useg_pf<ORDER, false, true>, n_rows, threads, 0, s, a, row_ids, par);
    return launch_pdl(k_useg_pf<ORDER, false, false>, n_rows, threads, 0, s, a, row_ids, par);
}

template <int ORDER, int V, bool LIM, bool VL>
cudaError_t launch_ring_k(const Plan &p, const StepArgs &a, cudaStream_t s, int threads,
                          const int32_t *row_ids, int n_rows)
{
    const size_t smem = (size_t)(threads / 32) * RingLayout<V>::warp_bytes;
    static bool configured[64] = {false};
    const int dev = p.device < 64 ? p.device : 63;
    if (!configured[dev]) {
        // the most any launch asks for (8 warps); the kernel's static arrays come on top
        cudaError_t e = cudaFuncSetAttribute(k_useg_ring<ORDER, V, LIM, VL>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             8 * RingLayout<V>::warp_bytes);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    return launch_pdl(k_useg_ring<ORDER, V, LIM, VL>, n_rows, threads, smem, s, a, row_ids);
}

template <int ORDER, int V>
cudaError_t launch_useg_ring(const Plan &p, const StepArgs &a, cudaStream_t s, int threads,
                             const int32_t *row_ids, int n_rows)
{
    const bool lim = a.limiter != 0, vl = a.scheme == RAM_VANLEER;
    if (lim && vl) return launch_ring_k<ORDER, V, true, true>(p, a, s, threads, row_ids, n_rows);
    if (lim) return launch_ring_k<ORDER, V, true, false>(p, a, s, threads, row_ids, n_rows);
    if (vl) return launch_ring_k<ORDER, V, false, true>(p, a, s, threads, row_ids, n_rows);
    return launch_ring_k<ORDER, V, false, false>(p, a, s, threads, row_ids, n_rows);
}

template <int ORDER>
cudaError_t launch_useg_f32(const Plan &p, const StepArgs &a, cudaStream_t s, int threads,
                            const int32_t *row_ids, int n_rows, const RowParams<float> *par)
{
    switch (p.seg_variant) {
    case 1: return launch_useg_pf<ORDER>(a, s, threads, row_ids, n_rows, par);
    case 2: return launch_useg_ring<ORDER, 8>(p, a, s, threads, row_ids, n_rows);
    default: return launch_useg_v<float, ORDER, 8>(a, s, threads, row_ids, n_rows, par);
    }
}

}  // namespace

// Rows for this kernel: the plan's warp-segment list (16-byte aligned rows of at
// least 512 cells, so that a lane's window wraps the row at most once); 8 (FP32)
// or 4 (FP64) cells per lane.  FP32 takes the plan's variant: 0 one segment in
// flight per warp, 1 the next segment's loads in flight in registers, 2 a ring of
// shared-memory stages per warp (with the shift parameters formed in the kernel).
cudaError_t launch_useg(const Plan &p, ram_dtype dt, const StepArgs &a, cudaStream_t s,
                        int order, const int32_t *row_ids, int n_rows)
{
    if (n_rows == 0) return cudaSuccess;
    // warps per row CTA: a row's segments take ceil(segments / warps) rounds and the
    // rows ceil(rows / resident CTAs) waves; the plan's choice trades the two
    const int threads = 32 * p.seg_warps;
    const RowParams<float> *pf = static_cast<const RowParams<float> *>(p.row_par);
    const RowParams<double> *pd = static_cast<const RowParams<double> *>(p.row_par);
    if (dt == RAM_F32) {
        if (order == 2) return launch_useg_f32<2>(p, a, s, threads, row_ids, n_rows, pf);
        if (order == 3) return launch_useg_f32<3>(p, a, s, threads, row_ids, n_rows, pf);
        return launch_useg_f32<4>(p, a, s, threads, row_ids, n_rows, pf);
    }
    if (order == 2) return launch_useg_v<double, 2, 4>(a, s, threads, row_ids, n_rows, pd);
    if (order == 3) return launch_useg_v<double, 3, 4>(a, s, threads, row_ids, n_rows, pd);
    return launch_useg_v<double, 4, 4>(a, s, threads, row_ids, n_rows, pd);
}

}  // namespace ram
