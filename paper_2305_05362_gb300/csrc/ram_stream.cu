// Streaming RAM step for FP32 uniform rows: independent warps, each with its own
// ring of shared-memory stages filled by asynchronous copies.
//
// Work unit: a pair of consecutive warp segments of one row, 64 x V consecutive
// cells, lane l holding cells l V .. l V + V - 1 of the first segment (A) and the
// same cells of the second (B) as the two halves of float2 registers, so that
// the arithmetic runs on the packed FP32 pipe (two cells per instruction).  The
// outermost H4 cells at each end of a pair are halo for the residual sub-steps
// (a van Leer sub-step reaches two cells, a donor sub-step one; H4 rounds that
// up to whole 16-byte vectors): consecutive pairs overlap by 2 H4 cells and each
// stores only its interior.  Pair k of a row owns output cells [k U, k U + U),
// U = 64 V - 2 H4.  Each warp takes a contiguous run of the pairs of all rows
// (row-major), so a warp meets only one or two rows; their shift parameters (K
// whole cells and the fraction's partial-integral coefficients, Sec. 3.2.1 on a
// uniform mesh) come from the parameter kernel launched just before.
//
// Per pair a lane rebuilds the PPM / PLM / order-4 partials of the V + 1 source
// cells its cells need (App. A, Eq. 18), forms Q' = right part of p + left part
// of p + 1 (Eq. 26) and runs the residual sub-steps (Eq. 6) in registers, with
// the two-cell halos exchanged by warp shuffles (lane 31's A neighbours lane 0's
// B).  The PPM limiters are written in the min/max-with-sign form (the ALU pipe
// runs at half the FMA rate):
//   2 dQ   = sign(D) min(|D|, 4 |dn|, 4 |up|) when dn up > 0, else 0   (App. A.2)
//   a', b' = median(0, a, 2b), median(0, b, 2a)                         (App. A.2)
// with D = Q_{i+1} - Q_{i-1}, a = QR - Q and b = Q - QL; the second line is the
// flat / overshoot rule (a b <= 0: flat; |b| > 2|a|: QL = 3Q - 2QR; |a| > 2|b|:
// QR = 3Q - 2QL).
#include <cuda_runtime.h>

#include <cstdint>

#include "ram_lane.cuh"
#include "ram_tma.cuh"

namespace ram {

const int kStreamVCandidates[] = {4, 8};
const int kStreamVCount = 2;

namespace {

constexpr int kSWarps = 4;     // warps per CTA
constexpr int kSStages = 3;    // stages per warp
constexpr int kSHaloMax = 16;  // H4 for RAM_MAX_NSUB van Leer sub-steps
static_assert(kSHaloMax >= 2 * RAM_MAX_NSUB && kSHaloMax % 4 == 0, "halo bound");

// Shift parameters of one row (the fields the pair kernel needs).
struct RowRec {
    int64_t cell_off;  // first cell of the row in the packed arrays
    int32_t n;         // cells in the row
    int32_t K;         // whole cells of the shift
    int32_t nsub;      // residual sub-steps (0: none)
    int32_t whole;     // the shift is a whole number of cells
    int32_t delta;     // source window offset inside its first 16-byte vector
    int32_t h4;        // halo cells at each end of a pair
    float cf;          // Courant number per unit dv of one sub-step
    float k[5];        // order 3: xi, c_R, -c_L; order 2: xi, slope; order 4: weights
    int32_t pad[2];
};
static_assert(sizeof(RowRec) == 64, "row record layout");

// One staged pair: the row's parameters and the pair's cells.
struct PairRec {
    RowRec row;
    int32_t c0;      // first cell of the pair (may be negative: cyclic)
    int32_t u0, u1;  // output cells [u0, u1) stored by this pair
    int32_t pad;
};
static_assert(sizeof(PairRec) == 80, "pair record layout");

template <int V>
struct SLayout {
    static constexpr int W = 64 * V;       // cells of a pair
    static constexpr int Wq = W + 8;       // staged source cells
    static constexpr int Wv = W + 4;       // staged dv nodes
    static constexpr int stage_floats = Wq + Wv;
    // per warp: [PairRec x S][RowRec of the producer's row][stages]
    static constexpr int rec_off = 0;
    static constexpr int row_off = rec_off + 80 * kSStages;
    static constexpr int stage_off = row_off + 64;
    static constexpr int warp_bytes = stage_off + kSStages * stage_floats * 4;
    static_assert(stage_off % 16 == 0 && (stage_floats * 4) % 16 == 0 && warp_bytes % 16 == 0,
                  "16-byte aligned stages");
};

// The row's parameters as the pair kernel uses them, from the parameter kernel's
// record.
__device__ __forceinline__ void row_rec(const RowParams<float> &P, int order, bool vl, RowRec &R)
{
    R.cell_off = P.cell_off;
    R.n = P.n;
    R.K = P.K;
    R.nsub = P.nsub;
    R.whole = P.whole;
    R.delta = (-P.K - 3) & 3;
    R.h4 = ((P.nsub * (vl ? 2 : 1) + 3) / 4) * 4;
    R.cf = P.cf;
    if (order == 3) {
        R.k[0] = P.c[3];
        R.k[1] = P.c[1];
        R.k[2] = -P.c[0];
        R.k[3] = R.k[4] = 0.0f;
    } else {
#pragma unroll
        for (int j = 0; j < 5; ++j) R.k[j] = P.c[j];
    }
    R.pad[0] = R.pad[1] = 0;
}

template <int V>
__device__ __forceinline__ void load_lane(const float *s, float (&w)[V + 8])
{
#pragma unroll
    for (int c = 0; c < (V + 8) / 4; ++c) {
        const float4 f4 = *reinterpret_cast<const float4 *>(s + 4 * c);
        w[4 * c] = f4.x;
        w[4 * c + 1] = f4.y;
        w[4 * c + 2] = f4.z;
        w[4 * c + 3] = f4.w;
    }
}

template <int ORDER, int V>
__global__ void __launch_bounds__(kSWarps * 32, V == 4 ? 6 : 4)
    k_stream(StepArgs a, const int32_t *rows, int n_list, int pairs_per_row,
             const RowParams<float> *pars)
{
    static_assert(V % 4 == 0, "lanes start on 16-byte vectors");
    using L = SLayout<V>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wb = smem_raw + (size_t)warp * L::warp_bytes;
    PairRec *rec = reinterpret_cast<PairRec *>(wb + L::rec_off);
    RowRec *prow = reinterpret_cast<RowRec *>(wb + L::row_off);
    float *stages = reinterpret_cast<float *>(wb + L::stage_off);

    // this warp's contiguous run of pair slots (row-major over the list)
    const long long G = (long long)gridDim.x * kSWarps;
    const long long g = (long long)blockIdx.x * kSWarps + warp;
    const long long total = (long long)n_list * pairs_per_row;
    const int s_begin = (int)(g * total / G);
    const int s_end = (int)((g + 1) * total / G);
    const bool has_dv = (a.mode != MODE_SHIFT) && (a.dv != nullptr);
    const bool vl = a.scheme == RAM_VANLEER;
    const bool lim = a.limiter != 0;
    const float *qin = static_cast<const float *>(a.q_in);
    const float *dvin = static_cast<const float *>(a.dv);

    // the shift parameters come from the parameter kernel launched just before
    pdl_wait();

    // producer cursor: slot, its row (list index) and pair index in the row
    int ip = s_begin;
    int ri = s_begin / pairs_per_row, k = s_begin - ri * pairs_per_row;
    int rcur = -1;  // list index whose parameters prow holds
    int fp = 0;     // stages filled
    auto issue_next = [&]() {
        while (ip < s_end) {
            if (ri != rcur) {
                __syncwarp();
                if (lane == 0) {
                    RowRec t;
                    row_rec(pars[rows[ri]], ORDER, vl, t);
                    *prow = t;
                }
                __syncwarp();
                rcur = ri;
            }
            const RowRec &R = *prow;
            const int kk = k;
            ++ip;
            if (++k == pairs_per_row) {
                k = 0;
                ++ri;
            }
            const int n = R.n;
            const int U = 64 * V - 2 * R.h4;
            const int u0 = kk * U;
            if (u0 >= n) continue;  // past the end of this row
            const int st = fp % kSStages;
            const int c0 = u0 - R.h4;
            if (lane == 0) {
                rec[st].row = R;
                rec[st].c0 = c0;
                rec[st].u0 = u0;
                rec[st].u1 = min(u0 + U, n);
            }
            float *sq = stages + (size_t)st * L::stage_floats;
            // source window: the vector holding cell c0 - K - 3 onwards (cyclic)
            const float *qrow = qin + R.cell_off;
            int qs = c0 - R.K - 3 - R.delta;
            if (qs < 0) qs += n;
            if (qs < 0) qs += n;
            for (int c = lane; c < L::Wq / 4; c += 32) {
                int idx = qs + 4 * c;
                if (idx >= n) idx -= n;
                cp_async16(sq + 4 * c, qrow + idx);
            }
            if (has_dv && R.nsub > 0) {
                const float *vrow = dvin + R.cell_off;
                const int vs = c0 < 0 ? c0 + n : c0;
                for (int c = lane; c < L::Wv / 4; c += 32) {
                    int idx = vs + 4 * c;
                    if (idx >= n) idx -= n;
                    cp_async16(sq + L::Wq + 4 * c, vrow + idx);
                }
            }
            cp_async_commit();
            ++fp;
            return;
        }
    };
    for (int s = 0; s < kSStages; ++s) issue_next();

    float cmax = 0.0f;
    for (int fc = 0; fc < fp; ++fc) {
        // this stage's copies are the oldest pending group of every lane
        const int pend = fp - 1 - fc;
        if (pend >= 2)
            cp_async_wait<2>();
        else if (pend == 1)
            cp_async_wait<1>();
        else
            cp_async_wait<0>();
        __syncwarp();
        const int st = fc % kSStages;
        const PairRec P = rec[st];
        const float *sq = stages + (size_t)st * L::stage_floats;
        float2 cur[V];
        {
            float wA[V + 8], wB[V + 8];
            load_lane<V>(sq + lane * V, wA);
            load_lane<V>(sq + 32 * V + lane * V, wB);
            float2 q[V + 5];
            switch (P.row.delta) {
            case 0:
#pragma unroll
                for (int j = 0; j < V + 5; ++j) q[j] = make_float2(wA[j], wB[j]);
                break;
            case 1:
#pragma unroll
                for (int j = 0; j < V + 5; ++j) q[j] = make_float2(wA[j + 1], wB[j + 1]);
                break;
            case 2:
#pragma unroll
                for (int j = 0; j < V + 5; ++j) q[j] = make_float2(wA[j + 2], wB[j + 2]);
                break;
            default:
#pragma unroll
                for (int j = 0; j < V + 5; ++j) q[j] = make_float2(wA[j + 3], wB[j + 3]);
                break;
            }
            remap_pair<ORDER, V>(q, P.row.whole, P.row.k, lim, cur);
        }
        if (has_dv && P.row.nsub > 0) {
            const float *sv = sq + L::Wq + lane * V;
            float2 v[V + 1];
#pragma unroll
            for (int c = 0; c < V / 4; ++c) {
                const float4 fa = *reinterpret_cast<const float4 *>(sv + 4 * c);
                const float4 fb = *reinterpret_cast<const float4 *>(sv + 32 * V + 4 * c);
                v[4 * c] = make_float2(fa.x, fb.x);
                v[4 * c + 1] = make_float2(fa.y, fb.y);
                v[4 * c + 2] = make_float2(fa.z, fb.z);
                v[4 * c + 3] = make_float2(fa.w, fb.w);
            }
            v[V] = make_float2(sv[V], sv[32 * V + V]);
            residual_pair<V>(cur, v, P.row.cf, P.row.nsub, vl, lane, cmax);
        }
        // store the interior vectors [u0, u1) of both segments
        float *qo = static_cast<float *>(a.q_out) + P.row.cell_off;
#pragma unroll
        for (int c = 0; c < V / 4; ++c) {
            const int ca = P.c0 + lane * V + 4 * c;
            if (ca >= P.u0 && ca + 4 <= P.u1)
                *reinterpret_cast<float4 *>(qo + ca) =
                    make_float4(cur[4 * c].x, cur[4 * c + 1].x, cur[4 * c + 2].x, cur[4 * c + 3].x);
            const int cb = ca + 32 * V;
            if (cb >= P.u0 && cb + 4 <= P.u1)
                *reinterpret_cast<float4 *>(qo + cb) =
                    make_float4(cur[4 * c].y, cur[4 * c + 1].y, cur[4 * c + 2].y, cur[4 * c + 3].y);
        }
        // every lane has read the stage: it may be refilled
        __syncwarp();
        issue_next();
    }
    if (__any_sync(0xffffffffu, cmax > 1.0f) && lane == 0) atomicOr(a.err, ERR_CFL);
}

template <int ORDER, int V>
cudaError_t launch_stream_v(const Plan &p, const StepArgs &a, cudaStream_t s)
{
    using L = SLayout<V>;
    const int n_list = (int)p.rows_seg_h[0][ORDER].size();
    if (n_list == 0) return cudaSuccess;
    const int umin = 64 * V - 2 * kSHaloMax;
    const int pairs_per_row = (p.stream_nmax[ORDER] + umin - 1) / umin;
    const size_t smem = (size_t)kSWarps * L::warp_bytes;
    static bool configured[64] = {false};
    const int dev = p.device < 64 ? p.device : 63;
    if (!configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_stream<ORDER, V>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    int sms = 0, fit = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_stream<ORDER, V>, kSWarps * 32, smem);
    if (fit < 1) fit = 1;
    const long long total = (long long)n_list * pairs_per_row;
    long long grid = (total + kSWarps - 1) / kSWarps;
    if (grid > (long long)sms * fit) grid = (long long)sms * fit;
    return launch_pdl(k_stream<ORDER, V>, (int)grid, kSWarps * 32, smem, s, a,
                      static_cast<const int32_t *>(p.rows_seg[0][ORDER]), n_list, pairs_per_row,
                      static_cast<const RowParams<float> *>(p.row_par));
}

}  // namespace

int stream_min_cells(int v) { return 64 * v + 8; }

cudaError_t launch_stream(const Plan &p, const StepArgs &a, cudaStream_t s, int order)
{
    // a pair's staged window must not exceed its row (at most one cyclic wrap)
    const bool v8 = p.stream_v == 8 && p.stream_nmin[order] >= stream_min_cells(8);
    if (order == 2) return v8 ? launch_stream_v<2, 8>(p, a, s) : launch_stream_v<2, 4>(p, a, s);
    if (order == 3) return v8 ? launch_stream_v<3, 8>(p, a, s) : launch_stream_v<3, 4>(p, a, s);
    return v8 ? launch_stream_v<4, 8>(p, a, s) : launch_stream_v<4, 4>(p, a, s);
}

}  // namespace ram
