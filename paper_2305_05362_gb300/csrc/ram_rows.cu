// Persistent, warp-specialised RAM step for uniform rows that fit in shared
// memory (the rings of a disk).
//
// Persistent CTAs loop over their rows.  Warp 0 is the producer: it issues TMA
// bulk copies of the row's Q and dv (plus cyclic halos) into a shared-memory ring
// of stages guarded by mbarriers, and stages the row's shift parameters (K whole
// cells, the fraction's partial-integral coefficients; computed in FP64 by the
// parameter kernel, Sec. 3.2.1 on a uniform mesh).  The consumer warps never
// touch FP64: each thread owns V consecutive output cells, rebuilds the
// PPM/PLM/order-4 partials of the V+1 source cells it needs from the staged row
// (App. A, Eq. 18), forms Q' = right part of p + left part of p+1 (Eq. 26), and
// runs the residual sub-steps (Eq. 6) through two ping-pong row buffers.  Every
// wait on an mbarrier is bounded; a wait that runs out sets the error word.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "ram_device.cuh"
#include "ram_lane.cuh"
#include "ram_tma.cuh"

namespace ram {
namespace {

// Cyclic halos.  A thread owning cells m0..m0+V-1 reads the staged row at
// source cells p0-2 .. p0+V+2 (p0 in [0, N)) and the ping-pong buffers at
// m0-2 .. m0+V+1 (m0 in [0, N)), so the staged halo must hold V+2 cells and the
// ping-pong halo V+1 cells beyond N (checked per V at compile time).
constexpr int kHaloS = 24;
constexpr int kHaloP = 16;
constexpr int kMaxStages = 3;
constexpr int kMaxStagesH = 3;

constexpr int kBatch = 32;  // rows whose parameters the producer warp computes at once
// shared-memory header: barriers, the row parameters and the consumers' abort flag
constexpr int kHeader = (6 * 8 + (kMaxStagesH + kBatch) * 80 + 4 + 127) / 128 * 128;

// Write V results of the group starting at m0 into a ping-pong row buffer, with
// the cyclic halo copies of the first and last kHaloP cells.
template <typename T, int V>
__device__ __forceinline__ void put_group(T *buf, int m0, int N, const T (&out)[V])
{
    if (m0 >= kHaloP && m0 + V <= N - kHaloP) {
#pragma unroll
        for (int j = 0; j < V; ++j) buf[m0 + j] = out[j];
        return;
    }
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const int m = m0 + j;
        if (m < N) {
            buf[m] = out[j];
            if (m < kHaloP) buf[N + m] = out[j];
            if (m >= N - kHaloP) buf[m - N] = out[j];
        }
    }
}

template <typename T, int ORDER, int V>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 288 : 544,
                                  sizeof(T) == 4 ? (V <= 5 ? 4 : (V <= 9 ? 3 : 2)) : 1)
    k_rows(StepArgs a, const RowPos *rpos, int n_rows, int ncap, int stages, int nwc,
           const RowParams<T> *pars)
{
    static_assert(V + 3 <= kHaloS && V + 1 <= kHaloP, "halo too small for V");
    static_assert(sizeof(RowParams<T>) <= 80 && kHeader % 128 == 0 &&
                      6 * 8 + (kMaxStagesH + kBatch) * 80 + 4 <= kHeader,
                  "header layout");
    static_assert((kHaloS * sizeof(T)) % 16 == 0 && (kHaloP * sizeof(T)) % 16 == 0,
                  "halos must keep 16-byte alignment");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int rowlen = ncap + 2 * kHaloS;  // staged row, with halos
    const int plen = ncap + 2 * kHaloP;    // ping-pong buffer
    // layout: [mbar full x3][mbar empty x3][params x3][batch params x32][abort]
    //         [Sq x stages][Sv x stages][A]
    // The residual sub-steps ping-pong between A and the stage's own Sq (free once
    // the remap has read it).
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
    uint64_t *empty = full + kMaxStages;
    RowParams<T> *par = reinterpret_cast<RowParams<T> *>(empty + kMaxStages);
    RowParams<T> *parb = par + kMaxStages;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(parb + kBatch);
    T *base = reinterpret_cast<T *>(smem_raw + kHeader);
    T *Sq = base;
    T *Sv = Sq + (size_t)stages * rowlen;
    T *PA = Sv + (size_t)stages * rowlen;
    (void)plen;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nct = nwc * 32;  // consumer threads
    const bool has_dv = (a.mode != MODE_SHIFT) && (a.dv != nullptr);

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 2);  // copy (expect_tx) + parameters
            mbar_init(&empty[s], nwc);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == 0) {
        // ---------------- producer: TMA and the rows' shift parameters ----------------
        // The copies of a row need only its position, not its shift, so lane 0
        // issues the first ones before waiting for the parameter kernel; the 32
        // lanes then fetch the parameters of up to 32 rows at once.  A stage's
        // full barrier expects two arrivals: the copy (with its byte count) and
        // the parameters.
        bool ok = true;
        const int my_rows = (n_rows - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
        const uint32_t hb = kHaloS * sizeof(T);
        int issued = 0;  // rows whose copies were issued
        int nfill = 0;   // fills issued (lane 0): fill f uses stage f % stages
        for (int kb = 0; kb < my_rows && ok; kb += kBatch) {
            const int k = kb + lane;
            const int kend = min(kb + kBatch, my_rows);
            int r = -1;
            RowPos row;
            if (k < my_rows) {
                row = rpos[blockIdx.x + k * gridDim.x];
                r = row.row;
            }
            // lane j holds row kb+j's record; lane 0 issues copies for the rows of
            // this batch whose stage is free without waiting (the first `stages`)
            auto issue = [&](int kk, int64_t off, int N) {
                const int s = kk % stages;
                const T *q = static_cast<const T *>(a.q_in) + off;
                uint32_t bytes = (uint32_t)(N * sizeof(T)) + 2 * hb;
                const T *dv = has_dv ? static_cast<const T *>(a.dv) + off : nullptr;
                if (has_dv) bytes += (uint32_t)(N * sizeof(T)) + hb;
                mbar_expect_tx(&full[s], bytes);
                T *sq = Sq + (size_t)s * rowlen;
                tma_load(sq + kHaloS, q, N * sizeof(T), &full[s]);
                tma_load(sq, q + N - kHaloS, hb, &full[s]);
                tma_load(sq + kHaloS + N, q, hb, &full[s]);
                if (has_dv) {
                    T *sv = Sv + (size_t)s * rowlen;
                    tma_load(sv + kHaloS, dv, N * sizeof(T), &full[s]);
                    tma_load(sv + kHaloS + N, dv, hb, &full[s]);
                }
                ++nfill;
            };
            const int pre = min(kend, stages) - kb;  // copies that need no empty wait
            for (int j = 0; j < pre; ++j) {
                const int64_t off = __shfl_sync(0xffffffffu, (long long)(k < my_rows ? row.cell_off : 0), j);
                const int N = __shfl_sync(0xffffffffu, k < my_rows ? row.n : 0, j);
                if (lane == 0) issue(kb + j, off, N);
            }
            issued = kb + (pre > 0 ? pre : 0);
            // the shift parameters come from the parameter kernel launched just before
            if (kb == 0) pdl_wait();
            if (k < my_rows) parb[lane] = pars[r];
            __syncwarp();
            if (lane == 0) {
                for (int kk = kb; kk < kend; ++kk) {
                    const int s = kk % stages;
                    if (kk >= issued) {
                        if (kk >= stages &&
                            !mbar_wait(&empty[s], ((kk / stages) - 1) & 1, a.wait_limit)) {
                            atomicOr(a.err, ERR_TIMEOUT);
                            ok = false;
                            break;
                        }
                        issue(kk, parb[kk - kb].cell_off, parb[kk - kb].n);
                    }
                    par[s] = parb[kk - kb];
                    mbar_arrive(&full[s]);  // the parameters of this stage are written
                }
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            __syncwarp();
        }
        // No copy may still be landing when the CTA exits, and after a timeout
        // the consumers may have returned without waiting for theirs: wait
        // (bounded, with the default number of tries) for the last fill of every
        // stage.  Each issued fill also got its parameter arrival, so its phase
        // completes once its bytes land; the earlier fills of a stage completed
        // before it could be refilled.
        if (lane == 0)
            for (int f = max(0, nfill - stages); f < nfill; ++f)
                mbar_wait(&full[f % stages], (f / stages) & 1);
        return;
    }

    // ---------------- consumers ----------------
    const int ct = threadIdx.x - 32;
    const bool lim = a.limiter != 0;
    const bool vl = a.scheme == RAM_VANLEER;
    T *pa = PA + kHaloP;
    int k = 0;
    for (int ri = blockIdx.x; ri < n_rows; ri += gridDim.x, ++k) {
        const int s = k % stages;
        // A wait that runs out skips the remap and raises the abort flag; every
        // consumer reads the flag after the same barrier, so all of them leave
        // together (a consumer that left alone would stall the others at the
        // next named barrier).  The flag of row k is read before the barrier
        // that ends row k, and a timeout at row k+1 is raised only after it.
        const bool got = mbar_wait(&full[s], (k / stages) & 1, a.wait_limit);
        if (!got) {
            *abort_flag = 1;
            atomicOr(a.err, ERR_TIMEOUT);
        }
        const RowParams<T> P = par[s];
        const int N = P.n;
        T *sq = Sq + (size_t)s * rowlen + kHaloS;  // valid on [-kHaloS, N+kHaloS)
        const T *sv = Sv + (size_t)s * rowlen + kHaloS;  // valid on [0, N+16)
        const int ngroups = got ? (N + V - 1) / V : 0;
        const int nsub = P.nsub;

        // remap (Eqs. 18, 26): Q' of every group of V output cells into pa
        for (int g = ct; g < ngroups; g += nct) {
            const int m0 = g * V;
            int p0 = m0 - P.K - 1;
            if (p0 < 0) p0 += N;
            T q[V + 5];
#pragma unroll
            for (int j = 0; j < V + 5; ++j) q[j] = sq[p0 - 2 + j];
            T out[V];
            if (sizeof(T) == 4)
                remap_group<T, ORDER, V>(q, P, lim, out);
            else
                remap_group_cs<T, ORDER, V>(q, P, lim, out);
            put_group<T, V>(pa, m0, N, out);
        }
        consumer_sync(nct);
        if (*abort_flag) return;

        // residual sub-steps (Eq. 6), ping-pong between A and the staged row
        T *src = pa, *dst = sq;
        T cmax = T(0);
        for (int sub = 0; sub < nsub; ++sub) {
            for (int g = ct; g < ngroups; g += nct) {
                const int m0 = g * V;
                T z[V + 4], vv[V + 1], out[V];
#pragma unroll
                for (int j = 0; j < V + 4; ++j) z[j] = src[m0 - 2 + j];
#pragma unroll
                for (int j = 0; j <= V; ++j) vv[j] = sv[m0 + j];
                if (sizeof(T) == 4) {
                    residual_group<T, V>(z, vv, P.cf, vl, cmax, out);
                } else {
                    bool bad = false;
                    residual_group_cs<T, V>(z, vv, P.cf, vl, bad, out);
                    if (bad) cmax = T(2);
                }
                put_group<T, V>(dst, m0, N, out);
            }
            consumer_sync(nct);
            T *t = src;
            src = dst;
            dst = t;
        }
        if (cmax > T(1)) atomicOr(a.err, ERR_CFL);

        // coalesced store of the finished row
        T *qout = static_cast<T *>(a.q_out) + P.cell_off;
        constexpr int VEC = 16 / sizeof(T);
        if (N % VEC == 0 && ((uintptr_t)qout % 16) == 0) {
            using V4 = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
            const V4 *s4 = reinterpret_cast<const V4 *>(src);
            V4 *d4 = reinterpret_cast<V4 *>(qout);
            for (int c = ct; c < N / VEC; c += nct) d4[c] = s4[c];
        } else {
            for (int c = ct; c < N; c += nct) qout[c] = src[c];
        }
        // the stage (row, dv and ping-pong use) is no longer read: hand it back;
        // the barrier keeps A intact until every thread has stored the row
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        consumer_sync(nct);
    }
}

}  // namespace

// Launch the persistent kernel for the uniform rows of one order that the plan
// assigned to it (TMA-eligible, shared-memory fit).  V = cells per consumer
// thread (odd, a tuning parameter).
template <typename T, int ORDER, int V>
static cudaError_t launch_rows_v(const Plan &p, const StepArgs &a, cudaStream_t s,
                                 const RowPos *rows, int n_rows, int ncap)
{
    const size_t es = sizeof(T);
    const size_t rowb = (size_t)(ncap + 2 * kHaloS) * es;
    const size_t pb = (size_t)(ncap + 2 * kHaloP) * es;
    // CTAs per SM: the plan's choice, within what the register budget of this V
    // allows; shared memory per CTA is the SM's share, filled with as many stages
    // (up to three) as fit
    const int cps_max = sizeof(T) == 4 ? (V <= 5 ? 4 : (V <= 9 ? 3 : 2)) : 1;
    int cps = p.rows_cps[sizeof(T) == 4 ? 0 : 1];
    if (cps > cps_max) cps = cps_max;
    if (cps < 1) cps = 1;
    int stages = 0;
    size_t smem = 0;
    for (; cps >= 1; --cps) {
        const size_t budget = (size_t)(227 * 1024) / cps - 1024;
        for (stages = kMaxStages; stages >= 1; --stages) {
            smem = kHeader + 2 * stages * rowb + pb;
            if (smem <= budget) break;
        }
        if (stages >= 1) break;
    }
    if (cps < 1 || stages < 1) return cudaErrorNotSupported;
    int groups = (ncap + V - 1) / V;
    const int nwc_max = sizeof(T) == 4 ? 8 : 16;  // within the launch bounds
    int nwc = (groups + 31) / 32;
    if (nwc > nwc_max) nwc = nwc_max;
    if (nwc < 4) nwc = 4;
    static bool configured[64] = {false};
    const int dev = p.device < 64 ? p.device : 63;
    if (!configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_rows<T, ORDER, V>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(227 * 1024));
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
    int fit = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, k_rows<T, ORDER, V>, 32 * (nwc + 1),
                                                  smem);
    if (fit < 1) fit = 1;
    if (fit > cps) fit = cps;
    const int grid = n_rows < sms * fit ? n_rows : sms * fit;
    return launch_pdl(k_rows<T, ORDER, V>, grid, 32 * (nwc + 1), smem, s, a, rows, n_rows,
                      ncap, stages, nwc, static_cast<const RowParams<T> *>(p.row_par));
}

template <typename T, int ORDER>
static cudaError_t launch_rows_t(const Plan &p, const StepArgs &a, cudaStream_t s,
                                 const RowPos *rows, int n_rows, int ncap)
{
    switch (p.rows_v[sizeof(T) == 4 ? 0 : 1]) {
    case 5: return launch_rows_v<T, ORDER, 5>(p, a, s, rows, n_rows, ncap);
    case 9: return launch_rows_v<T, ORDER, 9>(p, a, s, rows, n_rows, ncap);
    case 11: return launch_rows_v<T, ORDER, 11>(p, a, s, rows, n_rows, ncap);
    case 15: return launch_rows_v<T, ORDER, 15>(p, a, s, rows, n_rows, ncap);
    default: return launch_rows_v<T, ORDER, 7>(p, a, s, rows, n_rows, ncap);
    }
}

const int kRowsVCandidates[] = {5, 7, 9, 11, 15};
const int kRowsVCount = 5;

cudaError_t launch_rows(const Plan &p, ram_dtype dt, const StepArgs &a, cudaStream_t s,
                        int order, const RowPos *rows, int n_rows, int ncap)
{
    if (n_rows == 0) return cudaSuccess;
    if (dt == RAM_F32) {
        if (order == 2) return launch_rows_t<float, 2>(p, a, s, rows, n_rows, ncap);
        if (order == 3) return launch_rows_t<float, 3>(p, a, s, rows, n_rows, ncap);
        return launch_rows_t<float, 4>(p, a, s, rows, n_rows, ncap);
    }
    if (order == 2) return launch_rows_t<double, 2>(p, a, s, rows, n_rows, ncap);
    if (order == 3) return launch_rows_t<double, 3>(p, a, s, rows, n_rows, ncap);
    return launch_rows_t<double, 4>(p, a, s, rows, n_rows, ncap);
}

}  // namespace ram
