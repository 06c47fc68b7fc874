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
// shared-memory header: barriers and the row parameters
constexpr int kHeader = (6 * 8 + (kMaxStagesH + kBatch) * 80 + 127) / 128 * 128;

template <typename T>
__device__ __forceinline__ T half_vl(T dl, T dr)
{
    // half of the van Leer slope: dl dr / (dl + dr) when dl dr > 0, else 0
    const T p = dl * dr;
    return p > T(0) ? Num<T>::div(p, dl + dr) : T(0);
}

// Q' for V consecutive output cells.  q[0..V+4] holds source cells p0-2..p0+V+2
// where p0 = m0 - K - 1 is the source cell of the left part of output cell m0:
// Q'_m = (Q_p - A_p) + A_{p+1}, A the left partial integral at the edge offset.
//
// PPM (App. A) in difference form: with dif_i = Q_{i+1} - Q_i, D = dif_{i-1} +
// dif_i and E_i = 2 (dQ_{i+1} - dQ_i),
//   2 dQ_i = sign(D) min(|D|, 4 |dif_{i-1}|, 4 |dif_i|) if dif_{i-1} dif_i > 0 else 0,
//   a = QR - Q = dif_i / 2 - E_i / 12,   b = Q - QL = dif_{i-1} / 2 + E_{i-1} / 12,
// and the App. A.2 constraints (a b <= 0: flat; |b| > 2|a|: QL = 3Q - 2QR;
// |a| > 2|b|: QR = 3Q - 2QL) are a' = median(0, a, 2b), b' = median(0, b, 2a).
// The folded coefficients give A = xi Q + cR a' - cL b' (P.c[3] = xi, P.c[1] = cR,
// P.c[0] = cL).
template <typename T, int ORDER, int V>
__device__ __forceinline__ void remap_group(const T (&q)[V + 5], const RowParams<T> &P, bool lim,
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
        for (int i = 0; i < V + 4; ++i) dif[i] = q[i + 1] - q[i];
        T Dq[V + 3];  // 2 dQ of source cells p0-1 .. p0+V+1
#pragma unroll
        for (int i = 0; i < V + 3; ++i) {
            const T D = dif[i] + dif[i + 1];
            if (lim) {
                const T m = fmax(fmin(fabs(D), T(4) * minxs(dif[i], dif[i + 1])), T(0));
                Dq[i] = minxs(D, m);
            } else {
                Dq[i] = D;
            }
        }
        T E[V + 2];
#pragma unroll
        for (int i = 0; i < V + 2; ++i) E[i] = Dq[i + 1] - Dq[i];
        const T xi = P.c[3], cR = P.c[1], cL = P.c[0];
#pragma unroll
        for (int j = 0; j <= V; ++j) {
            const T a = fma(E[j + 1], T(-1) / T(12), T(0.5) * dif[j + 2]);
            const T b = fma(E[j], T(1) / T(12), T(0.5) * dif[j + 1]);
            T G;
            if (lim) {
                const T a2 = fma(E[j + 1], T(-1) / T(6), dif[j + 2]);  // 2a
                const T b2 = fma(E[j], T(1) / T(6), dif[j + 1]);       // 2b
                const T u = fmax(minxs(a, b2), T(0));                  // |a'|
                const T v = fmax(minxs(b, a2), T(0));                  // |b'|
                G = xorsign(fma(cR, u, -cL * v), a);
            } else {
                G = fma(cR, a, -cL * b);
            }
            A[j] = fma(xi, q[j + 2], G);
        }
    } else if (ORDER == 2) {
#pragma unroll
        for (int j = 0; j <= V; ++j) {
            const T dn = q[j + 2] - q[j + 1], up = q[j + 3] - q[j + 2];
            const T sl = lim ? T(2) * half_vl(dn, up) : T(0.5) * (dn + up);
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

// One residual sub-step for V cells m0..m0+V-1.  z[0..V+3] holds Q at cells
// m0-2..m0+V+1, v[0..V] the interface velocities at m0..m0+V (interface k is the
// left node of cell m0+k).  The flux through interface k (Eq. 6 with the PLM
// slope of Sec. 3.1 for van Leer, none for donor) carries the upwind value at the
// midpoint of the swept region:
//   F = c+ (Q_{k-1} + h_{k-1} (1 - c+)) + c- (Q_k - h_k (1 + c-)),
// c = v cf, c+ = max(c, 0), c- = c - c+, h the half van Leer slope.  cmax keeps
// the largest |c| (the CFL check).
template <typename T, int V>
__device__ __forceinline__ void residual_group(const T (&z)[V + 4], const T (&v)[V + 1], T cf,
                                               bool vl, T &cmax, T (&out)[V])
{
    T h[V + 2];  // half slopes of cells m0-1..m0+V
    if (vl) {
        T d[V + 3];
#pragma unroll
        for (int i = 0; i < V + 3; ++i) d[i] = z[i + 1] - z[i];
#pragma unroll
        for (int c = 0; c < V + 2; ++c) h[c] = half_vl(d[c], d[c + 1]);
    }
    T F[V + 1];
#pragma unroll
    for (int k = 0; k <= V; ++k) {
        const T c = v[k] * cf;
        const T ap = fmax(c, T(0));
        const T am = c - ap;
        cmax = fmax(cmax, fabs(c));
        T f = fma(ap, z[k + 1], am * z[k + 2]);
        if (vl) {
            const T wp = fma(-ap, ap, ap);   // c+ (1 - c+)
            const T wm = fma(-am, am, -am);  // -c- (1 + c-)
            f = fma(wp, h[k], fma(wm, h[k + 1], f));
        }
        F[k] = f;
    }
#pragma unroll
    for (int k = 0; k < V; ++k) out[k] = z[k + 2] - (F[k + 1] - F[k]);
}

template <typename T>
__device__ __forceinline__ T lim_dq(T dn, T up, bool lim)
{
    // delta<Q> of App. A on a uniform row from the two one-sided differences,
    // limited by App. A.2: sign * min(|d|, 2|dn|, 2|up|) where dn up > 0, else 0
    const T d = T(0.5) * (dn + up);
    if (!lim) return d;
    const T mm = fmin(fabs(dn), fabs(up));
    const T m = fmin(fabs(d), mm + mm);
    return (dn * up > T(0)) ? copysign(m, d) : T(0);
}

// The same two operations in compare-and-select form, for FP64 rows (whose
// arithmetic runs on the FP64 pipe, where the min/max form saves nothing and
// needs more registers).
//
// Q' for V consecutive output cells.  q[0..V+4] holds source cells p0-2..p0+V+2
// where p0 = m0 - K - 1 is the source cell of the left part of output cell m0.
// P.c holds the coefficients of the left partial at the edge offset xi; for PPM
// they are folded with Q6 = 6Q - 3(QL + QR):  A = QL c0 + QR c1 + Q c2.
template <typename T, int ORDER, int V>
__device__ __forceinline__ void remap_group_cs(const T (&q)[V + 5], const RowParams<T> &P, bool lim,
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
        for (int c = 1; c <= V + 3; ++c) dq[c - 1] = lim_dq(dif[c - 1], dif[c], lim);
        T face[V + 2];
        const T sixth = T(1) / T(6);
#pragma unroll
        for (int f = 0; f < V + 2; ++f)
            face[f] = fma(T(0.5), dif[f + 1], q[f + 1]) - (dq[f + 1] - dq[f]) * sixth;
#pragma unroll
        for (int j = 0; j <= V; ++j) {
            const T Q = q[j + 2];
            T L = face[j], R = face[j + 1];
            if (lim) {
                // App. A.2 with a = QR - Q, b = Q - QL: flat at an extremum (a b <= 0);
                // otherwise the parabola overshoots on the left when |b| > 2|a|
                // (QL = 3Q - 2QR) and on the right when |a| > 2|b| (QR = 3Q - 2QL).
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
            const T sl = lim ? T(2) * half_vl(dn, up) : T(0.5) * (dn + up);
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

// One residual sub-step for V cells m0..m0+V-1.  z[0..V+3] holds Q at cells
// m0-2..m0+V+1, v[0..V] the interface velocities at m0..m0+V (interface k is the
// left node of cell m0+k).  Donor: the flux carries the upwind value; van Leer:
// the upwind value corrected by the half slope at the midpoint of the swept
// region (Eq. 6 with the PLM slope of Sec. 3.1).
template <typename T, int V>
__device__ __forceinline__ void residual_group_cs(const T (&z)[V + 4], const T (&v)[V + 1], T cf,
                                               bool vl, bool &cfl_bad, T (&out)[V])
{
    T hs[V + 2];  // half slopes of cells m0-1..m0+V
    if (vl) {
#pragma unroll
        for (int c = 0; c < V + 2; ++c) hs[c] = half_vl(z[c + 1] - z[c], z[c + 2] - z[c + 1]);
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
    for (int k = 0; k < V; ++k) out[k] = z[k + 2] - (F[k + 1] - F[k]);
}

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
    static_assert(sizeof(RowParams<T>) <= 80 && kHeader % 128 == 0, "header layout");
    static_assert((kHaloS * sizeof(T)) % 16 == 0 && (kHaloP * sizeof(T)) % 16 == 0,
                  "halos must keep 16-byte alignment");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int rowlen = ncap + 2 * kHaloS;  // staged row, with halos
    const int plen = ncap + 2 * kHaloP;    // ping-pong buffer
    // layout: [mbar full x3][mbar empty x3][params x3][batch params x32]
    //         [Sq x stages][Sv x stages][A]
    // The residual sub-steps ping-pong between A and the stage's own Sq (free once
    // the remap has read it).
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
    uint64_t *empty = full + kMaxStages;
    RowParams<T> *par = reinterpret_cast<RowParams<T> *>(empty + kMaxStages);
    RowParams<T> *parb = par + kMaxStages;
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
                        if (kk >= stages && !mbar_wait(&empty[s], ((kk / stages) - 1) & 1)) {
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
        // after a timeout, wait (bounded) for the copies already in flight
        if (!ok && lane == 0)
            for (int s = 0; s < stages; ++s) mbar_wait(&full[s], 0);
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
        if (!mbar_wait(&full[s], (k / stages) & 1)) {
            if (ct == 0) atomicOr(a.err, ERR_TIMEOUT);
            return;
        }
        const RowParams<T> P = par[s];
        const int N = P.n;
        T *sq = Sq + (size_t)s * rowlen + kHaloS;  // valid on [-kHaloS, N+kHaloS)
        const T *sv = Sv + (size_t)s * rowlen + kHaloS;  // valid on [0, N+16)
        const int ngroups = (N + V - 1) / V;
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
