// Per-thread arithmetic of the uniform-row kernels: the remap of V consecutive
// output cells from their source window and one residual sub-step of V cells,
// in the min/max-with-sign form (FP32) and in compare-and-select form (FP64).
#pragma once

#include <cuda_runtime.h>

#include "ram_device.cuh"

namespace ram {

// a / b for the slope ratios of the uniform-row kernels: FP32 multiplies by the
// approximate reciprocal (one instruction more than the product; the ratios'
// denominators are sums of cell differences, far inside the FP32 range)
__device__ __forceinline__ float lane_div(float a, float b) { return a * rcp_approx(b); }
__device__ __forceinline__ double lane_div(double a, double b) { return a / b; }

template <typename T>
__device__ __forceinline__ T half_vl_relu(T dl, T dr)
{
    // the same half slope without a select (FP32 rows): max(dl dr, 0) /
    // (dl + dr + tiny).  The tiny term only matters where |dl + dr| < 1e-30, and
    // there dl dr is either <= 0 or below the FP32 range (zero)
    return lane_div(fmax(dl * dr, T(0)), dl + dr + T(1e-30));
}

template <typename T>
__device__ __forceinline__ T half_vl(T dl, T dr)
{
    // half of the van Leer slope: dl dr / (dl + dr) when dl dr > 0, else 0
    const T p = dl * dr;
    return p > T(0) ? lane_div(p, dl + dr) : T(0);
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
                // minxs(D, m) = sign(D) min(|D|, m) for m >= 0
                Dq[i] = minxs(D, fmax(T(4) * minxs(dif[i], dif[i + 1]), T(0)));
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

// The PPM remap of remap_group for a warp whose lanes hold V consecutive cells
// each (FP32, lean form), with every limited slope and every left partial
// formed once: a lane forms those of its own V source cells p0 .. p0+V-1 and
// takes the slope of cell p0-1 from the lane on its left, and the slope of cell
// p0+V and the partial of cell p0+V from the lane on its right.  q[0..V+4] holds
// source cells p0-2 .. p0+V+2 (this form reads q[1..V+2]).  Lanes 0 and 31 take
// their outer neighbours from the other end of the warp, which spoils the warp's
// first output cell and its last two: the caller keeps them as halo.
template <int V>
__device__ __forceinline__ void remap_warp3(const float (&q)[V + 5], const RowParams<float> &P,
                                            bool lim, float (&out)[V])
{
    if (P.whole) {
#pragma unroll
        for (int k = 0; k < V; ++k) out[k] = q[k + 3];
        return;
    }
    const unsigned full = 0xffffffffu;
    float dif[V + 1];  // dif[i] = Q(p0-1+i+1) - Q(p0-1+i), i = 0..V
#pragma unroll
    for (int i = 0; i <= V; ++i) dif[i] = q[i + 2] - q[i + 1];
    float Dq[V + 2];   // 2 dQ of cells p0-1 .. p0+V; own cells at Dq[1..V]
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const float D = dif[j] + dif[j + 1];
        Dq[j + 1] = lim ? minxs(D, fmaxf(4.0f * minxs(dif[j], dif[j + 1]), 0.0f)) : D;
    }
    Dq[0] = __shfl_up_sync(full, Dq[V], 1);
    Dq[V + 1] = __shfl_down_sync(full, Dq[1], 1);
    float E[V + 1];    // E[i] = Dq(p0+i) - Dq(p0+i-1)
#pragma unroll
    for (int i = 0; i <= V; ++i) E[i] = Dq[i + 1] - Dq[i];
    const float xi = P.c[3], cR = P.c[1], cL = P.c[0];
    float A[V + 1];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        // cell p0+j: right face from dif[j+1], E[j+1]; left face from dif[j], E[j]
        const float a = fmaf(E[j + 1], -1.0f / 12.0f, 0.5f * dif[j + 1]);
        const float b = fmaf(E[j], 1.0f / 12.0f, 0.5f * dif[j]);
        float G;
        if (lim) {
            const float a2 = fmaf(E[j + 1], -1.0f / 6.0f, dif[j + 1]);  // 2a
            const float b2 = fmaf(E[j], 1.0f / 6.0f, dif[j]);           // 2b
            const float u = fmaxf(minxs(a, b2), 0.0f);                  // |a'|
            const float v = fmaxf(minxs(b, a2), 0.0f);                  // |b'|
            G = xorsign(fmaf(cR, u, -cL * v), a);
        } else {
            G = fmaf(cR, a, -cL * b);
        }
        A[j] = fmaf(xi, q[j + 2], G);
    }
    A[V] = __shfl_down_sync(full, A[0], 1);
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
        for (int c = 0; c < V + 2; ++c) h[c] = half_vl_relu(d[c], d[c + 1]);
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

// One residual sub-step of a warp whose lanes hold V consecutive cells each
// (lane l cells l V .. l V + V - 1 of the warp's range), FP32.  c[k] = dv cf is
// the Courant number of the lane's face k (the left node of its cell k).  Every
// lane forms the half slopes of its own cells and the fluxes of its own faces;
// the neighbour cells and slope on the left and the flux on the right come from
// the adjacent lanes by shuffles, so no slope or flux is formed twice.  The
// flux is the one of residual_group, written with the upwind cell selected by
// the sign of c: F = c (Q_up + (1 - |c|) h_up), h_up the upwind half slope
// taken toward the face; lanes 0 and 31 take their outer
// neighbours from the other end of the warp, which spoils the outermost two
// cells of the warp's range per van Leer sub-step (one per donor sub-step):
// the caller keeps them as halo.
template <int V, bool VL>
__device__ __forceinline__ void residual_warp(float (&cur)[V], const float (&c)[V])
{
    const unsigned full = 0xffffffffu;
    const float zl = __shfl_up_sync(full, cur[V - 1], 1);
    float F[V];
    if (VL) {
        const float zr = __shfl_down_sync(full, cur[0], 1);
        float d[V + 1];  // d[i] = z_i - z_{i-1}, i = 0..V
        d[0] = cur[0] - zl;
#pragma unroll
        for (int i = 1; i < V; ++i) d[i] = cur[i] - cur[i - 1];
        d[V] = zr - cur[V - 1];
        float h[V];
#pragma unroll
        for (int i = 0; i < V; ++i) h[i] = half_vl_relu(d[i], d[i + 1]);
        const float hl = __shfl_up_sync(full, h[V - 1], 1);
#pragma unroll
        for (int k = 0; k < V; ++k) {
            // the upwind cell's value and half slope (the left cell for c > 0, the
            // right one, slope negated, otherwise): F = c (Q_up + (1 - |c|) h_up)
            const bool pos = c[k] > 0.0f;
            const float zu = pos ? (k ? cur[k - 1] : zl) : cur[k];
            const float hu = pos ? (k ? h[k - 1] : hl) : -h[k];
            F[k] = c[k] * fmaf(1.0f - fabsf(c[k]), hu, zu);
        }
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const float ap = fmaxf(c[k], 0.0f);
            const float am = c[k] - ap;
            F[k] = fmaf(ap, k ? cur[k - 1] : zl, am * cur[k]);
        }
    }
    const float Fr = __shfl_down_sync(full, F[0], 1);
#pragma unroll
    for (int k = 0; k < V - 1; ++k) cur[k] = cur[k] - (F[k + 1] - F[k]);
    cur[V - 1] = cur[V - 1] - (Fr - F[V - 1]);
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


// ---------------------------------------------------------------------------
// Packed FP32 forms: two segments per lane, one per half of a float2.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }

// Q' for the V output cells of one lane in two segments at once (the two halves
// of float2 registers: FP32 arithmetic on the packed pipe).  q[0..V+4] holds
// source cells p0-2 .. p0+V+2 with p0 = m0 - K - 1, m0 the lane's first cell;
// k holds the partial-integral coefficients (order 3: xi, cR, -cL; order 2:
// xi, slope; order 4: the five weights).
template <int ORDER, int V>
__device__ __forceinline__ void remap_pair(const float2 (&q)[V + 5], int whole, const float (&k)[5],
                                           bool lim, float2 (&out)[V])
{
    if (whole) {
#pragma unroll
        for (int k = 0; k < V; ++k) out[k] = q[k + 3];
        return;
    }
    float2 A[V + 1];  // left partial integral of source cells p0 .. p0+V
    if (ORDER == 3) {
        float2 dif[V + 4];
#pragma unroll
        for (int i = 0; i < V + 4; ++i) dif[i] = sub2(q[i + 1], q[i]);
        float2 Dq[V + 3];  // 2 dQ of source cells p0-1 .. p0+V+1
#pragma unroll
        for (int i = 0; i < V + 3; ++i) {
            const float2 D = __fadd2_rn(dif[i], dif[i + 1]);
            if (lim) {
                float2 t = make_float2(minxs(dif[i].x, dif[i + 1].x), minxs(dif[i].y, dif[i + 1].y));
                t = __fmul2_rn(t, f2(4.0f));
                // minxs(D, m) = sign(D) min(|D|, m) for m >= 0
                Dq[i] = make_float2(minxs(D.x, fmaxf(t.x, 0.0f)), minxs(D.y, fmaxf(t.y, 0.0f)));
            } else {
                Dq[i] = D;
            }
        }
        float2 E[V + 2];  // 2 (dQ_{j+1} - dQ_j) for j = p0-1 .. p0+V
#pragma unroll
        for (int i = 0; i < V + 2; ++i) E[i] = sub2(Dq[i + 1], Dq[i]);
        float2 h[V + 3];  // dif / 2 (index 1 .. V+2 used)
#pragma unroll
        for (int i = 1; i < V + 3; ++i) h[i] = __fmul2_rn(dif[i], f2(0.5f));
        const float2 k0 = f2(k[0]), k1 = f2(k[1]), k2 = f2(k[2]);
#pragma unroll
        for (int j = 0; j <= V; ++j) {
            // a = QR - Q = dif_j / 2 - E_j / 12,  b = Q - QL = dif_{j-1} / 2 + E_{j-1} / 12
            const float2 a = __ffma2_rn(E[j + 1], f2(-1.0f / 12.0f), h[j + 2]);
            const float2 b = __ffma2_rn(E[j], f2(1.0f / 12.0f), h[j + 1]);
            float2 G;
            if (lim) {
                const float2 a2 = __ffma2_rn(E[j + 1], f2(-1.0f / 6.0f), dif[j + 2]);
                const float2 b2 = __ffma2_rn(E[j], f2(1.0f / 6.0f), dif[j + 1]);
                const float2 u = make_float2(fmaxf(minxs(a.x, b2.x), 0.0f),
                                             fmaxf(minxs(a.y, b2.y), 0.0f));  // |a'|
                const float2 v = make_float2(fmaxf(minxs(b.x, a2.x), 0.0f),
                                             fmaxf(minxs(b.y, a2.y), 0.0f));  // |b'|
                G = __ffma2_rn(k1, u, __fmul2_rn(k2, v));
                G = make_float2(xorsign(G.x, a.x), xorsign(G.y, a.y));
            } else {
                G = __ffma2_rn(k1, a, __fmul2_rn(k2, b));
            }
            A[j] = __ffma2_rn(k0, q[j + 2], G);
        }
    } else if (ORDER == 2) {
        const float2 k0 = f2(k[0]), k1 = f2(k[1]);
#pragma unroll
        for (int j = 0; j <= V; ++j) {
            const float2 dn = sub2(q[j + 2], q[j + 1]), up = sub2(q[j + 3], q[j + 2]);
            float2 sl;
            if (lim) {
                const float2 p = __fmul2_rn(dn, up);
                const float2 s = __fadd2_rn(dn, up);
                const float2 hh = __fmul2_rn(p, make_float2(__fdividef(2.0f, s.x),
                                                            __fdividef(2.0f, s.y)));
                sl = make_float2(p.x > 0.0f ? hh.x : 0.0f, p.y > 0.0f ? hh.y : 0.0f);
            } else {
                sl = __fmul2_rn(__fadd2_rn(dn, up), f2(0.5f));
            }
            A[j] = __ffma2_rn(q[j + 2], k0, __fmul2_rn(sl, k1));
        }
    } else {
#pragma unroll
        for (int j = 0; j <= V; ++j) {
            float2 s = __fmul2_rn(f2(k[0]), q[j]);
#pragma unroll
            for (int i = 1; i < 5; ++i) s = __ffma2_rn(f2(k[i]), q[j + i], s);
            A[j] = s;
        }
    }
#pragma unroll
    for (int k = 0; k < V; ++k) out[k] = __fadd2_rn(sub2(q[k + 2], A[k]), A[k + 1]);
}

// The residual sub-steps (Eq. 6) of one lane's cells in both segments.  v[0..V]
// are the velocities at the lane's nodes m0..m0+V (node k is the left node of
// cell m0+k).  The flux through node k is
//   F = c+ (Q_{k-1} + h_{k-1} (1 - c+)) + c- (Q_k - h_k (1 + c-)),
// c+ = max(c, 0), c- = min(c, 0), c = v cf, h the half van Leer slope (0 for
// donor): the upwind value at the midpoint of the swept region.
template <int V>
__device__ __forceinline__ void residual_pair(float2 (&cur)[V], const float2 (&v)[V + 1], float cf,
                                              int nsub, bool vl, int lane, float &cmax)
{
    float2 ap[V + 1], am[V + 1];
#pragma unroll
    for (int k = 0; k <= V; ++k) {
        const float2 c = __fmul2_rn(v[k], f2(cf));
        ap[k] = make_float2(fmaxf(c.x, 0.0f), fmaxf(c.y, 0.0f));
        am[k] = sub2(c, ap[k]);
        cmax = fmaxf(cmax, fmaxf(fabsf(c.x), fabsf(c.y)));
    }
    const int up = (lane + 31) & 31, dn = (lane + 1) & 31;
    for (int sub = 0; sub < nsub; ++sub) {
        float2 z[V + 4];  // cells m0-2 .. m0+V+1
        {
            // lane 0's B continues lane 31's A; lane 31's A continues lane 0's B
            const float l2x = __shfl_sync(0xffffffffu, cur[V - 2].x, up);
            const float l2y = __shfl_sync(0xffffffffu, cur[V - 2].y, up);
            const float l1x = __shfl_sync(0xffffffffu, cur[V - 1].x, up);
            const float l1y = __shfl_sync(0xffffffffu, cur[V - 1].y, up);
            const float r1x = __shfl_sync(0xffffffffu, cur[0].x, dn);
            const float r1y = __shfl_sync(0xffffffffu, cur[0].y, dn);
            const float r2x = __shfl_sync(0xffffffffu, cur[1].x, dn);
            const float r2y = __shfl_sync(0xffffffffu, cur[1].y, dn);
            z[0] = make_float2(l2x, lane == 0 ? l2x : l2y);
            z[1] = make_float2(l1x, lane == 0 ? l1x : l1y);
            z[V + 2] = make_float2(lane == 31 ? r1y : r1x, r1y);
            z[V + 3] = make_float2(lane == 31 ? r2y : r2x, r2y);
        }
#pragma unroll
        for (int k = 0; k < V; ++k) z[k + 2] = cur[k];
        float2 F[V + 1];
        if (vl) {
            float2 d[V + 3];
#pragma unroll
            for (int i = 0; i < V + 3; ++i) d[i] = sub2(z[i + 1], z[i]);
            float2 h[V + 2];  // half slopes of cells m0-1 .. m0+V
#pragma unroll
            for (int c = 0; c < V + 2; ++c) {
                const float2 p = __fmul2_rn(d[c], d[c + 1]);
                const float2 s = __fadd2_rn(d[c], d[c + 1]);
                // max(p, 0) / (s + tiny): the half slope without a select (see half_vl_relu)
                const float2 st = __fadd2_rn(s, f2(1e-30f));
                h[c] = __fmul2_rn(make_float2(fmaxf(p.x, 0.0f), fmaxf(p.y, 0.0f)),
                                  make_float2(__fdividef(1.0f, st.x), __fdividef(1.0f, st.y)));
            }
#pragma unroll
            for (int k = 0; k <= V; ++k) {
                // c+ (1 - c+) and -c- (1 + c-) = c- (-1 - c-)
                const float2 wp = __fmul2_rn(ap[k], __ffma2_rn(ap[k], f2(-1.0f), f2(1.0f)));
                const float2 wm = __fmul2_rn(am[k], __ffma2_rn(am[k], f2(-1.0f), f2(-1.0f)));
                float2 f = __fmul2_rn(am[k], z[k + 2]);
                f = __ffma2_rn(ap[k], z[k + 1], f);
                f = __ffma2_rn(wp, h[k], f);
                F[k] = __ffma2_rn(wm, h[k + 1], f);
            }
        } else {
#pragma unroll
            for (int k = 0; k <= V; ++k) F[k] = __ffma2_rn(ap[k], z[k + 1], __fmul2_rn(am[k], z[k + 2]));
        }
#pragma unroll
        for (int k = 0; k < V; ++k) cur[k] = sub2(z[k + 2], sub2(F[k + 1], F[k]));
    }
}

}  // namespace ram
