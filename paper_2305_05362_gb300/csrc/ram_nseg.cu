// RAM step on FP32 rows with their own non-uniform mesh (Sec. 3 on an arbitrary
// periodic mesh), warp-segment form.
//
// One CTA per tile of a row (up to kNsegWarps * kNsegPerWarp segments of at most
// kNseg output cells).  The tile's prologue forms the row's shift once (S0:
// shift_params, FP64, one thread), then locates the source cells of the two
// outer edges of every segment (extended by the residual halo) through the
// plan's bucket table -- the index function of Sec. 3.2.1 tabulated on the
// row's own nodes -- and a short walk (Eq. 16).  Then every warp takes its
// segments one at a time, with no CTA barrier:
//   - the segment's source window is the source cells its shifted edges land in
//     plus a reconstruction halo of two cells per side; lane l takes the window
//     cells 4l..4l+3 (and 128+4l..128+4l+3): it loads their values and nodes,
//     with the stencil's halo, into registers, forms their widths (exact
//     differences of the fixed-point nodes, in units of the row's mean width)
//     and their reconstructions (PLM with the van Leer limiter, Sec. 3.1; PPM,
//     App. A with the limiter of App. A.2; order 4, the mean of the two quartic
//     interpolants of the cumulative mass), and stores the power-basis
//     coefficients of each cell's in-cell cumulative G_p(xi dx_p) (Eq. 18's
//     partial integrals) in the warp's shared memory;
//   - lane l then takes the output cells 4l..4l+3: their five shifted edges are
//     located among the window's nodes (one binary search, then a walk; Eq. 16),
//     G is evaluated at every edge once, and each output mass is Eq. 18 -- the
//     rest of the left source cell, the whole cells in between summed directly in
//     order, the start of the right source cell -- divided by the output width
//     (Eq. 26); an output cell whose edges both fall on the nodes of one source
//     cell takes that cell's value unchanged;
//   - with a residual step (Eq. 6) the segment is extended by the residual halo
//     on both sides and the sub-steps run in the warp's shared memory.
// Node positions are fractions of the period in units of 2^-64, so x - s and the
// periodic wrap are exact integer arithmetic.  Inside a segment positions are
// taken relative to the window's first node, where they increase (a segment and
// its halo span less than one period), and kept as 32-bit values in units of
// 2^qshift: the plan picks qshift per row so that every window fits and every
// cell still spans at least 2^20 units.
#include <cuda_runtime.h>

#include <cstdint>

#include "ram_device.cuh"

namespace ram {
namespace {

constexpr int kV = kNsegV;                   // window cells per lane and chunk (4)
constexpr int kVE = 3;                       // output cells per lane and pass
constexpr int kHR = kNsegHR;                 // reconstruction halo, cells per side
constexpr int kStride = 32 * kV - 4;         // reconstruction chunks: 128 cells, stride 124
constexpr int kCover = kStride + 32 * kV;    // cells the two chunks cover (252)
constexpr int kWcap = kCover - 2;            // window cells a warp can hold (250)
constexpr int kEmax = kNseg + 2 * kGenHalo;  // extended segment (residual halo)

constexpr int kSkewed = kCover + 4 + (kCover + 4) / 32 + 1;  // padded length of the per-window arrays
// window index -> padded index: one word after every 32, so that lanes storing
// cells 4 apart hit 32 different banks
__device__ __forceinline__ int pz(int s) { return s + (s >> 5); }

// Per-warp shared-memory layout (32-bit words).
struct NLayout {
    int r, q, h, iw, c, p, total;
};

__host__ __device__ inline NLayout nseg_layout(bool resid)
{
    NLayout L;
    int o = 0;
    auto put = [&o](int words) {
        const int at = o;
        o += (words + 3) / 4 * 4;
        return at;
    };
    L.r = put(kSkewed);       // window node positions (u32, window-relative)
    L.q = put(kSkewed);       // window cell values
    L.h = put(kSkewed);       // window cell widths (mean-width units)
    L.iw = put(kSkewed);      // 1 / width in position units
    // cumulative coefficients, 4 arrays; once the edges are done, the residual's
    // output widths, second state, velocities and fluxes in their place
    L.c = put(4 * kSkewed);
    L.p = put(resid ? kEmax : 0);  // the remapped segment, the residual's first state
    L.total = o;
    return L;
}

// ---- reconstruction (normalized widths, mean width 1) ----
// Every form gives the power-basis coefficients b[0..3] of the in-cell
// cumulative G(xi) = xi (b0 + xi (b1 + xi (b2 + xi b3))), already multiplied by
// the cell's width: G(1) is the cell's mass q h.

// PLM (Sec. 3.1): G/h = q xi + sigma h (xi^2 - xi)/2.  Limited: the van Leer
// harmonic mean of the one-sided slopes over centre spacings, zero at an
// extremum; otherwise the centred slope.
template <bool LIM>
__device__ __forceinline__ void recon_plm(float qm, float q0, float qp, float hm, float h0,
                                          float hp, float b[4])
{
    float sh;  // sigma * h0
    if (LIM) {
        const float dl = q0 - qm, dr = qp - q0;
        // 2 (dl/hl)(dr/hr) / (dl/hl + dr/hr), hl = (hm+h0)/2, hr = (h0+hp)/2
        const float den = dl * (h0 + hp) + dr * (hm + h0);
        sh = (dl * dr > 0.f) ? 4.f * dl * dr * h0 * rcp_approx(den) : 0.f;
    } else {
        sh = 2.f * (qp - qm) * h0 * rcp_approx(hm + 2.f * h0 + hp);
    }
    b[0] = h0 * (q0 - 0.5f * sh);
    b[1] = h0 * 0.5f * sh;
    b[2] = 0.f;
    b[3] = 0.f;
}

// delta<Q>_k of App. A.1 on a non-uniform mesh (widths a, b, c of cells k-1, k,
// k+1), limited by the first stage of App. A.2: sign(d) min(|d|, 2|dn|, 2|up|)
// where (Q_{k+1} - Q_k)(Q_k - Q_{k-1}) > 0, else 0.
template <bool LIM>
__device__ __forceinline__ float ppm_dq(float qm, float q0, float qp, float a, float b, float c)
{
    const float up = qp - q0, dn = q0 - qm;
    const float ab = a + b, bc = b + c;
    // b/(a+b+c) [ (2a+b)/(b+c) up + (b+2c)/(a+b) dn ], one reciprocal
    float d = b * ((2.f * a + b) * ab * up + (b + 2.f * c) * bc * dn) *
              rcp_approx((ab + c) * bc * ab);
    if (LIM) d = minxs(d, fmaxf(2.f * minxs(dn, up), 0.f));
    return d;
}

// interface value <Q>_{k+1/2} of App. A.1 (weights read with sums of widths),
// widths hm, h0, h1, h2 of cells k-1 .. k+2, one reciprocal of the common
// denominator (h0+h1)(2h0+h1)(2h1+h0)(hm+h0+h1+h2)
__device__ __forceinline__ float ppm_face(float q0, float q1, float dq0, float dq1, float hm,
                                          float h0, float h1, float h2)
{
    const float A = h0 + h1, B = 2.f * h0 + h1, C = 2.f * h1 + h0;
    const float S4 = hm + h0 + h1 + h2;
    const float a0 = hm + h0, a2 = h1 + h2;
    const float inv = rcp_approx(A * B * C * S4);
    const float kq = h0 * B * C * S4 + 2.f * h1 * h0 * (a0 * C - a2 * B);
    const float k1 = -h0 * a0 * A * C;  // coefficient of dq_{k+1}
    const float k0 = h1 * a2 * A * B;   // coefficient of dq_k
    return q0 + (kq * (q1 - q0) + k1 * dq1 + k0 * dq0) * inv;
}

// PPM parabola from its face values (App. A.2 second stage when limited) to the
// cumulative's coefficients: G/h = L xi + (R - L + Q6) xi^2 / 2 - Q6 xi^3 / 3.
template <bool LIM>
__device__ __forceinline__ void recon_ppm(float L, float R, float Q, float h, float b[4])
{
    if (LIM) {
        if ((R - Q) * (Q - L) <= 0.f) {
            L = Q;
            R = Q;
        } else {
            const float dd = R - L, qa = Q - 0.5f * (L + R);
            if (dd * qa > dd * dd * (1.f / 6.f))
                L = 3.f * Q - 2.f * R;
            else if (-dd * dd * (1.f / 6.f) > dd * qa)
                R = 3.f * Q - 2.f * L;
        }
    }
    const float Q6 = 6.f * Q - 3.f * (L + R);
    b[0] = h * L;
    b[1] = h * 0.5f * (R - L + Q6);
    b[2] = -h * Q6 * (1.f / 3.f);
    b[3] = 0.f;
}

// Order 4 (not in the paper): the mean of the quartic interpolants of the
// cumulative mass through the nodes {k-5/2..k+3/2} and {k-3/2..k+5/2}, in Newton
// form about x_{k-1/2} (z: node offsets in units of h0, v: cumulative mass / h0),
// expanded to the power basis.  q[0..4], h[0..4]: cells k-2 .. k+2.
template <bool LIM>
__device__ __forceinline__ void recon_quartic(const float *q, const float *h, float b[4])
{
    const float ih = rcp_approx(h[2]);
    const float z1 = -h[1] * ih, z0 = z1 - h[0] * ih;
    const float z4 = 1.f + h[3] * ih, z5 = z4 + h[4] * ih;
    const float v1 = -q[1] * h[1] * ih, v0 = v1 - q[0] * h[0] * ih;
    const float v3 = q[2], v4 = v3 + q[3] * h[3] * ih, v5 = v4 + q[4] * h[4] * ih;
    const float d1 = v3;
    const float f31 = (v1 - v3) * rcp_approx(z1 - 1.f);
    const float d2 = (f31 - d1) * rcp_approx(z1);
    const float f14 = (v4 - v1) * rcp_approx(z4 - z1);
    const float f314 = (f14 - f31) * rcp_approx(z4 - 1.f);
    const float d3 = (f314 - d2) * rcp_approx(z4);
    const float f40 = (v0 - v4) * rcp_approx(z0 - z4);
    const float f140 = (f40 - f14) * rcp_approx(z0 - z1);
    const float f3140 = (f140 - f314) * rcp_approx(z0 - 1.f);
    const float dL = (f3140 - d3) * rcp_approx(z0);
    const float f45 = (v5 - v4) * rcp_approx(z5 - z4);
    const float f145 = (f45 - f14) * rcp_approx(z5 - z1);
    const float f3145 = (f145 - f314) * rcp_approx(z5 - 1.f);
    const float dR = (f3145 - d3) * rcp_approx(z5);
    const float D = 0.5f * (dL + dR);
    // P(xi) = d1 + (xi - 1)(d2 + (xi - z1)(d3 + D (xi - z4))), G/h = xi P(xi)
    const float A0 = d3 - D * z4;                 // d3 + D(xi - z4) = A0 + D xi
    const float B0 = -z1 * A0, B1 = A0 - z1 * D;  // (xi - z1)(A0 + D xi)
    const float C0 = d2 + B0;                     // d2 + ... = C0 + B1 xi + D xi^2
    const float hh = h[2];
    float a1 = d1 - C0, a2 = C0 - B1, a3 = B1 - D, a4 = D;
    if (LIM) {
        // limited order 4: scaled toward the mean (Zhang-Shu), bounded by the cell
        // and its neighbours
        const float th = quartic_scaling_theta<float>(a1, a2, a3, a4, q[2],
                                                      fminf(q[2], fminf(q[1], q[3])),
                                                      fmaxf(q[2], fmaxf(q[1], q[3])));
        a1 = th * a1 + (1.f - th) * q[2];
        a2 *= th;
        a3 *= th;
        a4 *= th;
    }
    b[0] = hh * a1;
    b[1] = hh * a2;
    b[2] = hh * a3;
    b[3] = hh * a4;
}

// ---- packed pairs (two cells per float2, FP32 on the packed pipe) ----
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 s2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, s2(-1.f), a); }
__device__ __forceinline__ float2 rcp2(float2 a) { return f2(rcp_approx(a.x), rcp_approx(a.y)); }

// delta<Q> of App. A.1 for two cells (unlimited; see ppm_dq)
__device__ __forceinline__ float2 ppm_dq2(float2 qm, float2 q0, float2 qp, float2 a, float2 b,
                                          float2 c)
{
    const float2 up = sub2(qp, q0), dn = sub2(q0, qm);
    const float2 ab = add2(a, b), bc = add2(b, c);
    const float2 num = fma2(mul2(fma2(a, s2(2.f), b), ab), up, mul2(mul2(fma2(c, s2(2.f), b), bc), dn));
    const float2 den = mul2(mul2(add2(ab, c), bc), ab);
    return mul2(mul2(b, num), rcp2(den));
}

// interface values of App. A.1 for two interfaces (see ppm_face)
__device__ __forceinline__ float2 ppm_face2(float2 q0, float2 q1, float2 dq0, float2 dq1,
                                            float2 hm, float2 h0, float2 h1, float2 h2)
{
    const float2 A = add2(h0, h1), B = fma2(h0, s2(2.f), h1), C = fma2(h1, s2(2.f), h0);
    const float2 a0 = add2(hm, h0), a2 = add2(h1, h2);
    const float2 S4 = add2(a0, a2);
    const float2 AB = mul2(A, B), BC = mul2(B, C);
    const float2 inv = rcp2(mul2(AB, mul2(C, S4)));
    const float2 w1 = mul2(mul2(s2(2.f), mul2(h1, h0)), sub2(mul2(a0, C), mul2(a2, B)));
    const float2 kq = fma2(mul2(h0, BC), S4, w1);
    const float2 k1 = mul2(mul2(h0, a0), mul2(A, C));
    const float2 k0 = mul2(mul2(h1, a2), AB);
    const float2 t = fma2(k0, dq0, sub2(mul2(kq, sub2(q1, q0)), mul2(k1, dq1)));
    return fma2(t, inv, q0);
}

template <int ORDER>
__device__ __forceinline__ float eval_G(const float *c, int w, float xi)
{
    const int s = w;
    float g;
    if (ORDER == 2) {
        g = fmaf(xi, c[kSkewed + pz(s)], c[pz(s)]);
    } else if (ORDER == 3) {
        g = fmaf(xi, fmaf(xi, c[2 * kSkewed + pz(s)], c[kSkewed + pz(s)]), c[pz(s)]);
    } else {
        g = fmaf(xi, fmaf(xi, fmaf(xi, c[3 * kSkewed + pz(s)], c[2 * kSkewed + pz(s)]),
                          c[kSkewed + pz(s)]),
                 c[pz(s)]);
    }
    return xi * g;
}

// van Leer slope per unit length (Sec. 3.1) of cell u from its neighbours and
// the widths (mean-width units), zero at an extremum
__device__ __forceinline__ float vl_slope(const float *c, const float *w, int u)
{
    const float dl = c[u] - c[u - 1], dr = c[u + 1] - c[u];
    const float den = dl * (w[u] + w[u + 1]) + dr * (w[u - 1] + w[u]);
    return (dl * dr > 0.f) ? 4.f * dl * dr * rcp_approx(den) : 0.f;
}

// c in [0, 3n) reduced to [0, n)
__device__ __forceinline__ int wrap3(int c, int n)
{
    c = c >= n ? c - n : c;
    return c >= n ? c - n : c;
}

struct SegCtx {
    const uint64_t *X;
    const float *qin;
    float *qout;
    const float *dvp;
    int N, qshift, H, nsub, R;
    float scale, cf;
    uint64_t S;
    int *err;
};

// One segment of output cells [i0, i0 + cnt), extended by H on both sides.
template <int ORDER, bool LIM, bool RESID>
__device__ __forceinline__ void nseg_segment(const SegCtx &g, unsigned char *base,
                                             const NLayout &Lo, int lane, int i0, int cnt,
                                             int pA, int pB, uint64_t yA, uint64_t yB)
{
    uint32_t *sR = reinterpret_cast<uint32_t *>(base) + Lo.r;
    float *sQ = reinterpret_cast<float *>(base) + Lo.q;
    float *sH = reinterpret_cast<float *>(base) + Lo.h;
    float *sIW = reinterpret_cast<float *>(base) + Lo.iw;
    float *sC = reinterpret_cast<float *>(base) + Lo.c;
    const int N = g.N;
    const int ne = cnt + 2 * g.H;
    const int a0 = i0 - g.H < 0 ? i0 - g.H + N : i0 - g.H;  // first output cell (cyclic)
    const uint64_t xA = g.X[pA];
    int dist = pB - pA;
    dist = dist < 0 ? dist + N : dist;
    if (dist == 0) {
        // both outer edges in one source cell: inside it, or around the period
        const uint64_t wA = (pA + 1 < N ? g.X[pA + 1] : 0ull) - xA;
        if (yB - yA >= wA - (yA - xA)) dist = N;
    }
    const int W = dist + 1 + 2 * kHR;  // window cells
    if (W > kWcap) {
        if (lane == 0) atomicOr(g.err, ERR_WINDOW);
        return;
    }
    int cb = pA - kHR;
    cb = cb < 0 ? cb + N : cb;  // row cell of window cell 0
    // the nodes of the lane's first output edges, loaded before the window work
    uint64_t xo_first[kVE + 1];
    {
        const int j0 = lane * kVE;
#pragma unroll
        for (int e = 0; e <= kVE; ++e) xo_first[e] = g.X[wrap3(a0 + min(j0 + e, ne), N)];
    }
    const int qs = g.qshift;

    // ---- window cells: widths, positions and reconstructions, 4 per lane ----
    // Chunks of 128 cells overlapping by 4 (stride 124): lane l owns the chunk's
    // cells 4l..4l+3 and takes its stencil halo from lanes l-1 and l+1, so the
    // lanes at a chunk's ends lack one side; the overlap leaves those cells to
    // the neighbouring chunk (coefficients of local cells [lo, 126) are kept,
    // lo = 0 in the first chunk and 2 after it).
    for (int chunk = 0; kStride * chunk + 2 < W; ++chunk) {
        const int wc0 = kStride * chunk;
        const int w0 = wc0 + lane * kV;  // first of this lane's cells (window index)
        float q[kV];
        uint64_t xn[kV + 1];
        if (cb + wc0 + 32 * kV < N) {
            const uint64_t *xp = g.X + cb + w0;
            const float *qp = g.qin + cb + w0;
#pragma unroll
            for (int u = 0; u <= kV; ++u) {
                xn[u] = xp[u];
                if (u < kV) q[u] = qp[u];
            }
        } else {
#pragma unroll
            for (int u = 0; u <= kV; ++u) {
                // cells beyond the window read clamped (never used): cb + W < 3N
                const int c = wrap3(cb + min(w0 + u, W), N);
                xn[u] = g.X[c];
                if (u < kV) q[u] = g.qin[c];
            }
        }
        float h[kV];
        uint32_t r[kV + 1];
#pragma unroll
        for (int u = 0; u <= kV; ++u) r[u] = (uint32_t)((xn[u] - xA) >> qs);
#pragma unroll
        for (int u = 0; u < kV; ++u) h[u] = (float)(xn[u + 1] - xn[u]) * g.scale;
        // halo: cells -2, -1 of the lane from lane l-1, cells 4, 5 from lane l+1
        const float qm2 = __shfl_up_sync(0xffffffffu, q[2], 1), qm1 = __shfl_up_sync(0xffffffffu, q[3], 1);
        const float qp4 = __shfl_down_sync(0xffffffffu, q[0], 1), qp5 = __shfl_down_sync(0xffffffffu, q[1], 1);
        const float hm2 = __shfl_up_sync(0xffffffffu, h[2], 1), hm1 = __shfl_up_sync(0xffffffffu, h[3], 1);
        const float hp4 = __shfl_down_sync(0xffffffffu, h[0], 1), hp5 = __shfl_down_sync(0xffffffffu, h[1], 1);
        float b[kV][4];
        if (ORDER == 2) {
            if (LIM) {
                recon_plm<true>(qm1, q[0], q[1], hm1, h[0], h[1], b[0]);
                recon_plm<true>(q[0], q[1], q[2], h[0], h[1], h[2], b[1]);
                recon_plm<true>(q[1], q[2], q[3], h[1], h[2], h[3], b[2]);
                recon_plm<true>(q[2], q[3], qp4, h[2], h[3], hp4, b[3]);
            } else {
                // sigma h = 2 (q+ - q-) h / (h- + 2h + h+), pairs (0,2) and (1,3)
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const float2 qm = i == 0 ? f2(qm1, q[1]) : f2(q[0], q[2]);
                    const float2 qc = f2(q[i], q[i + 2]);
                    const float2 qp = i == 0 ? f2(q[1], q[3]) : f2(q[2], qp4);
                    const float2 hm = i == 0 ? f2(hm1, h[1]) : f2(h[0], h[2]);
                    const float2 hc = f2(h[i], h[i + 2]);
                    const float2 hp = i == 0 ? f2(h[1], h[3]) : f2(h[2], hp4);
                    const float2 sh = mul2(mul2(mul2(s2(2.f), sub2(qp, qm)), hc),
                                           rcp2(add2(fma2(hc, s2(2.f), hm), hp)));
                    const float2 b0 = mul2(hc, fma2(sh, s2(-0.5f), qc));
                    const float2 b1 = mul2(mul2(hc, s2(0.5f)), sh);
                    b[i][0] = b0.x;
                    b[i + 2][0] = b0.y;
                    b[i][1] = b1.x;
                    b[i + 2][1] = b1.y;
                }
            }
        } else if (ORDER == 3) {
            // delta<Q> of cells 0..3 (pairs (0,2), (1,3)); cell 4's from lane l+1
            float dq[kV + 1];
            if (LIM) {
                dq[0] = ppm_dq<true>(qm1, q[0], q[1], hm1, h[0], h[1]);
                dq[1] = ppm_dq<true>(q[0], q[1], q[2], h[0], h[1], h[2]);
                dq[2] = ppm_dq<true>(q[1], q[2], q[3], h[1], h[2], h[3]);
                dq[3] = ppm_dq<true>(q[2], q[3], qp4, h[2], h[3], hp4);
            } else {
                const float2 d02 = ppm_dq2(f2(qm1, q[1]), f2(q[0], q[2]), f2(q[1], q[3]),
                                           f2(hm1, h[1]), f2(h[0], h[2]), f2(h[1], h[3]));
                const float2 d13 = ppm_dq2(f2(q[0], q[2]), f2(q[1], q[3]), f2(q[2], qp4),
                                           f2(h[0], h[2]), f2(h[1], h[3]), f2(h[2], hp4));
                dq[0] = d02.x;
                dq[2] = d02.y;
                dq[1] = d13.x;
                dq[3] = d13.y;
            }
            dq[4] = __shfl_down_sync(0xffffffffu, dq[0], 1);
            // faces i + 1/2 of cells 0..3 (pairs (0,2), (1,3)); face -1/2 from lane l-1
            const float2 f02 = ppm_face2(f2(q[0], q[2]), f2(q[1], q[3]), f2(dq[0], dq[2]),
                                         f2(dq[1], dq[3]), f2(hm1, h[1]), f2(h[0], h[2]),
                                         f2(h[1], h[3]), f2(h[2], hp4));
            const float2 f13 = ppm_face2(f2(q[1], q[3]), f2(q[2], qp4), f2(dq[1], dq[3]),
                                         f2(dq[2], dq[4]), f2(h[0], h[2]), f2(h[1], h[3]),
                                         f2(h[2], hp4), f2(h[3], hp5));
            const float fm1 = __shfl_up_sync(0xffffffffu, f13.y, 1);
            const float fc[kV + 1] = {fm1, f02.x, f13.x, f02.y, f13.y};  // faces -1/2 .. 3+1/2
            if (LIM) {
#pragma unroll
                for (int i = 0; i < kV; ++i) recon_ppm<true>(fc[i], fc[i + 1], q[i], h[i], b[i]);
            } else {
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const float2 L = f2(fc[i], fc[i + 2]), R = f2(fc[i + 1], fc[i + 3]);
                    const float2 Q = f2(q[i], q[i + 2]), hc = f2(h[i], h[i + 2]);
                    const float2 Q6 = fma2(s2(-3.f), add2(L, R), mul2(s2(6.f), Q));
                    const float2 b0 = mul2(hc, L);
                    const float2 b1 = mul2(mul2(hc, s2(0.5f)), add2(sub2(R, L), Q6));
                    const float2 b2 = mul2(mul2(hc, s2(-1.f / 3.f)), Q6);
                    b[i][0] = b0.x;
                    b[i + 2][0] = b0.y;
                    b[i][1] = b1.x;
                    b[i + 2][1] = b1.y;
                    b[i][2] = b2.x;
                    b[i + 2][2] = b2.y;
                }
            }
        } else {
            const float qs_[kV + 4] = {qm2, qm1, q[0], q[1], q[2], q[3], qp4, qp5};
            const float hs_[kV + 4] = {hm2, hm1, h[0], h[1], h[2], h[3], hp4, hp5};
#pragma unroll
            for (int i = 0; i < kV; ++i) recon_quartic<LIM>(qs_ + i, hs_ + i, b[i]);
        }
        const int lo = chunk == 0 ? 0 : 2;
        const int sb = w0;
#pragma unroll
        for (int i = 0; i < kV; ++i) {
            const int s = sb + i;
            sR[pz(s)] = r[i];
            sQ[pz(s)] = q[i];
            sH[pz(s)] = h[i];
            sIW[pz(s)] = rcp_approx((float)(r[i + 1] - r[i]));
            const int wl = lane * kV + i;  // cell within the chunk
            if (wl >= lo && wl < kStride + 2) {
#pragma unroll
                for (int k = 0; k < ORDER; ++k) sC[k * kSkewed + pz(s)] = b[i][k];
            }
        }
        if (lane == 31) sR[pz(w0 + kV)] = r[kV];  // the chunk's last node
    }
    __syncwarp();

    float *sP = nullptr;
    if (RESID) sP = reinterpret_cast<float *>(base) + Lo.p;
    // ---- shifted edges and output masses (Eqs. 16, 18, 26) ----
    const uint64_t off = g.S + xA;  // window-relative position of a shifted node: x - off
    const int hiw = W - kHR;        // node after the last edge cell
    for (int jc = 0; jc < ne; jc += 32 * kVE) {
        const int j0 = jc + lane * kVE;
        // lanes past the end work on the last edge and store nothing
        uint64_t xo[kVE + 1];
        const bool inside = a0 + j0 + kVE < N && j0 + kVE <= ne;
#pragma unroll
        for (int e = 0; e <= kVE; ++e)
            xo[e] = inside ? xo_first[e] : g.X[wrap3(a0 + min(j0 + e, ne), N)];
        if (jc > 0 && inside) {
#pragma unroll
            for (int e = 0; e <= kVE; ++e) xo[e] = g.X[a0 + j0 + e];
        }
        int we[kVE + 1];
        uint32_t de[kVE + 1];
        float G[kVE + 1];
        int w = kHR;
#pragma unroll
        for (int e = 0; e <= kVE; ++e) {
            const uint32_t ry = (uint32_t)((xo[e] - off) >> qs);
            if (e == 0) {
                // the last node at or left of ry among nodes kHR .. hiw - 1: fixed steps
#pragma unroll
                for (int step = 128; step > 0; step >>= 1) {
                    const int m = w + step;
                    if (m < hiw && sR[pz(m)] <= ry) w = m;
                }
            } else {
                // a walk: mostly zero, one or two nodes
                if (w + 1 < hiw && sR[pz(w + 1)] <= ry) {
                    ++w;
                    while (w + 1 < hiw && sR[pz(w + 1)] <= ry) ++w;
                }
            }
            const uint32_t d = ry - sR[pz(w)];
            we[e] = w;
            de[e] = d;
            G[e] = eval_G<ORDER>(sC, w, (float)d * sIW[pz(w)]);
        }
#pragma unroll
        for (int e = 0; e < kVE; ++e) {
            const int wl = we[e], wr = we[e + 1];
            const float wo = (float)(xo[e + 1] - xo[e]) * g.scale;
            // Eq. 18: inside one source cell, or the rest of cell wl, the whole cells
            // in between and the start of cell wr
            float mass = G[e + 1] - G[e];
            if (wr != wl) {
                mass += sQ[pz(wl)] * sH[pz(wl)];
                for (int m = wl + 1; m < wr; ++m) mass += sQ[pz(m)] * sH[pz(m)];
            }
            // both edges on the nodes of one source cell: its value unchanged
            const float val = ((de[e] | de[e + 1]) == 0 && wr == wl + 1) ? sQ[pz(wl)]
                                                                         : mass * rcp_approx(wo);
            if (j0 + e < ne) {
                if (RESID) {
                    sP[j0 + e] = val;
                } else {
                    g.qout[i0 + j0 + e] = val;
                }
            }
        }
    }
    if (RESID) {
        // ---- residual sub-steps (Eq. 6) on the extended segment ----
        // the coefficient arrays are free once every lane has left the edges
        __syncwarp();
        float *sWo = sC, *sP2 = sC + kSkewed, *sV = sC + 2 * kSkewed, *sF = sC + 3 * kSkewed;
        static_assert(kSkewed >= kEmax + 1, "the residual's arrays fit the coefficient arrays");
        for (int j = lane; j < ne; j += 32)
            sWo[j] = (float)(g.X[wrap3(a0 + j + 1, N)] - g.X[wrap3(a0 + j, N)]) * g.scale;
        for (int j = lane; j <= ne; j += 32) sV[j] = g.dvp[wrap3(a0 + j, N)];
        __syncwarp();
        const int R = g.R;
        float *cur = sP, *nxt = sP2;
        bool cfl_bad = false;
        for (int ks = 0; ks < g.nsub; ++ks) {
            const int lo = ks * R + R, hi = ne - ks * R - R;
            for (int j = lo + lane; j <= hi; j += 32) {
                const float c = sV[j] * g.cf;
                float flux = 0.f;
                if (c > 0.f) {
                    const int u = j - 1;
                    float qh = cur[u];
                    if (R == 2) qh += 0.5f * vl_slope(cur, sWo, u) * (sWo[u] - c);
                    flux = c * qh;
                    cfl_bad |= c > sWo[u];
                } else if (c < 0.f) {
                    const int u = j;
                    float qh = cur[u];
                    if (R == 2) qh -= 0.5f * vl_slope(cur, sWo, u) * (sWo[u] + c);
                    flux = c * qh;
                    cfl_bad |= -c > sWo[u];
                }
                sF[j] = flux;
            }
            __syncwarp();
            for (int j = lo + lane; j < hi; j += 32)
                nxt[j] = cur[j] - (sF[j + 1] - sF[j]) * rcp_approx(sWo[j]);
            __syncwarp();
            float *tt = cur;
            cur = nxt;
            nxt = tt;
        }
        if (__any_sync(0xffffffffu, cfl_bad) && lane == 0) atomicOr(g.err, ERR_CFL);
        for (int j = lane; j < cnt; j += 32) g.qout[i0 + j] = cur[g.H + j];
    }
    __syncwarp();
}

template <bool LIM, bool RESID>
__global__ void __launch_bounds__(kNsegWarps * 32, 3)
    k_nseg(StepArgs a, const Tile *tiles)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Tile t = tiles[blockIdx.x];
    const RowInfo row = a.rows[t.row];
    const int N = row.n;
    const int seg = t.window;  // output cells per segment of this row
    const int nsegs = (t.count + seg - 1) / seg;
    if (warp >= nsegs) {
        pdl_wait();
        pdl_trigger();
        return;
    }
    const uint64_t *X = a.xfix + row.mesh_off;
    const int32_t *bt = a.buckets + row.bucket_off;

    // the residual halo of the row (the sub-step count as shift_params clamps it)
    int H = 0;
    if (RESID) {
        int ns = a.nsub ? a.nsub[t.row] : 1;
        ns = ns < 1 ? 1 : (ns > RAM_MAX_NSUB ? RAM_MAX_NSUB : ns);
        H = ns * (a.scheme == RAM_VANLEER ? 2 : 1);
    }
    // lane 2m + side holds the outer edge `side` of the warp's m-th segment
    // (segments warp, warp + kNsegWarps, ...); the nodes are plan data, read
    // before the wait
    const int kk = warp + (lane >> 1) * kNsegWarps;
    const bool locator = lane < 2 * kNsegPerWarp && kk < nsegs;
    uint64_t xe = 0;
    if (locator) {
        const int i0 = t.start + kk * seg;
        const int cnt = min(seg, t.start + t.count - i0);
        int e = (lane & 1) ? i0 + cnt + H : i0 - H;
        e = e < 0 ? e + N : (e >= N ? e - N : e);
        xe = X[e];
    }
    // the previous kernel in the stream may still be writing q and the phase
    pdl_wait();
    pdl_trigger();
    // S0 once per warp (FP64, lane 0); the row's first tile's first warp advances
    // the phase when no parameter kernel ran
    uint64_t S = 0;
    int nsub = 0;
    float cf = 0.f;
    if (lane == 0) {
        RowParams<float> P;
        shift_params<float>(a, row, t.row, a.row_phase != 0 && t.start == 0 && warp == 0, P);
        S = P.sfix;
        nsub = P.nsub;
        cf = P.cf * (float)row.cells_per_length;  // Courant number per unit dv
    }
    S = ((uint64_t)__shfl_sync(0xffffffffu, (uint32_t)(S >> 32), 0) << 32) |
        (uint64_t)__shfl_sync(0xffffffffu, (uint32_t)S, 0);
    nsub = __shfl_sync(0xffffffffu, nsub, 0);
    cf = __shfl_sync(0xffffffffu, cf, 0);
    int p = 0;
    const uint64_t y = xe - S;
    if (locator) {
        p = locate_cell(X, N, bt, row.bucket_bits, a.density, row.density, y);
    }

    const NLayout Lo = nseg_layout(RESID);
    unsigned char *base = smem_raw + (size_t)warp * Lo.total * 4;
    SegCtx g;
    g.X = X;
    g.qin = static_cast<const float *>(a.q_in) + row.cell_off;
    g.qout = static_cast<float *>(a.q_out) + row.cell_off;
    g.dvp = RESID ? static_cast<const float *>(a.dv) + row.cell_off : nullptr;
    g.N = N;
    g.qshift = row.qshift;
    g.H = H;
    g.nsub = nsub;
    g.R = (a.scheme == RAM_VANLEER) ? 2 : 1;
    g.scale = (float)N * 0x1p-64f;  // fixed-point length -> mean widths
    g.cf = cf;
    g.S = S;
    g.err = a.err;

#define RAM_NSEG_LOOP(ORD)                                                                 \
    for (int m = 0; m < kNsegPerWarp; ++m) {                                               \
        const int k = warp + m * kNsegWarps;                                               \
        if (k >= nsegs) break;                                                             \
        const int i0 = t.start + k * seg;                                                  \
        const int cnt = min(seg, t.start + t.count - i0);                                  \
        const int pA = __shfl_sync(0xffffffffu, p, 2 * m);                                 \
        const int pB = __shfl_sync(0xffffffffu, p, 2 * m + 1);                             \
        const uint64_t yA = ((uint64_t)__shfl_sync(0xffffffffu, (uint32_t)(y >> 32), 2 * m) \
                             << 32) | __shfl_sync(0xffffffffu, (uint32_t)y, 2 * m);         \
        const uint64_t yB =                                                                \
            ((uint64_t)__shfl_sync(0xffffffffu, (uint32_t)(y >> 32), 2 * m + 1) << 32) |   \
            __shfl_sync(0xffffffffu, (uint32_t)y, 2 * m + 1);                              \
        nseg_segment<ORD, LIM, RESID>(g, base, Lo, lane, i0, cnt, pA, pB, yA, yB);         \
    }
    if (row.order == 2) {
        RAM_NSEG_LOOP(2)
    } else if (row.order == 3) {
        RAM_NSEG_LOOP(3)
    } else {
        RAM_NSEG_LOOP(4)
    }
#undef RAM_NSEG_LOOP
}

}  // namespace

size_t nseg_smem_bytes(bool resid) { return (size_t)kNsegWarps * nseg_layout(resid).total * 4; }

int nseg_window_cap() { return kWcap; }

cudaError_t launch_nseg(const Plan &p, const StepArgs &a, cudaStream_t s)
{
    const int n = (int)p.tiles_nseg_h.size();
    if (n == 0) return cudaSuccess;
    const bool resid = a.mode != MODE_SHIFT && a.dv != nullptr;
    const size_t smem = nseg_smem_bytes(resid);
    if (smem > 227 * 1024) return cudaErrorNotSupported;
    void (*kern)(StepArgs, const Tile *) =
        p.limiter ? (resid ? k_nseg<true, true> : k_nseg<true, false>)
                  : (resid ? k_nseg<false, true> : k_nseg<false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, n, kNsegWarps * 32, smem, s, a, p.tiles_nseg);
}

}  // namespace ram
