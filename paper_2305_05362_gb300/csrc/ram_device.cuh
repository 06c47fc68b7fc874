// Device helpers shared by the RAM kernels: shift reduction (S0), the
// reconstructions of Sec. 3.1 / App. A on uniform rows, and the residual flux.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ram_internal.h"

namespace ram {

// 1/x from the hardware reciprocal approximation (rcp.approx: relative error
// about 2^-23; subnormal results flush to zero)
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// a / b in the cells' precision.  FP32: the product with the approximate
// reciprocal (two instructions; a few ulp, far below what the FP32 results are
// held to); FP64: the IEEE quotient.
template <typename T> struct Num;
template <> struct Num<float> {
    static __device__ __forceinline__ float div(float a, float b) { return a * rcp_approx(b); }
};
template <> struct Num<double> {
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
};

// min(|a|, |b|) carrying the sign sign(a) xor sign(b): positive when a and b have
// the same sign.  With it the limiters of App. A.2 need no compare-and-select:
// median(0, x, y) = sign(x) max(minxs(x, y), 0).
__device__ __forceinline__ float minxs(float a, float b)
{
    float d;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ double minxs(double a, double b)
{
    const double m = fmin(fabs(a), fabs(b));
    return __longlong_as_double(__double_as_longlong(m) |
                                ((__double_as_longlong(a) ^ __double_as_longlong(b)) &
                                 (long long)0x8000000000000000ull));
}
// g with its sign flipped where a is negative
__device__ __forceinline__ float xorsign(float g, float a)
{
    return __int_as_float(__float_as_int(g) ^ (__float_as_int(a) & 0x80000000));
}
__device__ __forceinline__ double xorsign(double g, double a)
{
    return __longlong_as_double(__double_as_longlong(g) ^
                                (__double_as_longlong(a) & (long long)0x8000000000000000ull));
}

// Reduce x to [0, p) with a floor-mod in FP64 (the shift may be any real).
__device__ __forceinline__ double reduce_mod(double x, double p)
{
    double r = __dsub_rn(x, __dmul_rn(p, floor(__ddiv_rn(x, p))));
    if (r >= p) r -= p;
    if (r < 0.0) r += p;
    if (r >= p) r = 0.0;
    return r;
}

// Floor-mod with a precomputed reciprocal of the period: no FP64 divide (an FP64
// divide costs hundreds of cycles of latency on this part).  The result is
// brought into [0, p) by the fix-ups below.
__device__ __forceinline__ double reduce_mod_rcp(double x, double p, double inv_p)
{
    double r = fma(-p, floor(x * inv_p), x);
    if (r >= p) r -= p;
    if (r < 0.0) r += p;
    if (r >= p) r = 0.0;
    return r;
}

// 1/n for the residual sub-step counts 0..RAM_MAX_NSUB
__device__ __forceinline__ double inv_small(int n)
{
    const double t[9] = {0.0, 1.0, 0.5, 1.0 / 3.0, 0.25, 0.2, 1.0 / 6.0, 1.0 / 7.0, 0.125};
    return t[n];
}

// van Leer harmonic slope (Sec. 3.1) in undivided form (slope x width) on a
// uniform row: 2 dl dr / (dl + dr) when dl dr > 0, else 0.
template <typename T>
__device__ __forceinline__ T vl_slope_u(T qm, T q0, T qp)
{
    T dl = q0 - qm, dr = qp - q0;
    T pr = dl * dr;
    return pr > T(0) ? Num<T>::div(T(2) * pr, dl + dr) : T(0);
}

// delta<Q>_i of App. A on a uniform row, limited by App. A.2 when lim.
template <typename T>
__device__ __forceinline__ T ppm_dq_u(T qm, T q0, T qp, bool lim)
{
    T d = T(0.5) * (qp - qm);
    if (lim) {
        T up = qp - q0, dn = q0 - qm;
        if (up * dn > T(0)) {
            T m = fmin(fabs(d), fmin(T(2) * fabs(dn), T(2) * fabs(up)));
            d = copysign(m, d);
        } else {
            d = T(0);
        }
    }
    return d;
}

// PPM parabola (QL, QR, Q6) of the centre cell from five uniform-row values
// (App. A: <Q>_{i+1/2} = (Q_i + Q_{i+1})/2 - (dQ_{i+1} - dQ_i)/6 on a uniform
// mesh; App. A.2 constraints when lim).
template <typename T>
__device__ __forceinline__ void ppm_u(T qm2, T qm1, T q0, T qp1, T qp2, bool lim, T &QL,
                                      T &QR, T &Q6)
{
    const T dqm = ppm_dq_u(qm2, qm1, q0, lim);
    const T dq0 = ppm_dq_u(qm1, q0, qp1, lim);
    const T dqp = ppm_dq_u(q0, qp1, qp2, lim);
    const T sixth = T(1) / T(6);
    T L = T(0.5) * (qm1 + q0) - (dq0 - dqm) * sixth;
    T R = T(0.5) * (q0 + qp1) - (dqp - dq0) * sixth;
    if (lim) {
        if ((R - q0) * (q0 - L) <= T(0)) {
            L = q0;
            R = q0;
        } else {
            const T dd = R - L;
            const T qa = q0 - T(0.5) * (L + R);
            if (dd * qa > dd * dd * sixth)
                L = T(3) * q0 - T(2) * R;
            else if (-dd * dd * sixth > dd * qa)
                R = T(3) * q0 - T(2) * L;
        }
    }
    QL = L;
    QR = R;
    Q6 = T(6) * q0 - T(3) * (L + R);
}

// Lagrange weights of the order-4 cumulative on a uniform row at offset xi
// (in cell widths): the mean of the quartics through the nodes
// {-2,-1,0,1,2} and {-1,0,1,2,3} (in cells, relative to the cell's left node),
// folded into five coefficients c[k] of Q_{i-2+k} so that G/dx = sum c[k] Q.
// The Lagrange denominators of five equally spaced nodes are 24, -6, 4, -6, 24.
template <typename U>
__device__ __forceinline__ void quartic_coeffs_u(U xi, U c[5])
{
    const U inv_den[5] = {U(1) / U(24), U(-1) / U(6), U(0.25), U(-1) / U(6), U(1) / U(24)};
    U w[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int side = 0; side < 2; ++side) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            U l = inv_den[k];
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if (j != k) l *= xi - (U)(side + j - 2);
            w[side + k] += U(0.5) * l;
        }
    }
    // node values relative to the cell's left node, in units of dx:
    // v = {-(Q_{i-2}+Q_{i-1}), -Q_{i-1}, 0, Q_i, Q_i+Q_{i+1}, Q_i+Q_{i+1}+Q_{i+2}}
    c[0] = -w[0];
    c[1] = -w[0] - w[1];
    c[2] = w[3] + w[4] + w[5];
    c[3] = w[4] + w[5];
    c[4] = w[5];
}

// Coefficients of the left partial integral G/dx at the edge offset xi for the
// row's order (computed in U, stored in T):
//   PLM  G/dx = Q xi + slope (xi^2 - xi)/2                      c = {xi, (xi^2 - xi)/2}
//   PPM  G/dx = QL (xi - xi^2/2) + QR xi^2/2 + Q6 (xi^2/2 - xi^3/3), folded with
//        Q6 = 6Q - 3(QL + QR) into coefficients of QL, QR and Q (c[0..2]; c[3] = xi,
//        the coefficient of Q once QL, QR are written as Q - b, Q + a)
//   order 4: Lagrange weights of the two quartics of the cumulative mass.
template <typename U, typename T>
__device__ __forceinline__ void partial_coeffs(int order, U xi, T (&c)[5])
{
    for (int j = 0; j < 5; ++j) c[j] = T(0);
    if (order == 2) {
        c[0] = (T)xi;
        c[1] = (T)(U(0.5) * (xi * xi - xi));
    } else if (order == 3) {
        const U c0 = xi - U(0.5) * xi * xi, c1 = U(0.5) * xi * xi;
        const U c6 = U(0.5) * xi * xi - xi * xi * xi * (U(1) / U(3));
        c[0] = (T)(c0 - U(3) * c6);
        c[1] = (T)(c1 - U(3) * c6);
        c[2] = (T)(U(6) * c6);
        c[3] = (T)xi;
    } else {
        U w[5];
        quartic_coeffs_u(xi, w);
        for (int j = 0; j < 5; ++j) c[j] = (T)w[j];
    }
}

// The shift parameters of one row for one launch (S0), in FP64: the bulk
// displacement s (the given shift, v0 dt, or zero for the residual step alone;
// a non-finite value is flagged and replaced by zero), the accumulated phase
// (advanced by s when update_phase), the fixed-point shift of rows with their
// own mesh, and for uniform rows sig = (s mod L) N / L split into K = floor(sig)
// whole cells and the fraction f, with the coefficients of the left partial
// integral at the edge offset xi = 1 - f (partial_coeffs); and cf = dt / (nsub
// dx), the Courant number per unit dv of one residual sub-step.  Returns xi.
// Every kernel that needs these values computes them with this function, so
// they agree bit for bit.
template <typename T>
__device__ __forceinline__ double shift_params(const StepArgs &a, const RowInfo &row, int r,
                                               bool update_phase, RowParams<T> &P)
{
    // every global read of the row first, so that their latencies overlap (the
    // parameter kernel runs on cold caches right before the row kernels)
    const bool has_dv = (a.mode != MODE_SHIFT) && (a.dv != nullptr);
    const bool do_phase = update_phase && a.mode == MODE_STEP && a.phase != nullptr;
    const double s_in = a.mode == MODE_SHIFT ? a.shift[r] : (a.mode == MODE_STEP ? a.v0[r] : 0.0);
    const int ns_in = has_dv ? (a.nsub ? a.nsub[r] : 1) : 0;
    const double ph_in = do_phase ? a.phase[r] : 0.0;
    const int N = row.n;
    P.cell_off = row.cell_off;
    P.n = N;
    double sft = a.mode == MODE_STEP ? __dmul_rn(s_in, a.dt) : s_in;
    if (!isfinite(sft)) {
        atomicOr(a.err, ERR_NONFINITE);
        sft = 0.0;
    }
    if (do_phase) a.phase[r] = reduce_mod_rcp(ph_in + sft, row.period, row.inv_period);
    const double sred = reduce_mod_rcp(sft, row.period, row.inv_period);
    // fixed-point shift for rows with their own mesh: nodes are stored as fractions
    // of the period in units of 2^-64, so x - s and the periodic wrap are exact
    // integer arithmetic (uniform rows locate their edges by index instead)
    // (uniform rows locate their edges by index; the adjoint of a limited plan
    // locates them by position on every row)
    const double t = sred * row.inv_period;  // in [0, 1]
    P.sfix = (t >= 1.0) ? 0ull : __double2ull_rn(t * 18446744073709551616.0);
    double sig = sred * row.cells_per_length;
    if (sig >= (double)N) sig -= (double)N;
    const double Kd = floor(sig);
    const double f = sig - Kd;
    P.K = (int)Kd;
    P.whole = (f == 0.0);
    const double xi = 1.0 - f;
    // the coefficients in the precision of the cells: FP64 work per row is what
    // decides K and f (an FP64 instruction costs a warp tens of cycles on this
    // part, so FP32 rows keep it to the few operations above)
    if (sizeof(T) == 4)
        partial_coeffs<float>(row.order, (float)xi, P.c);
    else
        partial_coeffs<double>(row.order, xi, P.c);
    int nsub = 0;
    P.cf = T(0);
    if (has_dv) {
        nsub = ns_in;
        if (nsub < 1 || nsub > RAM_MAX_NSUB) {
            atomicOr(a.err, ERR_NSUB);
            nsub = nsub < 1 ? 1 : RAM_MAX_NSUB;
        }
        if (sizeof(T) == 4)
            P.cf = (T)(row.uniform ? a.dt * row.cells_per_length : a.dt) / (T)nsub;
        else
            P.cf = row.uniform ? (T)(a.dt * row.cells_per_length * inv_small(nsub))
                               : (T)(a.dt * inv_small(nsub));
    }
    P.nsub = nsub;
    return xi;
}

// ---- two-float arithmetic for the shift of FP32 rows ----
// A value is carried as an unevaluated sum h + l of two floats (about 48
// significant bits).  The products use the error-free transformations of
// floating-point arithmetic: the exact product of two floats is p + e with
// p = fl(a b) and e = fma(a, b, -p), and for |a| >= |b| the exact sum is
// s + (b - (s - a)) with s = fl(a + b) (Dekker's fast two-sum).  All of it runs
// on the FP32 and integer pipes: an FP64 instruction costs a warp tens of cycles
// on this part, and every CTA of a row kernel would pay that on its critical
// path.
struct TwoFloat {
    float h, l;
};

__device__ __forceinline__ TwoFloat two_mul(TwoFloat a, TwoFloat b)
{
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    const float s = p + e;
    return {s, e - (s - p)};
}

// x as h + l from its bits (no FP64 instruction): h holds the leading 24 bits of
// the significand, l the next 29 rounded to 24.  False for a non-finite x or
// |x| >= 2^127; |x| < 2^-100 gives zero.
__device__ __forceinline__ bool split_f64(double x, TwoFloat &out)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned hi32 = (unsigned)(u >> 32);
    const int E = (int)((hi32 >> 20) & 0x7FFu) - 1023;
    out.h = 0.0f;
    out.l = 0.0f;
    if (E == 1024 || E > 126) return false;
    if (E < -100) return true;
    const unsigned long long M = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const unsigned sign = hi32 & 0x80000000u;
    out.h = __uint_as_float(sign | ((unsigned)(E + 127) << 23) | ((unsigned)(M >> 29) & 0x7FFFFFu));
    // the low 29 bits are worth R 2^(E - 52) = (R 2^-29) 2^(E - 23), E - 23 in [-123, 103]
    const float lo = __uint2float_rn((unsigned)(M & 0x1FFFFFFFu)) * 0x1p-29f *
                     __uint_as_float((unsigned)(E - 23 + 127) << 23);
    out.l = sign ? -lo : lo;
    return true;
}

// The shift parameters of one FP32 uniform row (S0 on a uniform mesh, Sec. 3.2.1),
// computed in two-float arithmetic: sig = s N / L, with s = v0 dt (step), the
// given shift, or zero (residual alone), is split into K = floor(sig) mod N
// whole cells and the fraction f, and xi = 1 - f gives the coefficients of the
// left partial integral (partial_coeffs); cf = dt N / (L nsub).  The same
// quantities as shift_params to about 2^-46 relative in sig, which the FP32
// cells do not resolve.  A non-finite shift, or one of 2^40 cells or more, is
// flagged (by `lead`) and replaced by zero.  The phase is not touched.
__device__ __forceinline__ void shift_params_two_float(const StepArgs &a, const RowInfo &row,
                                                       int r, bool lead, RowParams<float> &P)
{
    const bool has_dv = (a.mode != MODE_SHIFT) && (a.dv != nullptr);
    const double s_in = a.mode == MODE_SHIFT ? a.shift[r] : (a.mode == MODE_STEP ? a.v0[r] : 0.0);
    const int ns_in = has_dv ? (a.nsub ? a.nsub[r] : 1) : 0;
    const int N = row.n;
    P.cell_off = row.cell_off;
    P.n = N;
    P.sfix = 0ull;
    TwoFloat cpl, dtc = {0.0f, 0.0f}, sig = {0.0f, 0.0f};
    split_f64(row.cells_per_length, cpl);
    bool fin = true;
    if (a.mode != MODE_SHIFT) {
        TwoFloat dt;
        fin = split_f64(a.dt, dt);
        dtc = two_mul(dt, cpl);
    }
    if (a.mode == MODE_STEP || a.mode == MODE_SHIFT) {
        TwoFloat sv;
        fin = split_f64(s_in, sv) && fin;
        sig = two_mul(sv, a.mode == MODE_STEP ? dtc : cpl);
    }
    if (!fin || !(fabsf(sig.h) < 0x1p40f)) {
        if (lead) atomicOr(a.err, ERR_NONFINITE);
        sig.h = sig.l = 0.0f;
    }
    // floor(h + l) = floor(h) + floor(c), c = (h - floor(h)) + l: h - floor(h) is
    // exact, and c lies in (-1, 2)
    const float fh = floorf(sig.h);
    const float c = (sig.h - fh) + sig.l;
    float fc = floorf(c);
    float f = c - fc;
    if (f >= 1.0f) {  // c just below an integer
        f = 0.0f;
        fc += 1.0f;
    }
    int K;
    if (fabsf(fh) < 0x1p24f) {
        K = ((int)fh + (int)fc) % N;
    } else {
        K = (int)(((long long)fh + (long long)fc) % (long long)N);
    }
    if (K < 0) K += N;
    P.K = K;
    P.whole = (f == 0.0f);
    partial_coeffs<float>(row.order, 1.0f - f, P.c);
    int nsub = 0;
    P.cf = 0.0f;
    if (has_dv) {
        nsub = ns_in;
        if (nsub < 1 || nsub > RAM_MAX_NSUB) {
            if (lead) atomicOr(a.err, ERR_NSUB);
            nsub = nsub < 1 ? 1 : RAM_MAX_NSUB;
        }
        P.cf = (dtc.h + dtc.l) / (float)nsub;
    }
    P.nsub = nsub;
}

// The phase update of shift_params on its own (MODE_STEP with a phase array):
// phase += v0 dt (zero when not finite), reduced to [0, L), in FP64.
__device__ __forceinline__ void advance_phase(const StepArgs &a, const RowInfo &row, int r)
{
    if (a.mode != MODE_STEP || a.phase == nullptr) return;
    double sft = __dmul_rn(a.v0[r], a.dt);
    if (!isfinite(sft)) sft = 0.0;
    a.phase[r] = reduce_mod_rcp(a.phase[r] + sft, row.period, row.inv_period);
}

// Limited order 4: the scaling toward the cell mean of the maximum-principle
// limiter of Zhang & Shu (2010).  a1..a4 are the power-basis coefficients of the
// in-cell cumulative G(xi h) / h = a1 xi + a2 xi^2 + a3 xi^3 + a4 xi^4, so the
// profile is q(xi) = a1 + 2 a2 xi + 3 a3 xi^2 + 4 a4 xi^3; its extremes over the
// cell are at the ends or at the real roots of q' inside it.  Returns the largest
// theta in [0, 1] with Q + theta (q - Q) inside [lo, hi] on the whole cell.
template <typename T>
__device__ __forceinline__ T quartic_scaling_theta(T a1, T a2, T a3, T a4, T Q, T lo, T hi)
{
    T qmax = a1, qmin = a1;  // xi = 0
    const T q1 = a1 + T(2) * a2 + T(3) * a3 + T(4) * a4;  // xi = 1
    qmax = fmax(qmax, q1);
    qmin = fmin(qmin, q1);
    // q'(xi) = 2 a2 + 6 a3 xi + 12 a4 xi^2
    const T A = T(12) * a4, B = T(6) * a3, C = T(2) * a2;
    T r[2];
    int nr = 0;
    if (fabs(A) > T(1e-30)) {
        const T disc = B * B - T(4) * A * C;
        if (disc >= T(0)) {
            const T sq = sqrt(disc);
            r[0] = (-B - sq) / (T(2) * A);
            r[1] = (-B + sq) / (T(2) * A);
            nr = 2;
        }
    } else if (fabs(B) > T(1e-30)) {
        r[0] = -C / B;
        nr = 1;
    }
    for (int k = 0; k < nr; ++k) {
        const T x = r[k];
        if (x > T(0) && x < T(1)) {
            const T v = a1 + x * (T(2) * a2 + x * (T(3) * a3 + x * T(4) * a4));
            qmax = fmax(qmax, v);
            qmin = fmin(qmin, v);
        }
    }
    T th = T(1);
    if (qmax > hi && qmax - Q > T(0)) th = fmin(th, (hi - Q) / (qmax - Q));
    if (qmin < lo && qmin - Q < T(0)) th = fmin(th, (lo - Q) / (qmin - Q));
    return fmax(th, T(0));
}

// The index function of Sec. 3.2.1 for a row generated by a mesh-density function
// (App. B.1, the periodic bump): the nodes satisfy u(x_j) = j / N with u the
// normalised cumulative of the density, so the cell holding x is floor(N u(x)).
// u is evaluated in FP32 from its closed form; the caller corrects the guess
// against the row's exact nodes (at most a step or two).
__device__ __forceinline__ int density_index(const Density &d, int n, uint64_t y)
{
    const float x = d.x_min + d.L * ((float)(y >> 40) * 0x1p-24f);  // position of y
    const float t = fabsf(x);
    const float w = d.b - d.a;
    const float tt = fminf(fmaxf(t, d.a), d.b);
    // integral of the unnormalised density from 0 to |x|, signed
    float pr = (1.f + d.c) * fminf(t, d.a) + (tt - d.a) +
               d.c * (0.5f * (tt - d.a) + w * (0.5f / 3.14159265358979f) *
                                              __sinf(3.14159265358979f * (tt - d.a) / w)) +
               fmaxf(t - d.b, 0.f);
    pr = x < 0.f ? -pr : pr;
    const float u = (pr - d.prim_min) * d.inv_norm;
    const int p = (int)floorf(u * (float)n);
    return p < 0 ? 0 : (p >= n ? n - 1 : p);
}

// The source cell p of a row with x_p <= y < x_{p+1} (Eq. 16), y a position as a
// fraction of the period in units of 2^-64 (the nodes X likewise, X[0] = 0): a
// first guess from the index function of the row's density when it has one,
// else from the plan's bucket table (the index function tabulated on the row's
// own nodes), then a walk along the exact nodes.
__device__ __forceinline__ int locate_cell(const uint64_t *X, int n, const int32_t *bt, int bits,
                                           const Density *dens, int di, uint64_t y)
{
    int p;
    if (di >= 0) {
        p = density_index(dens[di], n, y);
        while (p > 0 && X[p] > y) --p;
    } else {
        p = bt[y >> (64 - bits)];
    }
    while (p + 1 < n && X[p + 1] <= y) ++p;
    return p;
}

// Wait until the kernels this one depends on (programmatic dependent launch)
// have finished and their writes are visible; a no-op for a normal launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Let the next kernel in the stream launch now (it waits for this one's results
// with pdl_wait).
__device__ __forceinline__ void pdl_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// i reduced to [0, n).  The tiled kernels call it per cell with i within one
// period of the row, where one compare-and-add does it; a 64-bit remainder (a
// long software sequence) is left for the far cases (rows shorter than a halo).
__device__ __forceinline__ int wrap_index(int64_t i, int n)
{
    if (i >= -(int64_t)n && i < 2 * (int64_t)n) {
        int x = (int)i;
        if (x < 0)
            x += n;
        else if (x >= n)
            x -= n;
        return x;
    }
    int64_t k = i % n;
    return (int)(k < 0 ? k + n : k);
}

// x >= 0 reduced to [0, n), with the same fast path.
__device__ __forceinline__ int wrap_pos(int x, int n)
{
    if (x < n) return x;
    if (x < 2 * n) return x - n;
    return x % n;
}

}  // namespace ram
