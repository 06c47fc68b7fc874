// RAM step on rows with their own non-uniform mesh (Sec. 3 on an arbitrary
// periodic mesh), and the per-row mass diagnostic.
//
// Steps without a residual run k_gwarp (below): warps split each tile, each lane
// locates its own edges and gathers the source stencils from the cache, with no
// shared memory or barriers.  Steps with a residual run k_general:
//
// One CTA per tile of output cells.  The tile's source window -- the source
// cells its shifted edges land in, plus the reconstruction halo -- is found
// from the plan's bucket table (the index function of Sec. 3.2.1 tabulated on
// the row's own nodes) and staged in shared memory.  Node positions are
// fixed-point fractions of the period (units of 2^-64), so x - s and the
// periodic wrap are exact integer arithmetic.  Then, on chip:
//   - the prefix sum of the window's cell masses M = Q dx (Eq. 3): a block scan,
//     two-float compensated for FP32 cells (exact products, ~48-bit sums), FP64
//     for FP64 cells;
//   - every shifted edge is located in the window (Eq. 16; a binary search for
//     the first of a thread's run of edges, a walk for the others) and the
//     in-cell cumulative G_p(d) of its source cell's reconstruction is
//     evaluated (PLM / PPM of App. A / order 4);
//   - each output cell's mass is Eq. 18: right part of p(i), the whole cells in
//     between as a difference of the scan, left part of p(i+1); Q = M / dx
//     (Eq. 26);
//   - the residual sub-steps (Eq. 6) with per-cell widths.
// Short rows are one tile covering the whole row cyclically (a launch of their
// own, sized for the largest of them).
#include <cuda_runtime.h>

#include <cstdint>

#include "ram_device.cuh"

namespace ram {
namespace {

constexpr int kHalo = kGenHalo;  // residual halo, cells per side (max)
constexpr int kHR = kGenHR;      // reconstruction halo, cells per side

// ---------------- compensated accumulation ----------------
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ DF fast_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}

template <typename T> struct Acc;

template <> struct Acc<float> {
    using A = DF;
    static __device__ __forceinline__ A zero() { return {0.f, 0.f}; }
    // the exact product q dx as a two-float value
    static __device__ __forceinline__ A mass(float q, float dx)
    {
        const float p = q * dx;
        return {p, fmaf(q, dx, -p)};
    }
    static __device__ __forceinline__ A add(A a, A b)
    {
        const DF s = two_sum(a.hi, b.hi);
        return fast_two_sum(s.hi, s.lo + a.lo + b.lo);
    }
    static __device__ __forceinline__ float diff(A a, A b) { return (a.hi - b.hi) + (a.lo - b.lo); }
    static __device__ __forceinline__ A shfl_up(A a, int d)
    {
        return {__shfl_up_sync(0xffffffffu, a.hi, d), __shfl_up_sync(0xffffffffu, a.lo, d)};
    }
    static __device__ __forceinline__ A shfl_down(A a, int d)
    {
        return {__shfl_down_sync(0xffffffffu, a.hi, d), __shfl_down_sync(0xffffffffu, a.lo, d)};
    }
    static __device__ __forceinline__ double to_double(A a) { return (double)a.hi + (double)a.lo; }
};

template <> struct Acc<double> {
    using A = double;
    static __device__ __forceinline__ A zero() { return 0.0; }
    static __device__ __forceinline__ A mass(double q, double dx) { return q * dx; }
    static __device__ __forceinline__ A add(A a, A b) { return a + b; }
    static __device__ __forceinline__ double diff(A a, A b) { return a - b; }
    static __device__ __forceinline__ A shfl_up(A a, int d) { return __shfl_up_sync(0xffffffffu, a, d); }
    static __device__ __forceinline__ A shfl_down(A a, int d)
    {
        return __shfl_down_sync(0xffffffffu, a, d);
    }
    static __device__ __forceinline__ double to_double(A a) { return a; }
};

// Exclusive prefix sums S[v] = sum_{u=lo}^{v-1} q[u] dx[u] for v = lo..hi (S[hi] is the
// total), over the whole block.  wt: 32 accumulators of shared scratch.
template <typename T>
__device__ void block_scan(const T *q, const T *dx, int lo, int hi, typename Acc<T>::A *S,
                           typename Acc<T>::A *wt)
{
    using AC = Acc<T>;
    using A = typename AC::A;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int n = hi - lo;
    const int per = (n + nth - 1) / nth;
    const int b = lo + min(n, tid * per), e = lo + min(n, (tid + 1) * per);
    A local = AC::zero();
    for (int v = b; v < e; ++v) local = AC::add(local, AC::mass(q[v], dx[v]));
    A incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const A t = AC::shfl_up(incl, o);
        if (lane >= o) incl = AC::add(t, incl);
    }
    if (lane == 31) wt[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = nth >> 5;
        A x = lane < nw ? wt[lane] : AC::zero();
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const A t = AC::shfl_up(x, o);
            if (lane >= o) x = AC::add(t, x);
        }
        if (lane < nw) wt[lane] = x;
    }
    __syncthreads();
    A excl = AC::shfl_up(incl, 1);
    if (lane == 0) excl = AC::zero();
    A run = warp > 0 ? AC::add(wt[warp - 1], excl) : excl;
    for (int v = b; v < e; ++v) {
        S[v] = run;
        run = AC::add(run, AC::mass(q[v], dx[v]));
    }
    if (e == hi && b < e) S[hi] = run;
    if (n == 0 && tid == 0) S[lo] = AC::zero();
    __syncthreads();
}

// ---------------- reconstruction at a window slot (Sec. 3.1, App. A) ----------------

// van Leer slope per unit length with centre spacings (Sec. 3.1); centred slope
// when the limiter is off
template <typename T>
__device__ __forceinline__ T plm_slope(const T *q, const T *dx, int p, bool lim)
{
    const T hl = T(0.5) * (dx[p - 1] + dx[p]), hr = T(0.5) * (dx[p] + dx[p + 1]);
    if (!lim) return Num<T>::div(q[p + 1] - q[p - 1], hl + hr);
    const T dl = Num<T>::div(q[p] - q[p - 1], hl), dr = Num<T>::div(q[p + 1] - q[p], hr);
    const T pr = dl * dr;
    return pr > T(0) ? Num<T>::div(T(2) * pr, dl + dr) : T(0);
}

// delta<Q>_k of App. A on a non-uniform mesh (limited by App. A.2)
template <typename T>
__device__ __forceinline__ T ppm_dq(const T *q, const T *dx, int k, bool lim)
{
    const T a = dx[k - 1], b = dx[k], c = dx[k + 1];
    const T up = q[k + 1] - q[k], dn = q[k] - q[k - 1];
    T d = Num<T>::div(b, a + b + c) *
          (Num<T>::div(T(2) * a + b, b + c) * up + Num<T>::div(b + T(2) * c, a + b) * dn);
    if (lim) {
        if (up * dn > T(0)) {
            const T m = fmin(fabs(d), fmin(T(2) * fabs(dn), T(2) * fabs(up)));
            d = copysign(m, d);
        } else {
            d = T(0);
        }
    }
    return d;
}

// interface value <Q>_{k+1/2} of App. A (with sums of widths in the weights)
template <typename T>
__device__ __forceinline__ T ppm_face(const T *q, const T *dx, int k, T dqk, T dqk1)
{
    const T hm = dx[k - 1], h0 = dx[k], h1 = dx[k + 1], h2 = dx[k + 2];
    const T w1 = Num<T>::div(T(2) * h1 * h0, h0 + h1) *
                 (Num<T>::div(hm + h0, T(2) * h0 + h1) - Num<T>::div(h2 + h1, T(2) * h1 + h0));
    const T w2 = -h0 * Num<T>::div(hm + h0, T(2) * h0 + h1);
    const T w3 = h1 * Num<T>::div(h1 + h2, h0 + T(2) * h1);
    const T sum4 = hm + h0 + h1 + h2;
    return q[k] + Num<T>::div(h0, h0 + h1) * (q[k + 1] - q[k]) +
           Num<T>::div(w1 * (q[k + 1] - q[k]) + w2 * dqk1 + w3 * dqk, sum4);
}

// in-cell cumulative G_p(xi dx_p) = integral of q_p over its first xi of the cell
template <typename T, int ORDER>
__device__ T cell_G(const T *q, const T *dx, int p, T xi, bool lim)
{
    const T h = dx[p];
    if (ORDER == 2) {
        const T s = plm_slope(q, dx, p, lim);
        return h * (q[p] * xi + T(0.5) * s * h * (xi * xi - xi));
    } else if (ORDER == 3) {
        const T dqm = ppm_dq(q, dx, p - 1, lim), dq0 = ppm_dq(q, dx, p, lim),
                dqp = ppm_dq(q, dx, p + 1, lim);
        T L = ppm_face(q, dx, p - 1, dqm, dq0), R = ppm_face(q, dx, p, dq0, dqp);
        const T Q = q[p];
        if (lim) {
            if ((R - Q) * (Q - L) <= T(0)) {
                L = Q;
                R = Q;
            } else {
                const T dd = R - L, qa = Q - T(0.5) * (L + R);
                if (dd * qa > dd * dd * (T(1) / T(6)))
                    L = T(3) * Q - T(2) * R;
                else if (-dd * dd * (T(1) / T(6)) > dd * qa)
                    R = T(3) * Q - T(2) * L;
            }
        }
        const T Q6 = T(6) * Q - T(3) * (L + R);
        const T x2 = xi * xi;
        return h * (L * (xi - T(0.5) * x2) + R * T(0.5) * x2 +
                    Q6 * (T(0.5) * x2 - x2 * xi * (T(1) / T(3))));
    } else {
        // mean of the quartic interpolants of the cumulative mass through the nodes
        // {p-5/2..p+3/2} and {p-3/2..p+5/2}, in Newton form about x_{p-1/2}
        // (z: node offsets in units of dx_p; v: cumulative mass / dx_p)
        const T z0 = -Num<T>::div(dx[p - 2] + dx[p - 1], h), z1 = -Num<T>::div(dx[p - 1], h);
        const T z4 = T(1) + Num<T>::div(dx[p + 1], h);
        const T z5 = z4 + Num<T>::div(dx[p + 2], h);
        const T m2 = q[p - 2] * dx[p - 2], m1 = q[p - 1] * dx[p - 1];
        const T p1 = q[p + 1] * dx[p + 1], p2 = q[p + 2] * dx[p + 2];
        const T v0 = -Num<T>::div(m2 + m1, h), v1 = -Num<T>::div(m1, h), v3 = q[p];
        const T v4 = v3 + Num<T>::div(p1, h), v5 = v4 + Num<T>::div(p2, h);
        const T d1 = v3;                                        // f[z2,z3]
        const T f31 = Num<T>::div(v1 - v3, z1 - T(1));          // f[z3,z1]
        const T d2 = Num<T>::div(f31 - d1, z1);                 // f[z2,z3,z1]
        const T f14 = Num<T>::div(v4 - v1, z4 - z1);            // f[z1,z4]
        const T f314 = Num<T>::div(f14 - f31, z4 - T(1));       // f[z3,z1,z4]
        const T d3 = Num<T>::div(f314 - d2, z4);                // f[z2,z3,z1,z4]
        const T f40 = Num<T>::div(v0 - v4, z0 - z4);
        const T f140 = Num<T>::div(f40 - f14, z0 - z1);
        const T f3140 = Num<T>::div(f140 - f314, z0 - T(1));
        const T dL = Num<T>::div(f3140 - d3, z0);
        const T f45 = Num<T>::div(v5 - v4, z5 - z4);
        const T f145 = Num<T>::div(f45 - f14, z5 - z1);
        const T f3145 = Num<T>::div(f145 - f314, z5 - T(1));
        const T dR = Num<T>::div(f3145 - d3, z5);
        const T D = T(0.5) * (dL + dR);
        const T g = xi * (d1 + (xi - T(1)) * (d2 + (xi - z1) * (d3 + D * (xi - z4))));
        if (!lim) return h * g;
        // limited order 4: the profile scaled toward the mean (Zhang-Shu), bounded by
        // the cell and its neighbours; the power-basis coefficients of G/h first
        const T A0 = d3 - D * z4, B0 = -z1 * A0, B1 = A0 - z1 * D, C0 = d2 + B0;
        const T th = quartic_scaling_theta<T>(d1 - C0, C0 - B1, B1 - D, D, q[p],
                                              fmin(q[p], fmin(q[p - 1], q[p + 1])),
                                              fmax(q[p], fmax(q[p - 1], q[p + 1])));
        return h * (th * g + (T(1) - th) * q[p] * xi);
    }
}

__device__ __forceinline__ float u64_to(uint64_t v, float) { return __ull2float_rn(v); }
__device__ __forceinline__ double u64_to(uint64_t v, double) { return __ull2double_rn(v); }

template <typename T>
__device__ __forceinline__ T vl_slope_nu(const T *c, const T *w, int u)
{
    const T hl = T(0.5) * (w[u - 1] + w[u]), hr = T(0.5) * (w[u] + w[u + 1]);
    const T dl = Num<T>::div(c[u] - c[u - 1], hl), dr = Num<T>::div(c[u + 1] - c[u], hr);
    const T pr = dl * dr;
    return pr > T(0) ? Num<T>::div(T(2) * pr, dl + dr) : T(0);
}

// Byte offsets of the general kernel's shared arrays (window of wcap cells,
// wcap + 1 nodes; qcap output cells, qcap + 1 edges; the residual's arrays only
// when a residual step runs); one function serves the kernel's carve-up and the
// launcher's size.
struct GLayout {
    size_t sY, sS, sXo, wt, sQ, sDX, sEG, sDXo, sP, sP2, sV, sF, sEp, total;
};

template <typename T>
__host__ __device__ inline GLayout general_layout(int wcap, int qcap, bool resid)
{
    using A = typename Acc<T>::A;
    GLayout L;
    size_t o = 0;
    auto put = [&o](size_t bytes) {
        const size_t at = o;
        o += (bytes + 15) / 16 * 16;
        return at;
    };
    L.sY = put(sizeof(uint64_t) * (wcap + 1));
    L.sS = put(sizeof(A) * (wcap + 1));
    L.sXo = put(sizeof(uint64_t) * (qcap + 1));
    L.wt = put(sizeof(A) * 32);
    L.sQ = put(sizeof(T) * wcap);
    L.sDX = put(sizeof(T) * wcap);
    L.sEG = put(sizeof(T) * (qcap + 1));
    L.sDXo = put(sizeof(T) * qcap);
    L.sP = put(sizeof(T) * qcap);
    L.sP2 = put(resid ? sizeof(T) * qcap : 0);
    L.sV = put(resid ? sizeof(T) * (qcap + 1) : 0);
    L.sF = put(resid ? sizeof(T) * (qcap + 1) : 0);
    L.sEp = put(sizeof(int) * (qcap + 1));
    L.total = o;
    return L;
}

template <typename T, int ORDER>
__global__ void __launch_bounds__(512)
    k_general(StepArgs a, int wcap, int qcap, int resid, int wait, const RowParams<T> *pars)
{
    using AC = Acc<T>;
    using A = typename AC::A;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const GLayout L = general_layout<T>(wcap, qcap, resid != 0);
    uint64_t *sY = reinterpret_cast<uint64_t *>(smem_raw + L.sY);    // wcap + 1
    A *sS = reinterpret_cast<A *>(smem_raw + L.sS);                  // wcap + 1
    uint64_t *sXo = reinterpret_cast<uint64_t *>(smem_raw + L.sXo);  // qcap + 1
    A *wt = reinterpret_cast<A *>(smem_raw + L.wt);                  // 32
    T *sQ = reinterpret_cast<T *>(smem_raw + L.sQ);                  // wcap
    T *sDX = reinterpret_cast<T *>(smem_raw + L.sDX);                // wcap
    T *sEG = reinterpret_cast<T *>(smem_raw + L.sEG);                // qcap + 1
    T *sDXo = reinterpret_cast<T *>(smem_raw + L.sDXo);              // qcap
    T *sP = reinterpret_cast<T *>(smem_raw + L.sP);                  // qcap
    T *sP2 = reinterpret_cast<T *>(smem_raw + L.sP2);                // qcap
    T *sV = reinterpret_cast<T *>(smem_raw + L.sV);                  // qcap + 1
    T *sF = reinterpret_cast<T *>(smem_raw + L.sF);                  // qcap + 1
    int *sEp = reinterpret_cast<int *>(smem_raw + L.sEp);            // qcap + 1

    __shared__ int s_plo, s_W, s_bad;
    __shared__ uint64_t s_xbase;

    const int tid = threadIdx.x, nth = blockDim.x;
    const Tile tile = a.tiles[blockIdx.x];
    const RowInfo row = a.rows[tile.row];
    const int N = row.n;
    const uint64_t *X = a.xfix + row.mesh_off;
    const T *DX = (sizeof(T) == 4) ? reinterpret_cast<const T *>(a.dx32 + row.mesh_off)
                                   : reinterpret_cast<const T *>(a.dx64 + row.mesh_off);
    const int32_t *bt = a.buckets + row.bucket_off;
    const T *qin = static_cast<const T *>(a.q_in) + row.cell_off;
    T *qout = static_cast<T *>(a.q_out) + row.cell_off;
    const bool lim = a.limiter != 0;

    // The first general launch of a step waits for the parameter kernel; the
    // later ones are launched once it has (each launch lets the next start as
    // soon as its own wait is over) and touch other rows, so they run alongside.
    if (wait) pdl_wait();
    pdl_trigger();
    const RowParams<T> P = pars[tile.row];
    const uint64_t S = P.sfix;
    const int nsub = P.nsub;
    const int R = (a.scheme == RAM_VANLEER) ? 2 : 1;
    const int H = nsub * R;
    const int T_out = tile.count;
    const int nq = T_out + 2 * H;
    const bool whole = tile.window == 0;

    // ---- the source window, and the output side's nodes, widths and dv ----
    // Lanes 0 and 1 locate the source cells of the tile's two outer edges at the
    // same time (each a short chain of dependent loads: the node, its bucket, a
    // walk); the other threads meanwhile load the output side, which does not
    // depend on the window.
    if (tid < 32) {
        int plo = 0, W = N + 2 * kHR;
        uint64_t xbase = 0;
        if (!whole) {
            int p = 0;
            if (tid < 2) {
                const int e = tid == 0 ? wrap_index((int64_t)tile.start - H, N)
                                       : wrap_index((int64_t)tile.start + T_out + H, N);
                p = locate_cell(X, N, bt, row.bucket_bits, a.density, row.density, X[e] - S);
            }
            const int phi = __shfl_sync(0xffffffffu, p, 1);
            plo = p;
            W = (phi - plo + N) % N + 1 + 2 * kHR;
            if (tid == 0) xbase = X[plo];
        }
        if (tid == 0) {
            s_plo = plo;
            s_W = W;
            s_xbase = xbase;
            s_bad = (W > wcap);
            if (s_bad) atomicOr(a.err, ERR_WINDOW);
        }
    }
    // output cells a-H .. a+T+H (cyclic): node positions, widths, dv
    for (int j = tid; j <= nq; j += nth) {
        const int e = wrap_index((int64_t)tile.start - H + j, N);
        sXo[j] = X[e];
        if (j < nq) sDXo[j] = DX[e];
    }
    const T *dvp = (a.mode != MODE_SHIFT && a.dv != nullptr)
                       ? static_cast<const T *>(a.dv) + row.cell_off
                       : nullptr;
    if (nsub > 0)
        for (int j = tid; j <= nq; j += nth) sV[j] = dvp[wrap_index((int64_t)tile.start - H + j, N)];
    __syncthreads();
    if (s_bad) return;
    const int plo = s_plo, W = s_W;
    const uint64_t xbase = s_xbase;
    const int wb = wrap_index((int64_t)plo - kHR, N);  // cell of slot 0
    for (int w = tid; w < W; w += nth) {
        const int c = wrap_pos(wb + w, N);
        sQ[w] = qin[c];
        sDX[w] = DX[c];
    }
    for (int w = kHR + tid; w <= W - kHR; w += nth) sY[w] = X[wrap_pos(wb + w, N)] - xbase;
    __syncthreads();

    // ---- prefix sum of the window masses (Eq. 18's whole-cell sums) ----
    block_scan<T>(sQ, sDX, kHR, W - kHR, sS, wt);

    // ---- shifted edges: source cell, offset, in-cell cumulative (Eq. 16) ----
    // A thread takes a contiguous run of edges: the first is located by binary
    // search over the window's nodes, the next ones by walking on from there
    // (shifted edges and nodes both increase; a whole-row tile's edges drop back
    // once, at the seam, and are searched again).
    const int ne = nq + 1;
    const int per = (ne + nth - 1) / nth;
    const int j0 = min(ne, tid * per), j1 = min(ne, j0 + per);
    int lo = kHR;
    for (int j = j0; j < j1; ++j) {
        const uint64_t y = sXo[j] - S - xbase;
        if (j == j0 || y < sY[lo]) {
            lo = kHR;
            int hi = W - kHR;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (sY[mid] <= y)
                    lo = mid;
                else
                    hi = mid;
            }
        } else {
            while (lo + 1 < W - kHR && sY[lo + 1] <= y) ++lo;
        }
        const uint64_t d = y - sY[lo];
        const uint64_t width = sY[lo + 1] - sY[lo];
        const T xi = Num<T>::div(u64_to(d, T(0)), u64_to(width, T(0)));
        sEp[j] = lo;
        sEG[j] = (d == 0) ? T(0) : cell_G<T, ORDER>(sQ, sDX, lo, xi, lim);
    }
    __syncthreads();

    // ---- output masses (Eq. 18) and cell averages (Eq. 26) ----
    for (int j = tid; j < nq; j += nth) {
        const int pL = sEp[j], pR = sEp[j + 1];
        const uint64_t yL = sXo[j] - S - xbase, yR = sXo[j + 1] - S - xbase;
        const bool wrap = whole && (yR <= yL);
        const T GL = sEG[j], GR = sEG[j + 1];
        T val;
        const int pnext = (whole && pL + 1 == N + kHR) ? kHR : pL + 1;
        const bool exact = (yL == sY[pL]) && (yR == sY[pR]) && (pR == pnext) && !(pL == pR) &&
                           (sY[pL + 1] - sY[pL]) == (sXo[j + 1] - sXo[j]);
        if (exact) {
            val = sQ[pL];  // the output cell is exactly one source cell: copy it
        } else {
            T mass;
            if (!wrap && pL == pR) {
                mass = GR - GL;
            } else {
                T whole_cells;
                if (wrap)
                    whole_cells = AC::diff(sS[W - kHR], sS[pL + 1]) + AC::diff(sS[pR], sS[kHR]);
                else
                    whole_cells = AC::diff(sS[pR], sS[pL + 1]);
                mass = (sQ[pL] * sDX[pL] - GL) + whole_cells + GR;
            }
            val = Num<T>::div(mass, sDXo[j]);
        }
        sP[j] = val;
    }

    // ---- residual sub-steps (Eq. 6) with per-cell widths ----
    T *cur = sP, *nxt = sP2;
    if (nsub > 0) {
        const T h = P.cf;  // sub-step length
        const bool vl = a.scheme == RAM_VANLEER;
        __syncthreads();
        for (int k = 0; k < nsub; ++k) {
            const int lo = k * R + R, hi = nq - k * R - R;
            bool cfl_bad = false;
            for (int j = lo + tid; j <= hi; j += nth) {
                const T c = sV[j] * h;
                T flux = T(0);
                if (c > T(0)) {
                    const int u = j - 1;
                    T qh = cur[u];
                    if (vl) qh += T(0.5) * vl_slope_nu(cur, sDXo, u) * (sDXo[u] - c);
                    flux = c * qh;
                    cfl_bad |= c > sDXo[u];
                } else if (c < T(0)) {
                    const int u = j;
                    T qh = cur[u];
                    if (vl) qh -= T(0.5) * vl_slope_nu(cur, sDXo, u) * (sDXo[u] + c);
                    flux = c * qh;
                    cfl_bad |= -c > sDXo[u];
                }
                sF[j] = flux;
            }
            if (cfl_bad) atomicOr(a.err, ERR_CFL);
            __syncthreads();
            for (int j = lo + tid; j < hi; j += nth)
                nxt[j] = cur[j] - Num<T>::div(sF[j + 1] - sF[j], sDXo[j]);
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

// The shift step alone (no residual) on non-uniform rows, without shared
// memory: the warps of a CTA split a tile's output cells into chunks of 32 V,
// lane l taking V consecutive cells.  Per output edge a lane locates the source
// cell of the shifted node (the bucket table for its first edge, then a walk
// along the row's nodes; Eq. 16), gathers the cell's stencil from global memory
// (cached) and evaluates the in-cell cumulative (cell_G); per output cell it
// sums the whole source cells between its two edges directly (Eq. 18, in the
// order of the cells) and divides by the cell's width (Eq. 26).  No barriers:
// the warps and CTAs interleave their loads and arithmetic freely.
template <typename T, int ORDER, int V>
__global__ void __launch_bounds__(512)
    k_gwarp(StepArgs a, int wait, const RowParams<T> *pars)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const Tile tile = a.tiles[blockIdx.x];
    const RowInfo row = a.rows[tile.row];
    const int N = row.n;
    const uint64_t *X = a.xfix + row.mesh_off;
    const T *DX = (sizeof(T) == 4) ? reinterpret_cast<const T *>(a.dx32 + row.mesh_off)
                                   : reinterpret_cast<const T *>(a.dx64 + row.mesh_off);
    const int32_t *bt = a.buckets + row.bucket_off;
    const T *qin = static_cast<const T *>(a.q_in) + row.cell_off;
    T *qout = static_cast<T *>(a.q_out) + row.cell_off;
    const bool lim = a.limiter != 0;

    if (wait) pdl_wait();
    pdl_trigger();
    const uint64_t S = pars[tile.row].sfix;
    constexpr int HS = ORDER == 2 ? 1 : 2;  // stencil half-width of cell_G

    for (int c0 = warp * 32 * V; c0 < tile.count; c0 += nwarps * 32 * V) {
        const int i0 = c0 + lane * V;  // this lane's first output cell in the tile
        const int nc = min(V, tile.count - i0);
        if (nc <= 0) continue;
        // the lane's nc + 1 edges: source cell, shifted position, in-cell cumulative
        int pe[V + 1];
        uint64_t ye[V + 1];
        T G[V + 1];
        int p = 0;
        uint64_t yprev = 0;
#pragma unroll
        for (int k = 0; k <= V; ++k) {
            if (k > nc) break;
            // edge nodes run from tile.start to at most N (node N is node 0)
            const int en = tile.start + i0 + k;
            const int e = en < N ? en : en - N;
            const uint64_t y = X[e] - S;
            if (k == 0 || y < yprev) {
                p = locate_cell(X, N, bt, row.bucket_bits, a.density, row.density, y);
            } else {
                while (p + 1 < N && X[p + 1] <= y) ++p;
            }
            yprev = y;
            const uint64_t xp = X[p];
            const uint64_t xn = p + 1 < N ? X[p + 1] : 0ull;  // the period's end is 2^64 = 0
            const uint64_t d = y - xp;
            pe[k] = p;
            ye[k] = y;
            if (d == 0) {
                G[k] = T(0);
            } else {
                T qs[2 * HS + 1], ds[2 * HS + 1];
                if (p >= HS && p + HS < N) {
#pragma unroll
                    for (int u = 0; u <= 2 * HS; ++u) {
                        qs[u] = qin[p - HS + u];
                        ds[u] = DX[p - HS + u];
                    }
                } else {
#pragma unroll
                    for (int u = 0; u <= 2 * HS; ++u) {
                        const int c = wrap_index((int64_t)p - HS + u, N);
                        qs[u] = qin[c];
                        ds[u] = DX[c];
                    }
                }
                const T xi = Num<T>::div(u64_to(d, T(0)), u64_to(xn - xp, T(0)));
                G[k] = cell_G<T, ORDER>(qs, ds, HS, xi, lim);
            }
        }
#pragma unroll
        for (int k = 0; k < V; ++k) {
            if (k >= nc) break;
            const int g = tile.start + i0 + k;  // output cell (< N)
            const int pL = pe[k], pR = pe[k + 1];
            const uint64_t dL = ye[k] - X[pL], dR = ye[k + 1] - X[pR];
            const uint64_t wsrc = (pL + 1 < N ? X[pL + 1] : 0ull) - X[pL];
            const uint64_t wout = (g + 1 < N ? X[g + 1] : 0ull) - X[g];
            const int pnext = pL + 1 < N ? pL + 1 : 0;
            T val;
            if (dL == 0 && dR == 0 && pR == pnext && pL != pR && wsrc == wout) {
                val = qin[pL];  // the output cell is exactly one source cell: copy it
            } else {
                T mass;
                if (pL == pR && dR > dL) {
                    mass = G[k + 1] - G[k];  // inside one source cell
                } else {
                    // the rest of cell pL, the whole cells up to pR (cyclic), the start of pR
                    mass = qin[pL] * DX[pL] - G[k];
                    int m = pnext;
                    while (m != pR) {
                        mass += qin[m] * DX[m];
                        m = m + 1 < N ? m + 1 : 0;
                    }
                    mass += G[k + 1];
                }
                val = Num<T>::div(mass, DX[g]);
            }
            qout[g] = val;
        }
    }
}

// A list of non-uniform tiles of one order for the general kernels: every row's
// (FP64) or the rows the FP32 warp-segment kernel does not take.
struct GenList {
    const Tile *tiles;
    int n, whole;
    const int32_t *wcap, *qcap;  // [2]: whole-row and windowed classes
};

GenList gen_list(const Plan &p, int order, bool f32)
{
    if (f32 && p.nu_kernel == 1)
        return {p.tiles_general32[order], (int)p.tiles_general32_h[order].size(),
                p.gen32_whole[order], p.gen32_wcap[order], p.gen32_qcap[order]};
    return {p.tiles_general[order], (int)p.tiles_general_h[order].size(), p.gen_whole[order],
            p.gen_wcap[order], p.gen_qcap[order]};
}

template <typename T, int ORDER>
cudaError_t launch_general_class(const Plan &p, const GenList &gl, const StepArgs &a0,
                                 cudaStream_t s, int first, int count, int wcap, int qcap,
                                 int &launched)
{
    if (count == 0) return cudaSuccess;
    const bool resid = a0.mode != MODE_SHIFT && a0.dv != nullptr;
    const size_t smem = general_layout<T>(wcap, qcap, resid).total;
    if (smem > 227 * 1024) return cudaErrorNotSupported;
    static size_t configured[64] = {0};
    const int dev = p.device < 64 ? p.device : 63;
    if (smem > configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_general<T, ORDER>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured[dev] = smem;
    }
    StepArgs a = a0;
    a.tiles = gl.tiles + first;
    a.n_tiles = count;
    // the plan's threads per CTA (every phase of a tile strides over its cells)
    const int threads = p.threads < 512 ? p.threads : 512;
    cudaError_t e = launch_pdl(k_general<T, ORDER>, count, threads, smem, s, a, wcap, qcap,
                               resid ? 1 : 0, launched == 0 ? 1 : 0,
                               static_cast<const RowParams<T> *>(p.row_par));
    if (e == cudaSuccess) ++launched;
    return e;
}

// Whole-row tiles (short rows) and windowed tiles run as two launches, each with
// the shared memory of its own largest tile (plan-time sizes).
// output cells per lane of k_gwarp (FP32: three amortise a lane's bucket lookup
// and loads better than two; measured on the 512-row batch)
template <typename T> constexpr int kGwarpV = sizeof(T) == 4 ? 3 : 2;

template <typename T, int ORDER>
cudaError_t launch_general_t(const Plan &p, const StepArgs &a0, cudaStream_t s, int &launched)
{
    const GenList gl = gen_list(p, ORDER, sizeof(T) == 4);
    const int n = gl.n;
    if (n == 0) return cudaSuccess;
    if (a0.mode == MODE_SHIFT || a0.dv == nullptr) {
        // no residual: the shared-memory-free kernel takes every tile in one launch
        StepArgs a = a0;
        a.tiles = gl.tiles;
        a.n_tiles = n;
        const int threads = p.threads < 512 ? p.threads : 512;
        cudaError_t e = launch_pdl(k_gwarp<T, ORDER, kGwarpV<T>>, n, threads, 0, s, a,
                                   launched == 0 ? 1 : 0,
                                   static_cast<const RowParams<T> *>(p.row_par));
        if (e == cudaSuccess) ++launched;
        return e;
    }
    const int nw = gl.whole;
    cudaError_t e = launch_general_class<T, ORDER>(p, gl, a0, s, 0, nw, gl.wcap[0], gl.qcap[0],
                                                   launched);
    if (e != cudaSuccess) return e;
    return launch_general_class<T, ORDER>(p, gl, a0, s, nw, n - nw, gl.wcap[1], gl.qcap[1],
                                          launched);
}

// ---------------- per-row mass (Eq. 10) ----------------
template <typename T>
__global__ void __launch_bounds__(256) k_mass(const RowInfo *rows, const float *dx32,
                                              const double *dx64, const T *q, double *out)
{
    using AC = Acc<T>;
    using A = typename AC::A;
    __shared__ A wsum[32];
    const RowInfo row = rows[blockIdx.x];
    const T *qr = q + row.cell_off;
    const T *dxr = (sizeof(T) == 4) ? reinterpret_cast<const T *>(dx32 + row.mesh_off)
                                    : reinterpret_cast<const T *>(dx64 + row.mesh_off);
    const T dxu = (T)row.dx;
    A acc = AC::zero();
    for (int i = threadIdx.x; i < row.n; i += blockDim.x)
        acc = AC::add(acc, AC::mass(qr[i], row.uniform ? dxu : dxr[i]));
    for (int o = 16; o > 0; o >>= 1) acc = AC::add(acc, AC::shfl_down(acc, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        A x = lane < (int)(blockDim.x >> 5) ? wsum[lane] : AC::zero();
        for (int o = 16; o > 0; o >>= 1) x = AC::add(x, AC::shfl_down(x, o));
        if (lane == 0) out[blockIdx.x] = AC::to_double(x);
    }
}

}  // namespace

cudaError_t launch_general(const Plan &p, ram_dtype dt, const StepArgs &a, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    int launched = 0;  // general launches so far in this step
    if (dt == RAM_F32) {
        // rows with their own mesh: the warp-segment kernel, then the rows it does
        // not take on the general kernels
        if (p.nu_kernel == 1 && (e = launch_nseg(p, a, s)) != cudaSuccess) return e;
        if ((e = launch_general_t<float, 2>(p, a, s, launched)) != cudaSuccess) return e;
        if ((e = launch_general_t<float, 3>(p, a, s, launched)) != cudaSuccess) return e;
        return launch_general_t<float, 4>(p, a, s, launched);
    }
    if ((e = launch_general_t<double, 2>(p, a, s, launched)) != cudaSuccess) return e;
    if ((e = launch_general_t<double, 3>(p, a, s, launched)) != cudaSuccess) return e;
    return launch_general_t<double, 4>(p, a, s, launched);
}

cudaError_t launch_row_mass(const Plan &p, ram_dtype dt, const void *q, double *out,
                            cudaStream_t s)
{
    if (dt == RAM_F32)
        k_mass<float><<<p.n_rows, 256, 0, s>>>(p.rows, p.dx32, p.dx64,
                                                static_cast<const float *>(q), out);
    else
        k_mass<double><<<p.n_rows, 256, 0, s>>>(p.rows, p.dx32, p.dx64,
                                                 static_cast<const double *>(q), out);
    return cudaGetLastError();
}

}  // namespace ram
