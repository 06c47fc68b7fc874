// Transpose of one RAM step on rows with their own mesh (limiter off: the linear
// step; RAM_ADJOINT plans with the limiter on: every row, the PLM / PPM step
// linearised at its input), donor residual.
//
// The remap with the limiter off is linear: output mass M'_i (Eq. 18) is the sum
// over the source cells p that the shifted output cell overlaps of
// G_p(xi_hi) - G_p(xi_lo), the in-cell cumulative of p's reconstruction between
// the overlap's ends (xi in units of p's width), and G_p is linear in the values
// of p's stencil.  Its transpose is a gather by source cell: source cell p,
// shifted by +s, overlaps a few output cells (found like the forward edges, with
// the bucket table on x + s); with u_i = g'_i / dx_i (the transpose of Eq. 26)
// the cotangent of G_p's coefficients is
//   nu_{p,k} = sum_i u_i (xi_hi^k - xi_lo^k)      (k = 1, 2, 3: PLM / PPM)
// or, for order 4, the same sums over the quartics' Lagrange weights.  Then the
// reconstruction's transpose (PLM centred slope; PPM faces and delta<Q> of App. A
// without the limiter; the quartic's node masses) gathers them into g_in over the
// stencil.  A tile of source cells computes nu on itself plus a halo of three
// cells per side, then the two stencil passes in shared memory.
//
// The donor residual sub-steps (Eq. 6) with per-cell widths have the transpose
//   lf_j = g_j / dx_j - g_{j-1} / dx_{j-1},  g_up(j) += c_j lf_j,
//   dL/d dv_j += (dt / nsub) Q_up(j) lf_j
// over the sub-steps in reverse, with the forward states recomputed from the
// shifted field (kept in the plan's adjoint scratch); the upwind side at dv = 0
// is the left cell.
#include <cuda_runtime.h>

#include <cstdint>

#include "ram_device.cuh"

namespace ram {
namespace {

constexpr int kAH = 3;  // halo of the reconstruction transpose, cells per side

__device__ __forceinline__ float u64f(uint64_t v, float) { return __ull2float_rn(v); }
__device__ __forceinline__ double u64f(uint64_t v, double) { return __ull2double_rn(v); }

// Order 4: the mean of the two quartics' Lagrange weights at offset xi (units of
// the cell width h) on the node offsets z[0..5] (z[2] = 0, z[3] = 1), folded into
// the weights of the five masses m_{p-2..p+2}: G = sum_j w_j m_{p-2+j}.
template <typename T>
__device__ __forceinline__ void quartic_mass_weights(const T z[6], T xi, T w[5])
{
    T l[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int side = 0; side < 2; ++side) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            T v = T(1);
#pragma unroll
            for (int j = 0; j < 5; ++j)
                if (j != k) v *= Num<T>::div(xi - z[side + j], z[side + k] - z[side + j]);
            l[side + k] += T(0.5) * v;
        }
    }
    // node values (times h): {-(m0+m1), -m1, 0, m2, m2+m3, m2+m3+m4}
    w[0] = -l[0];
    w[1] = -l[0] - l[1];
    w[2] = l[3] + l[4] + l[5];
    w[3] = l[4] + l[5];
    w[4] = l[5];
}

// A value with its derivatives along the five stencil values Q_{p-2..p+2}.
template <typename T> struct D5 {
    T v, d[5];
};
template <typename T> __device__ __forceinline__ D5<T> d5(T v, int seed)
{
    D5<T> r;
    r.v = v;
#pragma unroll
    for (int k = 0; k < 5; ++k) r.d[k] = T(k == seed ? 1 : 0);
    return r;
}
template <typename T> __device__ __forceinline__ D5<T> d5add(const D5<T> &a, const D5<T> &b, T sb = T(1))
{
    D5<T> r;
    r.v = a.v + sb * b.v;
#pragma unroll
    for (int k = 0; k < 5; ++k) r.d[k] = a.d[k] + sb * b.d[k];
    return r;
}
template <typename T> __device__ __forceinline__ D5<T> d5scale(const D5<T> &a, T s)
{
    D5<T> r;
    r.v = a.v * s;
#pragma unroll
    for (int k = 0; k < 5; ++k) r.d[k] = a.d[k] * s;
    return r;
}
template <typename T> __device__ __forceinline__ D5<T> d5mul(const D5<T> &a, const D5<T> &b)
{
    D5<T> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < 5; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <typename T> __device__ __forceinline__ D5<T> d5div(const D5<T> &a, const D5<T> &b)
{
    D5<T> r;
    const T ib = Num<T>::div(T(1), b.v);
    r.v = a.v * ib;
#pragma unroll
    for (int k = 0; k < 5; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
    return r;
}

// The contribution w[k] of source cell p to g_in at cell p-2+k: the cotangents nu
// of its cumulative's power-basis coefficients (G = sum_k b_k xi^(k+1)) times the
// coefficients' derivatives along Q_{p-2..p+2}, for the limited PLM (Sec. 3.1) or
// PPM (App. A, App. A.2) linearised at the stencil values qs (every limiter branch
// taken as the values decide).  hs: the stencil widths.
template <typename T, int ORDER>
__device__ __forceinline__ void limited_block(const T qs[5], const T hs[5], const T nu[3], T w[5])
{
    D5<T> Q[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) Q[k] = d5<T>(qs[k], k);
    const T h = hs[2];
    D5<T> b[3];
    if (ORDER == 2) {
        const T hl = T(0.5) * (hs[1] + hs[2]), hr = T(0.5) * (hs[2] + hs[3]);
        const D5<T> dl = d5scale(d5add(Q[2], Q[1], T(-1)), Num<T>::div(T(1), hl));
        const D5<T> dr = d5scale(d5add(Q[3], Q[2], T(-1)), Num<T>::div(T(1), hr));
        D5<T> sig = d5<T>(T(0), -1);
        if (dl.v * dr.v > T(0)) sig = d5div(d5scale(d5mul(dl, dr), T(2)), d5add(dl, dr));
        b[0] = d5scale(d5add(Q[2], sig, T(-0.5) * h), h);  // h (Q - sigma h / 2)
        b[1] = d5scale(sig, T(0.5) * h * h);                // h^2 sigma / 2
        b[2] = d5<T>(T(0), -1);
    } else {
        D5<T> dq[3];  // delta<Q> of cells p-1, p, p+1 (stencil 1, 2, 3)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int k = c + 1;
            const T a = hs[k - 1], bb = hs[k], cc = hs[k + 1];
            const T f = Num<T>::div(bb, a + bb + cc);
            const D5<T> up = d5add(Q[k + 1], Q[k], T(-1)), dn = d5add(Q[k], Q[k - 1], T(-1));
            D5<T> d = d5add(d5scale(up, f * Num<T>::div(T(2) * a + bb, bb + cc)), dn,
                            f * Num<T>::div(bb + T(2) * cc, a + bb));
            if (up.v * dn.v > T(0)) {
                // sign(d) min(|d|, 2|dn|, 2|up|), the smallest taken by value
                const T sd = d.v >= T(0) ? T(1) : T(-1);
                D5<T> m = d5scale(d, sd);
                const D5<T> an = d5scale(dn, dn.v >= T(0) ? T(2) : T(-2));
                const D5<T> au = d5scale(up, up.v >= T(0) ? T(2) : T(-2));
                if (an.v < m.v) m = an;
                if (au.v < m.v) m = au;
                d = d5scale(m, sd);
            } else {
                d = d5<T>(T(0), -1);
            }
            dq[c] = d;
        }
        D5<T> face[2];  // faces p - 1/2 (k = 1) and p + 1/2 (k = 2)
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const int k = f + 1;
            const T hm = hs[k - 1], h0 = hs[k], h1 = hs[k + 1], h2 = hs[k + 2];
            const T w1 = Num<T>::div(T(2) * h1 * h0, h0 + h1) *
                         (Num<T>::div(hm + h0, T(2) * h0 + h1) - Num<T>::div(h2 + h1, T(2) * h1 + h0));
            const T w2 = -h0 * Num<T>::div(hm + h0, T(2) * h0 + h1);
            const T w3 = h1 * Num<T>::div(h1 + h2, h0 + T(2) * h1);
            const T is4 = Num<T>::div(T(1), hm + h0 + h1 + h2);
            const T cq = Num<T>::div(h0, h0 + h1) + w1 * is4;
            const D5<T> del = d5add(Q[k + 1], Q[k], T(-1));
            face[f] = d5add(d5add(d5add(Q[k], del, cq), dq[f + 1], w2 * is4), dq[f], w3 * is4);
        }
        D5<T> L = face[0], R = face[1];
        const D5<T> &Qc = Q[2];
        if ((R.v - Qc.v) * (Qc.v - L.v) <= T(0)) {
            L = Qc;
            R = Qc;
        } else {
            const T dd = R.v - L.v, qa = Qc.v - T(0.5) * (L.v + R.v);
            if (dd * qa > dd * dd * (T(1) / T(6)))
                L = d5add(d5scale(Qc, T(3)), R, T(-2));
            else if (-dd * dd * (T(1) / T(6)) > dd * qa)
                R = d5add(d5scale(Qc, T(3)), L, T(-2));
        }
        const D5<T> Q6 = d5add(d5scale(Qc, T(6)), d5add(L, R), T(-3));
        b[0] = d5scale(L, h);
        b[1] = d5scale(d5add(d5add(R, L, T(-1)), Q6), T(0.5) * h);
        b[2] = d5scale(Q6, -h * (T(1) / T(3)));
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) w[k] = nu[0] * b[0].d[k] + nu[1] * b[1].d[k] + nu[2] * b[2].d[k];
}

// Shared-memory layout of the remap transpose for a tile of tn source cells.
template <typename T> struct ALayout {
    static __host__ __device__ size_t bytes(int tn)
    {
        const int m = tn + 2 * kAH;
        return sizeof(T) * (size_t)(7 * m + 24);
    }
};

template <typename T, int ORDER, bool LIM>
__global__ void __launch_bounds__(256)
    k_adj_remap_nu(StepArgs a, const RowParams<T> *pars, const T *gprime, T *g_in, int tcap)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = tcap + 2 * kAH;
    // widths: W(j) = dx of cell a0 - kAH + j for j = -2 .. nm + 2
    T *sdx_raw = reinterpret_cast<T *>(smem_raw);
    T *sdx = sdx_raw + 2;
    T *sq = sdx_raw + m + 8;  // cotangents, per stage
    T *s1 = sq + m;
    T *s2 = s1 + m;
    T *s3 = s2 + m;
    T *s4 = s3 + m;
    T *sq0_raw = s4 + m;  // limited: the step input on the widths' cells
    T *sq0 = sq0_raw + 2;

    const Tile tile = a.tiles[blockIdx.x];
    const RowInfo row = a.rows[tile.row];
    const int N = row.n;
    const int tid = threadIdx.x, nth = blockDim.x;
    const uint64_t *X = a.xfix + row.mesh_off;
    const T *DX = (sizeof(T) == 4) ? reinterpret_cast<const T *>(a.dx32 + row.mesh_off)
                                   : reinterpret_cast<const T *>(a.dx64 + row.mesh_off);
    const int32_t *bt = a.buckets + row.bucket_off;
    const T *gp = gprime + row.cell_off;
    pdl_wait();
    const uint64_t S = pars[tile.row].sfix;
    const int a0 = tile.start, tn = tile.count;
    const int nm = tn + 2 * kAH;  // cells a0-3 .. a0+tn+3
    const T *q0 = static_cast<const T *>(a.q_in) + row.cell_off;
    for (int j = tid; j < nm + 5; j += nth) {
        const int c = wrap_index((int64_t)a0 - kAH - 2 + j, N);
        sdx_raw[j] = DX[c];
        if (LIM) sq0_raw[j] = q0[c];
    }
    __syncthreads();

    // ---- nu of every source cell of the tile and its halo ----
    for (int j = tid; j < nm; j += nth) {
        const int p = wrap_index((int64_t)a0 - kAH + j, N);
        const uint64_t y0 = X[p] + S;                       // shifted left node
        const uint64_t wp = (p + 1 < N ? X[p + 1] : 0ull) - X[p];  // width (fixed point)
        const T h = sdx[j];
        int i = locate_cell(X, N, bt, row.bucket_bits, a.density, row.density, y0);
        T lo = T(0);
        T nu[5] = {0, 0, 0, 0, 0};
        T z[6];
        if (ORDER == 4) {
            const T ih = Num<T>::div(T(1), h);
            z[2] = T(0);
            z[3] = T(1);
            z[1] = -sdx[j - 1] * ih;
            z[0] = z[1] - sdx[j - 2] * ih;
            z[4] = T(1) + sdx[j + 1] * ih;
            z[5] = z[4] + sdx[j + 2] * ih;
        }
        T wlo[5] = {0, 0, 0, 0, 0};
        // the shifted cell [y0, y0 + wp) overlaps output cells i, i+1, ...
        for (int guard = 0; guard <= N; ++guard) {
            const uint64_t rr = (i + 1 < N ? X[i + 1] : 0ull) - y0;  // output cell's right end
            const bool last = rr >= wp;
            const T hi = last ? T(1) : Num<T>::div(u64f(rr, T(0)), u64f(wp, T(0)));
            const T u = Num<T>::div(gp[i], DX[i]);
            if (ORDER == 4) {
                T whi[5];
                quartic_mass_weights<T>(z, hi, whi);
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    nu[k] += u * (whi[k] - wlo[k]);
                    wlo[k] = whi[k];
                }
            } else {
                T ph = hi, pl = lo;
#pragma unroll
                for (int k = 0; k < ORDER; ++k) {
                    nu[k] += u * (ph - pl);
                    ph *= hi;
                    pl *= lo;
                }
            }
            if (last) break;
            lo = hi;
            i = i + 1 < N ? i + 1 : 0;
        }
        if (LIM) {
            // the limited reconstruction linearised at the step input: this cell's
            // contributions to g_in at cells p-2 .. p+2
            T qs[5], hs[5], w[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                qs[k] = sq0[j - 2 + k];
                hs[k] = sdx[j - 2 + k];
            }
            const T nu3[3] = {nu[0], nu[1], nu[2]};
            limited_block<T, ORDER == 2 ? 2 : 3>(qs, hs, nu3, w);
            sq[j] = w[0];
            s1[j] = w[1];
            s2[j] = w[2];
            s3[j] = w[3];
            s4[j] = w[4];
        } else if (ORDER == 2) {
            // G = h [xi Q + sh (xi^2 - xi) / 2], sh = 2 (Q+ - Q-) h / (h- + 2h + h+)
            const T hm = sdx[j - 1], hp = sdx[j + 1];
            sq[j] = h * nu[0];                                          // d/dQ_p
            s1[j] = h * T(0.5) * (nu[1] - nu[0]) *                      // d/d sh ...
                    Num<T>::div(T(2) * h, hm + T(2) * h + hp);          // ... times d sh/d Q+
        } else if (ORDER == 3) {
            // G = h [L xi + (R - L + Q6) xi^2 / 2 - Q6 xi^3 / 3], Q6 = 6Q - 3(L + R)
            sq[j] = h * (T(3) * nu[1] - T(2) * nu[2]);  // d/dQ_p
            s1[j] = h * (nu[0] - T(2) * nu[1] + nu[2]);  // d/dL (face p - 1/2)
            s2[j] = h * (nu[2] - nu[1]);                  // d/dR (face p + 1/2)
        } else {
#pragma unroll
            for (int k = 0; k < 5; ++k) (k == 0 ? sq : k == 1 ? s1 : k == 2 ? s2 : k == 3 ? s3 : s4)[j] = nu[k];
        }
    }
    __syncthreads();

    // ---- the reconstruction's transpose over the stencil ----
    T *gi = g_in + row.cell_off;
    if (LIM) {
        // cell m gathers w[k] of cells p = m + 2 - k
        for (int t = tid; t < tn; t += nth) {
            const int j = t + kAH;
            gi[a0 + t] = sq[j + 2] + s1[j + 1] + s2[j] + s3[j - 1] + s4[j - 2];
        }
        return;
    }
    if (ORDER == 2) {
        // g_m = dQ_m + t_{m-1} - t_{m+1}, t = d/d sh * d sh/d Q+
        for (int t = tid; t < tn; t += nth) {
            const int j = t + kAH;
            gi[a0 + t] = sq[j] + s1[j - 1] - s1[j + 1];
        }
        return;
    }
    if (ORDER == 4) {
        // masses m = Q dx: g_m = dx_m sum_{p = m-2..m+2} w-cotangent of m in p
        for (int t = tid; t < tn; t += nth) {
            const int j = t + kAH;
            const T acc = s4[j - 2] + s3[j - 1] + s2[j] + s1[j + 1] + sq[j + 2];
            gi[a0 + t] = sdx[j] * acc;
        }
        return;
    }
    // PPM: the cotangent of face k + 1/2 is dR(k) + dL(k+1) (window indices 1 .. nm-2,
    // in s3); then the faces' dependence on Q and delta<Q>
    for (int j = 1 + tid; j < nm - 1; j += nth) s3[j] = s2[j] + s1[j + 1];
    __syncthreads();
    // face k = Q_k + c_q (Q_{k+1} - Q_k) + w2/S4 dQ_{k+1} + w3/S4 dQ_k (App. A)
    // cotangents of delta<Q>_k (s4), for k = 2 .. nm-3
    for (int j = 2 + tid; j < nm - 2; j += nth) {
        // delta<Q>_k enters face k (w3 weight) and face k-1 (w2 weight)
        T acc = T(0);
        {
            const T hm = sdx[j - 1], h0 = sdx[j], h1 = sdx[j + 1], h2 = sdx[j + 2];
            const T w3 = h1 * Num<T>::div(h1 + h2, h0 + T(2) * h1);
            acc += s3[j] * Num<T>::div(w3, hm + h0 + h1 + h2);
        }
        {
            const int k = j - 1;
            const T hm = sdx[k - 1], h0 = sdx[k], h1 = sdx[k + 1], h2 = sdx[k + 2];
            const T w2 = -h0 * Num<T>::div(hm + h0, T(2) * h0 + h1);
            acc += s3[k] * Num<T>::div(w2, hm + h0 + h1 + h2);
        }
        s4[j] = acc;
    }
    __syncthreads();
    for (int t = tid; t < tn; t += nth) {
        const int j = t + kAH;  // cell m
        T g = sq[j];
        // faces k = m (coefficient 1 - c) and k = m - 1 (coefficient c)
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const int k = j - f;
            const T hm = sdx[k - 1], h0 = sdx[k], h1 = sdx[k + 1], h2 = sdx[k + 2];
            const T w1 = Num<T>::div(T(2) * h1 * h0, h0 + h1) *
                         (Num<T>::div(hm + h0, T(2) * h0 + h1) - Num<T>::div(h2 + h1, T(2) * h1 + h0));
            const T c = Num<T>::div(h0, h0 + h1) + Num<T>::div(w1, hm + h0 + h1 + h2);
            g += s3[k] * (f == 0 ? T(1) - c : c);
        }
        // delta<Q>_k = alpha (Q_{k+1} - Q_k) + beta (Q_k - Q_{k-1}) for k = m-1, m, m+1
#pragma unroll
        for (int f = -1; f <= 1; ++f) {
            const int k = j + f;
            const T aa = sdx[k - 1], bb = sdx[k], cc = sdx[k + 1];
            const T alpha = Num<T>::div(bb, aa + bb + cc) * Num<T>::div(T(2) * aa + bb, bb + cc);
            const T beta = Num<T>::div(bb, aa + bb + cc) * Num<T>::div(bb + T(2) * cc, aa + bb);
            // d delta<Q>_k / dQ_m: m = k+1 -> alpha, m = k -> beta - alpha, m = k-1 -> -beta
            const T d = f == -1 ? alpha : (f == 0 ? beta - alpha : -beta);
            g += s4[k] * d;
        }
        gi[a0 + t] = g;
    }
}

// Donor residual transpose on a tile of cells [a0, a0+tn) with a halo of nsub
// cells per side: gprime on the tile, and dL/d dv added on the tile's interfaces.
template <typename T>
__global__ void __launch_bounds__(256)
    k_adj_resid_nu(StepArgs a, const RowParams<T> *pars, const T *qs, const T *g_out, T *gprime,
                   T *g_dv, int tcap)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wc = tcap + 2 * RAM_MAX_NSUB + 2;
    T *sdx = reinterpret_cast<T *>(smem_raw);  // wc
    T *sc = sdx + wc;                           // wc + 1: dv h (signed swept length)
    T *g0 = sc + wc + 1;                        // wc
    T *g1 = g0 + wc;                            // wc
    T *lf = g1 + wc;                            // wc + 1
    T *st = lf + wc + 1;                        // (RAM_MAX_NSUB + 1) x wc forward states

    const Tile tile = a.tiles[blockIdx.x];
    const RowInfo row = a.rows[tile.row];
    const int N = row.n;
    const int tid = threadIdx.x, nth = blockDim.x;
    const T *DX = (sizeof(T) == 4) ? reinterpret_cast<const T *>(a.dx32 + row.mesh_off)
                                   : reinterpret_cast<const T *>(a.dx64 + row.mesh_off);
    pdl_wait();
    const RowParams<T> P = pars[tile.row];
    const int ns = P.nsub;
    const T h = (T)(a.dt / (double)(ns > 0 ? ns : 1));  // sub-step length dt / nsub
    const int a0 = tile.start, tn = tile.count;
    const int c0 = a0 - ns;  // first cell of the halo
    const int nc = tn + 2 * ns;
    const T *dv = static_cast<const T *>(a.dv) + row.cell_off;
    const T *q = qs + row.cell_off;
    const T *g = g_out + row.cell_off;
    for (int i = tid; i < nc; i += nth) {
        const int c = wrap_index((int64_t)c0 + i, N);
        sdx[i] = DX[c];
        st[i] = q[c];
        g0[i] = g[c];
    }
    for (int i = tid; i <= nc; i += nth) sc[i] = dv[wrap_index((int64_t)c0 + i, N)] * h;
    __syncthreads();
    // forward sub-steps: state k+1 on [k+1, nc-k-1) from state k
    for (int k = 0; k + 1 < ns; ++k) {
        const T *qk = st + (size_t)k * wc;
        T *qn = st + (size_t)(k + 1) * wc;
        for (int i = k + 1 + tid; i < nc - k - 1; i += nth) {
            const T cL = sc[i], cR = sc[i + 1];
            const T FL = cL * (cL > T(0) ? qk[i - 1] : qk[i]);
            const T FR = cR * (cR > T(0) ? qk[i] : qk[i + 1]);
            qn[i] = qk[i] - Num<T>::div(FR - FL, sdx[i]);
        }
        __syncthreads();
    }
    T *cur = g0, *nxt = g1;
    T *gd = g_dv ? g_dv + row.cell_off : nullptr;
    for (int k = ns - 1; k >= 0; --k) {
        const T *qk = st + (size_t)k * wc;
        const int lo = ns - k, hi = nc - (ns - k);  // g^(k) valid on [lo, hi)
        // lf_j for interfaces j in [lo, hi]: g_j / dx_j - g_{j-1} / dx_{j-1}
        for (int j = lo + tid; j <= hi; j += nth)
            lf[j] = Num<T>::div(cur[j], sdx[j]) - Num<T>::div(cur[j - 1], sdx[j - 1]);
        __syncthreads();
        if (gd)
            for (int j = ns + tid; j < ns + tn; j += nth) {
                const T c = sc[j];
                const T qup = c >= T(0) ? qk[j - 1] : qk[j];
                gd[wrap_index((int64_t)c0 + j, N)] += lf[j] * h * qup;
            }
        for (int i = lo + tid; i < hi; i += nth) {
            T v = cur[i];
            const T cL = sc[i], cR = sc[i + 1];
            if (cR >= T(0)) v += cR * lf[i + 1];  // F_{i+1} takes Q_i when c >= 0
            if (cL < T(0)) v += cL * lf[i];       // F_i takes Q_i when c < 0
            nxt[i] = v;
        }
        __syncthreads();
        T *t = cur;
        cur = nxt;
        nxt = t;
    }
    T *gpo = gprime + row.cell_off;
    for (int i = tid; i < tn; i += nth) gpo[a0 + i] = cur[ns + i];
}

template <typename T, int ORDER, bool LIM>
cudaError_t launch_adj_remap_nu(const Plan &p, const StepArgs &a, const void *gp, void *g_in,
                                cudaStream_t s)
{
    const int n = (int)p.tiles_adj_nu_h[ORDER].size();
    if (n == 0) return cudaSuccess;
    const int tcap = p.adj_nu_tcap;
    const size_t smem = ALayout<T>::bytes(tcap);
    cudaError_t e = cudaFuncSetAttribute(k_adj_remap_nu<T, ORDER, LIM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    StepArgs b = a;
    b.tiles = p.tiles_adj_nu[ORDER];
    b.n_tiles = n;
    return launch_pdl(k_adj_remap_nu<T, ORDER, LIM>, n, 256, smem, s, b,
                      static_cast<const RowParams<T> *>(p.row_par), static_cast<const T *>(gp),
                      static_cast<T *>(g_in), tcap);
}

template <typename T>
cudaError_t launch_adj_nu_t(const Plan &p, const StepArgs &a, const void *g_out, void *g_in,
                            void *g_dv, cudaStream_t s)
{
    const void *gp = g_out;
    const bool resid = a.dv != nullptr;
    if (resid) {
        // the shifted field (the residual step's input) into the scratch
        T *qs = static_cast<T *>(p.adj_scratch);
        T *gprime = qs + p.n_cells;
        // the step's shift alone (MODE_STEP without dv) of the input, by the
        // general kernels (they read the shift from the parameter kernel's output)
        StepArgs f = a;
        f.q_out = qs;
        f.dv = nullptr;
        const ram_dtype dt = sizeof(T) == 4 ? RAM_F32 : RAM_F64;
        cudaError_t e = cudaSuccess;
        if (p.adj_all) {
            // every row: the shift's own parameters (no residual), the uniform and
            // the general kernels, then the step's parameters back for the transposes
            e = launch_params(p, dt, f, s);
            if (e == cudaSuccess) e = launch_uniform(p, dt, f, s);
            if (e == cudaSuccess) e = launch_general(p, dt, f, s);
            if (e == cudaSuccess) e = launch_params(p, dt, a, s);
        } else {
            e = launch_general(p, dt, f, s);
        }
        if (e != cudaSuccess) return e;
        const int tcap = p.adj_nu_tcap;
        const int wc = tcap + 2 * RAM_MAX_NSUB + 2;
        const size_t smem = sizeof(T) * ((size_t)5 * wc + 2 + (size_t)(RAM_MAX_NSUB + 1) * wc);
        if (smem > 227 * 1024) return cudaErrorNotSupported;
        e = cudaFuncSetAttribute(k_adj_resid_nu<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        bool first = true;
        for (int o = 2; o <= 4; ++o) {
            const int nt = (int)p.tiles_adj_nu_h[o].size();
            if (nt == 0) continue;
            StepArgs b = a;
            b.tiles = p.tiles_adj_nu[o];
            b.n_tiles = nt;
            const RowParams<T> *pars = static_cast<const RowParams<T> *>(p.row_par);
            if (first) {
                // the shift launches above do not wait for each other: the first
                // reader of the scratch takes the stream's full ordering
                k_adj_resid_nu<T><<<nt, 256, smem, s>>>(b, pars, qs, static_cast<const T *>(g_out),
                                                         gprime, static_cast<T *>(g_dv), tcap);
                e = cudaGetLastError();
                first = false;
            } else {
                e = launch_pdl(k_adj_resid_nu<T>, nt, 256, smem, s, b, pars,
                               static_cast<const T *>(qs), static_cast<const T *>(g_out), gprime,
                               static_cast<T *>(g_dv), tcap);
            }
            if (e != cudaSuccess) return e;
        }
        gp = gprime;
    } else if (p.adj_all) {
        cudaError_t e = launch_params(p, sizeof(T) == 4 ? RAM_F32 : RAM_F64, a, s);
        if (e != cudaSuccess) return e;
    }
    if (p.adj_all) {
        // limited PLM / PPM linearised at the step input
        cudaError_t e = launch_adj_remap_nu<T, 2, true>(p, a, gp, g_in, s);
        if (e == cudaSuccess) e = launch_adj_remap_nu<T, 3, true>(p, a, gp, g_in, s);
        return e;
    }
    cudaError_t e = launch_adj_remap_nu<T, 2, false>(p, a, gp, g_in, s);
    if (e == cudaSuccess) e = launch_adj_remap_nu<T, 3, false>(p, a, gp, g_in, s);
    if (e == cudaSuccess) e = launch_adj_remap_nu<T, 4, false>(p, a, gp, g_in, s);
    return e;
}

}  // namespace

cudaError_t launch_adjoint_nu(const Plan &p, ram_dtype dt, const StepArgs &a, const void *g_out,
                              void *g_in, void *g_dv, cudaStream_t s)
{
    if (dt == RAM_F32) return launch_adj_nu_t<float>(p, a, g_out, g_in, g_dv, s);
    return launch_adj_nu_t<double>(p, a, g_out, g_in, g_dv, s);
}

}  // namespace ram
