// Planning: mesh validation, row classification, device copies of the mesh and
// the tile lists (Sec. 2 mesh; Sec. 3.2 and 3.2.1 edge index).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "ram_internal.h"

namespace ram {
namespace {

// Uniform rows: every width within 8 eps L of L/N (nodes computed in FP64 as
// x_0 + L j / N deviate from exact uniformity by a few eps L).
bool row_is_uniform(const double *x, int n)
{
    const double L = x[n] - x[0];
    const double h = L / n;
    const double tol = 8.0 * 2.220446049250313e-16 * std::fabs(L);
    for (int i = 0; i < n; ++i)
        if (std::fabs((x[i + 1] - x[i]) - h) > tol) return false;
    return true;
}

ram_status check_nodes(const double *x, int n)
{
    for (int j = 0; j <= n; ++j)
        if (!std::isfinite(x[j])) return RAM_ERR_MESH;
    for (int j = 0; j < n; ++j)
        if (!(x[j + 1] > x[j])) return RAM_ERR_MESH;
    return RAM_OK;
}

// Fixed-point node positions: fraction of the period in units of 2^-64.
// Position differences and the periodic wrap are then exact integer arithmetic.
bool fixed_point_nodes(const double *x, int n, uint64_t *out)
{
    const double L = x[n] - x[0];
    const double two64 = 18446744073709551616.0;
    uint64_t prev = 0;
    for (int j = 0; j < n; ++j) {
        double t = (x[j] - x[0]) / L;
        uint64_t v;
        if (j == 0)
            v = 0;
        else if (t >= 1.0)
            return false;
        else
            v = (uint64_t)(t * two64);
        if (j > 0 && v <= prev) return false;  // widths below 2^-64 L
        out[j] = v;
        prev = v;
    }
    return true;
}

template <typename T>
cudaError_t upload(T **dst, const T *src, size_t count)
{
    if (count == 0) {
        *dst = nullptr;
        return cudaSuccess;
    }
    cudaError_t e = cudaMalloc((void **)dst, count * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
}

void free_lists(Plan &p)
{
    cudaFree(p.tiles_nseg);
    p.tiles_nseg = nullptr;
    for (int o = 0; o < 5; ++o) {
        cudaFree(p.tiles_adj_nu[o]);
        p.tiles_adj_nu[o] = nullptr;
    }
    for (int o = 0; o < 5; ++o) {
        cudaFree(p.tiles_uniform[o]);
        cudaFree(p.tiles_general[o]);
        cudaFree(p.tiles_general32[o]);
        p.tiles_uniform[o] = p.tiles_general[o] = p.tiles_general32[o] = nullptr;
        for (int d = 0; d < 2; ++d) {
            cudaFree(p.rows_fit[d][o]);
            cudaFree(p.rows_fit_pos[d][o]);
            p.rows_fit_pos[d][o] = nullptr;
            cudaFree(p.tiles_rest[d][o]);
            cudaFree(p.rows_seg[d][o]);
            cudaFree(p.tiles_rest_seg[d][o]);
            p.rows_fit[d][o] = nullptr;
            p.tiles_rest[d][o] = nullptr;
            p.rows_seg[d][o] = nullptr;
            p.tiles_rest_seg[d][o] = nullptr;
        }
    }
}

void free_device(Plan &p)
{
    cudaFree(p.rows);
    free_lists(p);
    cudaFree(p.xfix);
    cudaFree(p.dx32);
    cudaFree(p.dx64);
    cudaFree(p.buckets);
    cudaFree(p.density);
    p.density = nullptr;
    cudaFree(p.err);
    cudaFree(p.row_par);
    p.row_par = nullptr;
    cudaFree(p.adj_scratch);
    p.adj_scratch = nullptr;
    cudaFree(p.a4_scratch);
    p.a4_scratch = nullptr;
    p.rows = nullptr;
    p.xfix = nullptr;
    p.dx32 = nullptr;
    p.dx64 = nullptr;
    p.buckets = nullptr;
    p.err = nullptr;
}

// Widths of a row twice over (cyclic sums without index wraps).
std::vector<double> doubled_widths(const double *x, int n)
{
    std::vector<double> w2(2 * (size_t)n);
    for (int i = 0; i < n; ++i) w2[i] = w2[i + n] = x[i + 1] - x[i];
    return w2;
}

// The longest physical extent of `span` consecutive cells (cyclic), and the most
// source cells an interval that long can touch, over every placement: for every
// start st, cells st..e-1 fit strictly inside it; it also touches cell e and the
// cell st-1 it may start in.
int most_cells_touched(const std::vector<double> &w2, int n, int span)
{
    double len_max = 0.0, acc = 0.0;
    for (int k = 0; k < span; ++k) acc += w2[k % (2 * n)];
    len_max = acc;
    for (int st = 1; st < n; ++st) {
        acc += w2[(st + span - 1) % (2 * n)] - w2[st - 1];
        len_max = std::max(len_max, acc);
    }
    int best = 0;
    acc = 0.0;
    int e = 0;
    for (int st = 0; st < n; ++st) {
        if (e < st) {
            e = st;
            acc = 0.0;
        }
        while (e < st + n && acc + w2[e] < len_max) acc += w2[e++];
        best = std::max(best, e - st + 2);
        if (e > st) acc -= w2[st];
    }
    return std::min(best, n + 1);
}

// Units (a power of two of fixed-point length, 2^qs) in which the FP32
// warp-segment kernel keeps window-relative positions as 32-bit values: every
// window of up to `wb` cells must span less than 2^31 units, and every cell at
// least 2^21 (so that in-cell offsets keep about 21 significant bits); -1 when
// the row's widths vary too much for both.
int position_shift(const std::vector<double> &w2, int n, int wb, double L)
{
    double acc = 0.0, len_max = 0.0, w_min = w2[0];
    for (int k = 0; k < wb; ++k) acc += w2[k % (2 * n)];
    len_max = acc;
    for (int st = 1; st < n; ++st) {
        acc += w2[(st + wb - 1) % (2 * n)] - w2[st - 1];
        len_max = std::max(len_max, acc);
    }
    for (int i = 0; i < n; ++i) w_min = std::min(w_min, w2[i]);
    const double two64 = 18446744073709551616.0;
    const double lfix = std::min(len_max / L, 1.0) * two64;
    int qs = std::max(0, (int)std::floor(std::log2(lfix)) - 30);
    if (std::ldexp(lfix, -qs) >= 2147483648.0) ++qs;
    if (std::ldexp(w_min / L * two64, -qs) < 2097152.0) return -1;
    return qs;
}

// The general kernels' per-order launch shapes of a tile list: whole-row tiles
// (window 0) first, and for each class the largest window and output extent.
void general_caps(const Plan &p, std::vector<Tile> &tl, int32_t &whole, int32_t wcap[2],
                  int32_t qcap[2])
{
    std::stable_partition(tl.begin(), tl.end(), [](const Tile &t) { return t.window == 0; });
    whole = 0;
    for (int c = 0; c < 2; ++c) wcap[c] = qcap[c] = 0;
    for (const Tile &t : tl) {
        const int c = t.window == 0 ? 0 : 1;
        if (c == 0) ++whole;
        const int w = c == 0 ? p.rows_h[t.row].n + 2 * kGenHR : t.window;
        wcap[c] = std::max(wcap[c], w);
        qcap[c] = std::max(qcap[c], t.count + 2 * kGenHalo);
    }
}

}  // namespace

// Split every row into near-equal tiles of at most tile_cells output cells and
// bound the source window of each non-uniform tile: the number of source cells
// that an interval as long as the tile (plus the residual halo) can touch,
// maximised over all placements, plus the reconstruction halo.
ram_status build_tiles(Plan &p)
{
    free_lists(p);
    p.tiles_nseg_h.clear();
    p.nseg_rows = 0;
    for (int o = 0; o < 5; ++o) p.tiles_adj_nu_h[o].clear();
    for (int o = 0; o < 5; ++o) {
        p.tiles_uniform_h[o].clear();
        p.tiles_general_h[o].clear();
        p.tiles_general32_h[o].clear();
        for (int d = 0; d < 2; ++d) {
            p.rows_fit_h[d][o].clear();
            p.rows_fit_pos_h[d][o].clear();
            p.tiles_rest_h[d][o].clear();
            p.ncap_fit[d][o] = 0;
            p.rows_seg_h[d][o].clear();
            p.tiles_rest_seg_h[d][o].clear();
            if (d == 0) {
                p.stream_nmax[o] = 0;
                p.stream_nmin[o] = 0;
            }
        }
    }
    p.window_max = 0;
    const int halo_res = kGenHalo;  // residual halo, cells per side
    const int tg = std::max(64, p.tile_cells / 2);  // output cells per non-uniform tile
    for (int r = 0; r < p.n_rows; ++r) {
        const RowInfo &ri = p.rows_h[r];
        const int n = ri.n;
        if (ri.uniform && p.adj_all)
            for (int a = 0; a < n; a += p.adj_nu_tcap)
                p.tiles_adj_nu_h[ri.order].push_back(Tile{r, a, std::min(p.adj_nu_tcap, n - a), 0});
        if (ri.uniform) {
            const int nt = (n + p.tile_cells - 1) / p.tile_cells;
            for (int t = 0; t < nt; ++t) {
                const int a = (int)((int64_t)n * t / nt);
                const int b = (int)((int64_t)n * (t + 1) / nt);
                const Tile tl{r, a, b - a, 0};
                p.tiles_uniform_h[ri.order].push_back(tl);
                // persistent whole-row kernel: TMA needs 16-byte aligned row starts and
                // lengths, and the row (plus halos) must fit the shared-memory stages
                for (int d = 0; d < 2; ++d) {
                    const int es = d == 0 ? 4 : 8;
                    const bool fit = n >= 32 && n <= rows_kernel_max_cells((ram_dtype)d) &&
                                     (n * es) % 16 == 0 && (ri.cell_off * es) % 16 == 0;
                    if (fit) {
                        if (t == 0) {
                            p.rows_fit_h[d][ri.order].push_back(r);
                            p.rows_fit_pos_h[d][ri.order].push_back(RowPos{ri.cell_off, r, n});
                            int cap = (n + 15) / 16 * 16;
                            if (cap > p.ncap_fit[d][ri.order]) p.ncap_fit[d][ri.order] = cap;
                        }
                    } else {
                        p.tiles_rest_h[d][ri.order].push_back(tl);
                    }
                    // warp-segment kernel: 16-byte aligned rows of at least 512 cells
                    const bool seg = n >= 512 && (n * es) % 16 == 0 &&
                                     (ri.cell_off * es) % 16 == 0;
                    if (seg) {
                        if (t == 0) {
                            p.rows_seg_h[d][ri.order].push_back(r);
                            if (d == 0) {
                                p.stream_nmax[ri.order] = std::max(p.stream_nmax[ri.order], n);
                                p.stream_nmin[ri.order] = p.stream_nmin[ri.order] == 0
                                                              ? n
                                                              : std::min(p.stream_nmin[ri.order], n);
                            }
                        }
                    } else {
                        p.tiles_rest_seg_h[d][ri.order].push_back(tl);
                    }
                }
            }
            continue;
        }
        const double *x = (p.flags & RAM_SHARED_MESH) ? p.nodes_h.data()
                                                       : p.nodes_h.data() + p.row_offset[r] + r;
        const std::vector<double> w2 = doubled_widths(x, n);
        // the adjoint's tiles: plain runs of at most adj_nu_tcap cells
        for (int a = 0; a < n; a += p.adj_nu_tcap)
            p.tiles_adj_nu_h[ri.order].push_back(Tile{r, a, std::min(p.adj_nu_tcap, n - a), 0});
        // FP32: the warp-segment kernel, with segments short enough that a segment
        // and its largest residual halo span less than a period, and a source
        // window that fits its shared-memory region
        bool nseg = false;
        p.rows_h[r].qshift = 0;
        if (n >= kNsegMinCells) {
            // the longest segment whose source window, residual halo included, fits
            // the warp's window; preferably one whose window without a residual
            // fits half of it (one pass of the reconstruction)
            const int cap = nseg_window_cap();
            const int seg_max = std::min(kNseg, n - 1 - 2 * kGenHalo);
            int seg = 0, wb = 0;
            for (int pass = 0; pass < 2 && seg == 0; ++pass) {
                for (int sg = seg_max; sg >= 1; sg -= (sg > 8 ? 8 : sg)) {
                    const int w1 = most_cells_touched(w2, n, sg + 2 * kGenHalo) + 2 * kNsegHR + 1;
                    const int w0 = most_cells_touched(w2, n, sg) + 2 * kNsegHR + 1;
                    if (w1 <= cap && (pass == 1 || w0 <= cap / 2)) {
                        seg = sg;
                        wb = w1;
                        break;
                    }
                    if (sg < kNseg / 3) break;
                }
            }
            int qs = -1;
            if (seg > 0) qs = position_shift(w2, n, wb, x[n] - x[0]);
            if (qs >= 0) {
                nseg = true;
                ++p.nseg_rows;
                p.rows_h[r].qshift = qs;
                const int per_tile = seg * kNsegWarps * kNsegPerWarp;
                for (int a = 0; a < n; a += per_tile)
                    p.tiles_nseg_h.push_back(Tile{r, a, std::min(per_tile, n - a), seg});
            }
        }
        std::vector<Tile> &g32 = p.tiles_general32_h[ri.order];
        // non-uniform row: one cyclic tile for short rows, else windowed tiles
        if (n <= 2 * tg + 4 * halo_res) {
            p.tiles_general_h[ri.order].push_back(Tile{r, 0, n, 0});
            if (!nseg) g32.push_back(Tile{r, 0, n, 0});
            continue;
        }
        const int nt = (n + tg - 1) / tg;
        // the longest physical extent of a tile's output cells with their halo,
        // [a - halo, b + halo) (cyclic), bounds the source cells of every tile
        double len_max = 0.0;
        for (int t = 0; t < nt; ++t) {
            const int a = (int)((int64_t)n * t / nt);
            const int b = (int)((int64_t)n * (t + 1) / nt);
            const int span = (b - a) + 2 * halo_res;
            const int first = ((a - halo_res) % n + n) % n;
            double len = 0.0;
            for (int k = 0; k < span; ++k) len += w2[(first + k) % (2 * n)];
            len_max = std::max(len_max, len);
        }
        // most source cells an interval of that length can touch (one pass over the
        // row): for every start s, cells s..e-1 fit strictly inside it; it also
        // touches cell e and the cell s-1 it may start in
        int best = 0;
        double acc = 0.0;
        int e = 0;
        for (int st = 0; st < n; ++st) {
            if (e < st) {
                e = st;
                acc = 0.0;
            }
            while (e < st + n && acc + w2[e] < len_max) acc += w2[e++];
            best = std::max(best, e - st + 2);
            if (e > st) acc -= w2[st];
        }
        best = std::min(best, n + 1);
        const int window = best + 2 * 2 + 2;  // reconstruction halo (2 per side) + slack
        p.window_max = std::max(p.window_max, window);
        for (int t = 0; t < nt; ++t) {
            const int a = (int)((int64_t)n * t / nt);
            const int b = (int)((int64_t)n * (t + 1) / nt);
            p.tiles_general_h[ri.order].push_back(Tile{r, a, b - a, window});
            if (!nseg) g32.push_back(Tile{r, a, b - a, window});
        }
    }
    // tiles of one reconstruction order next to each other: CTAs that run at the
    // same time mostly run the same code
    std::stable_sort(p.tiles_nseg_h.begin(), p.tiles_nseg_h.end(),
                     [&p](const Tile &a, const Tile &b) {
                         return p.rows_h[a.row].order < p.rows_h[b.row].order;
                     });
    if (upload(&p.tiles_nseg, p.tiles_nseg_h.data(), p.tiles_nseg_h.size()) != cudaSuccess)
        return RAM_ERR_NOMEM;
    for (int o = 2; o <= 4; ++o)
        if (upload(&p.tiles_adj_nu[o], p.tiles_adj_nu_h[o].data(), p.tiles_adj_nu_h[o].size()) !=
            cudaSuccess)
            return RAM_ERR_NOMEM;
    // the rows' position units (qshift) live in the device row table
    if (p.rows && cudaMemcpy(p.rows, p.rows_h.data(), sizeof(RowInfo) * p.rows_h.size(),
                             cudaMemcpyHostToDevice) != cudaSuccess)
        return RAM_ERR_CUDA;
    for (int o = 2; o <= 4; ++o) {
        // the general kernel runs whole-row tiles (window 0) and windowed tiles as
        // two launches, each with the shared memory its own largest tile needs
        general_caps(p, p.tiles_general_h[o], p.gen_whole[o], p.gen_wcap[o], p.gen_qcap[o]);
        general_caps(p, p.tiles_general32_h[o], p.gen32_whole[o], p.gen32_wcap[o],
                     p.gen32_qcap[o]);
        if (upload(&p.tiles_general32[o], p.tiles_general32_h[o].data(),
                   p.tiles_general32_h[o].size()) != cudaSuccess)
            return RAM_ERR_NOMEM;
        if (upload(&p.tiles_uniform[o], p.tiles_uniform_h[o].data(),
                   p.tiles_uniform_h[o].size()) != cudaSuccess)
            return RAM_ERR_NOMEM;
        if (upload(&p.tiles_general[o], p.tiles_general_h[o].data(),
                   p.tiles_general_h[o].size()) != cudaSuccess)
            return RAM_ERR_NOMEM;
        for (int d = 0; d < 2; ++d) {
            if (upload(&p.rows_fit[d][o], p.rows_fit_h[d][o].data(),
                       p.rows_fit_h[d][o].size()) != cudaSuccess)
                return RAM_ERR_NOMEM;
            if (upload(&p.rows_fit_pos[d][o], p.rows_fit_pos_h[d][o].data(),
                       p.rows_fit_pos_h[d][o].size()) != cudaSuccess)
                return RAM_ERR_NOMEM;
            if (upload(&p.tiles_rest[d][o], p.tiles_rest_h[d][o].data(),
                       p.tiles_rest_h[d][o].size()) != cudaSuccess)
                return RAM_ERR_NOMEM;
            if (upload(&p.rows_seg[d][o], p.rows_seg_h[d][o].data(),
                       p.rows_seg_h[d][o].size()) != cudaSuccess)
                return RAM_ERR_NOMEM;
            if (upload(&p.tiles_rest_seg[d][o], p.tiles_rest_seg_h[d][o].data(),
                       p.tiles_rest_seg_h[d][o].size()) != cudaSuccess)
                return RAM_ERR_NOMEM;
        }
    }
    return RAM_OK;
}

}  // namespace ram

using namespace ram;

extern "C" ram_status ram_plan_mesh(const ram_mesh_desc *desc, int device, ram_plan *out)
{
    if (!out) return RAM_ERR_ARG;
    *out = nullptr;
    if (!desc || desc->n_rows < 1 || !desc->row_offset || !desc->nodes) return RAM_ERR_ARG;
    const int32_t nr = desc->n_rows;
    const int64_t *ro = desc->row_offset;
    if (ro[0] != 0) return RAM_ERR_ARG;
    for (int r = 0; r < nr; ++r) {
        int64_t n = ro[r + 1] - ro[r];
        if (n < 1) return RAM_ERR_MESH;
        if (n > (int64_t)1 << 30) return RAM_ERR_UNSUPPORTED;
    }
    const bool shared = (desc->flags & RAM_SHARED_MESH) != 0;
    if (shared)
        for (int r = 1; r < nr; ++r)
            if (ro[r + 1] - ro[r] != ro[1] - ro[0]) return RAM_ERR_ARG;
    for (int r = 0; r < nr; ++r) {
        int o = desc->order ? desc->order[r] : desc->default_order;
        if (o < 2 || o > 4) return RAM_ERR_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return RAM_ERR_CUDA;
    int prev_dev = 0;
    cudaGetDevice(&prev_dev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaSetDevice(prev_dev);
        return RAM_ERR_CUDA;
    }

    Plan *p = new (std::nothrow) Plan();
    if (!p) {
        cudaSetDevice(prev_dev);
        return RAM_ERR_NOMEM;
    }
    p->device = device;
    p->n_rows = nr;
    p->n_cells = ro[nr];
    p->flags = desc->flags;
    p->limiter = (desc->flags & RAM_LIMITER_OFF) ? 0 : 1;
    // FP32 warp-segment rows default to the shared-memory ring form, 3 warps per
    // row CTA (the fastest measured on the disks; the autotuner may change it)
    p->seg_variant = 2;
    p->seg_warps = 3;
    p->row_offset.assign(ro, ro + nr + 1);
    p->adj_all = ((desc->flags & RAM_ADJOINT) && p->limiter) ? 1 : 0;
    const size_t n_nodes = shared ? (size_t)(ro[1] + 1) : (size_t)(ro[nr] + nr);
    p->nodes_h.assign(desc->nodes, desc->nodes + n_nodes);

    ram_status st = RAM_OK;
    // mesh checks and classification
    std::vector<uint64_t> xfix;
    std::vector<float> dx32;
    std::vector<double> dx64;
    std::vector<int32_t> buckets;
    // order 4 with the limiter on (the scaled quartic) runs on the general kernels:
    // the uniform-row kernels fold a row's partial integrals into constants
    bool limited4 = false;
    for (int r = 0; r < nr; ++r)
        limited4 |= p->limiter && (desc->order ? desc->order[r] : desc->default_order) == 4;
    p->rows_h.resize(nr);
    for (int r = 0; r < nr && st == RAM_OK; ++r) {
        const int n = (int)(ro[r + 1] - ro[r]);
        const double *x = shared ? p->nodes_h.data() : p->nodes_h.data() + ro[r] + r;
        RowInfo &ri = p->rows_h[r];
        ri.density = -1;
        ri.cell_off = ro[r];
        ri.n = n;
        ri.order = desc->order ? desc->order[r] : desc->default_order;
        ri.period = x[n] - x[0];
        ri.cells_per_length = (double)n / ri.period;
        ri.dx = ri.period / n;
        ri.inv_period = 1.0 / ri.period;
        if (shared && r > 0) {
            ri.uniform = p->rows_h[0].uniform;
            ri.mesh_off = p->rows_h[0].mesh_off;
            ri.bucket_off = p->rows_h[0].bucket_off;
            ri.bucket_bits = p->rows_h[0].bucket_bits;
            continue;
        }
        st = check_nodes(x, n);
        if (st != RAM_OK || !(ri.period > 0.0) || !std::isfinite(ri.period)) {
            st = RAM_ERR_MESH;
            break;
        }
        // a shared mesh serves every row, so one limited order-4 row sends them all
        ri.uniform = (row_is_uniform(x, n) && !(limited4 && (shared || ri.order == 4))) ? 1 : 0;
        if (ri.uniform && !p->adj_all) {
            ri.mesh_off = 0;
            ri.bucket_off = 0;
            ri.bucket_bits = 0;
            continue;
        }
        // non-uniform row (or any row of a limited adjoint plan): fixed-point nodes,
        // widths and the bucket table
        ri.mesh_off = (int64_t)xfix.size();
        size_t base = xfix.size();
        xfix.resize(base + n);
        dx32.resize(base + n);
        dx64.resize(base + n);
        if (!fixed_point_nodes(x, n, xfix.data() + base)) {
            st = RAM_ERR_MESH;
            break;
        }
        for (int i = 0; i < n; ++i) {
            dx64[base + i] = x[i + 1] - x[i];
            dx32[base + i] = (float)dx64[base + i];
        }
        int bits = 1;
        while ((1LL << bits) < 2LL * n && bits < 40) ++bits;
        ri.bucket_bits = bits;
        ri.bucket_off = (int64_t)buckets.size();
        const int64_t nb = 1LL << bits;
        buckets.resize(buckets.size() + nb);
        int32_t *bt = buckets.data() + ri.bucket_off;
        int cell = 0;
        for (int64_t b = 0; b < nb; ++b) {
            uint64_t start = (uint64_t)b << (64 - bits);
            while (cell + 1 < n && xfix[base + cell + 1] <= start) ++cell;
            bt[b] = cell;
        }
    }
    if (st == RAM_OK) {
        for (int r = 0; r < nr; ++r) p->n_uniform_rows += p->rows_h[r].uniform ? 1 : 0;
        // the A4 correction is the uniform-mesh formula, on the PPM remap
        if (desc->flags & RAM_A4) {
            p->a4 = 1;
            for (int r = 0; r < nr; ++r)
                if (!p->rows_h[r].uniform || p->rows_h[r].order != 3) st = RAM_ERR_UNSUPPORTED;
        }
    }
    if (st == RAM_OK) {
        if (upload(&p->rows, p->rows_h.data(), p->rows_h.size()) != cudaSuccess ||
            upload(&p->xfix, xfix.data(), xfix.size()) != cudaSuccess ||
            upload(&p->dx32, dx32.data(), dx32.size()) != cudaSuccess ||
            upload(&p->dx64, dx64.data(), dx64.size()) != cudaSuccess ||
            upload(&p->buckets, buckets.data(), buckets.size()) != cudaSuccess ||
            cudaMalloc((void **)&p->err, sizeof(int)) != cudaSuccess ||
            cudaMalloc(&p->row_par, sizeof(RowParams<double>) * (size_t)nr) != cudaSuccess ||
            ((desc->flags & RAM_ADJOINT) && (p->n_uniform_rows < nr || p->adj_all) &&
             cudaMalloc(&p->adj_scratch, 2 * sizeof(double) * (size_t)p->n_cells) != cudaSuccess) ||
            ((desc->flags & RAM_A4) &&
             cudaMalloc(&p->a4_scratch, 2 * sizeof(double) * (size_t)p->n_cells) != cudaSuccess) ||
            cudaMemset(p->err, 0, sizeof(int)) != cudaSuccess)
            st = RAM_ERR_NOMEM;
    }
    if (st == RAM_OK) st = build_tiles(*p);
    if (st == RAM_OK && cudaDeviceSynchronize() != cudaSuccess) st = RAM_ERR_CUDA;
    if (st != RAM_OK) {
        free_device(*p);
        delete p;
        cudaSetDevice(prev_dev);
        return st;
    }
    cudaSetDevice(prev_dev);
    *out = reinterpret_cast<ram_plan>(p);
    return RAM_OK;
}

extern "C" ram_status ram_plan_destroy(ram_plan plan)
{
    if (!plan) return RAM_OK;
    Plan *p = reinterpret_cast<Plan *>(plan);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    free_device(*p);
    cudaSetDevice(prev);
    delete p;
    return RAM_OK;
}

extern "C" ram_status ram_plan_query(ram_plan plan, ram_plan_info *info)
{
    if (!plan || !info) return RAM_ERR_ARG;
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    info->n_rows = p->n_rows;
    info->n_cells = p->n_cells;
    info->n_uniform_rows = p->n_uniform_rows;
    int nu = 0, ng = 0;
    for (int o = 2; o <= 4; ++o) {
        nu += (int)p->tiles_uniform_h[o].size();
        ng += (int)p->tiles_general_h[o].size();
    }
    info->n_tiles_uniform = nu;
    info->n_tiles_general = ng;
    info->tile_cells = p->tile_cells;
    info->threads = p->threads;
    info->device = p->device;
    info->n_nseg_rows = p->nseg_rows;
    int nd = 0;
    for (const RowInfo &ri : p->rows_h) nd += ri.density >= 0 ? 1 : 0;
    info->n_density_rows = nd;
    return RAM_OK;
}

extern "C" ram_status ram_plan_set_tiling(ram_plan plan, int32_t tile_cells, int32_t threads)
{
    if (!plan) return RAM_ERR_ARG;
    if (tile_cells < 64 || tile_cells > 8192 || threads < 64 || threads > 1024 ||
        threads % 32 != 0)
        return RAM_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(plan);
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(p->device) != cudaSuccess) return RAM_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaSetDevice(prev);
        return RAM_ERR_CUDA;
    }
    const int32_t old_tc = p->tile_cells, old_th = p->threads;
    p->tile_cells = tile_cells;
    p->threads = threads;
    ram_status st = build_tiles(*p);
    if (st != RAM_OK) {
        p->tile_cells = old_tc;
        p->threads = old_th;
        build_tiles(*p);
    }
    cudaSetDevice(prev);
    return st;
}

extern "C" ram_status ram_plan_set_wait_limit(ram_plan plan, uint32_t limit)
{
    if (!plan) return RAM_ERR_ARG;
    reinterpret_cast<Plan *>(plan)->wait_limit = limit;
    return RAM_OK;
}

extern "C" ram_status ram_plan_check_errors(ram_plan plan)
{
    if (!plan) return RAM_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(plan);
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(p->device) != cudaSuccess) return RAM_ERR_CUDA;
    int word = 0;
    ram_status st = RAM_OK;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&word, p->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(p->err, 0, sizeof(int)) != cudaSuccess) {
        st = RAM_ERR_CUDA;
    } else if (word & ERR_TIMEOUT) {
        st = RAM_ERR_TIMEOUT;
    } else if (word & ERR_NONFINITE) {
        st = RAM_ERR_NONFINITE;
    } else if (word & ERR_NSUB) {
        st = RAM_ERR_ARG;
    } else if (word & ERR_WINDOW) {
        st = RAM_ERR_UNSUPPORTED;
    } else if (word & ERR_CFL) {
        st = RAM_ERR_CFL;
    }
    cudaSetDevice(prev);
    return st;
}

extern "C" const char *ram_status_string(ram_status s)
{
    switch (s) {
    case RAM_OK: return "ok";
    case RAM_ERR_ARG: return "invalid argument";
    case RAM_ERR_MESH: return "invalid mesh";
    case RAM_ERR_CFL: return "residual CFL number above 1";
    case RAM_ERR_CUDA: return "CUDA runtime error";
    case RAM_ERR_TIMEOUT: return "device-side wait timed out";
    case RAM_ERR_NOMEM: return "out of memory";
    case RAM_ERR_UNSUPPORTED: return "unsupported request";
    case RAM_ERR_NONFINITE: return "non-finite shift";
    }
    return "unknown status";
}

extern "C" int32_t ram_version(void) { return 100; }

namespace {

// integral from 0 to x of the unnormalised periodic-bump density (signed)
double bump_primitive(const ram_density &d, double x)
{
    const double t = std::fabs(x), w = d.b - d.a;
    const double tt = std::min(std::max(t, d.a), d.b);
    const double pr = (1.0 + d.c) * std::min(t, d.a) + (tt - d.a) +
                      d.c * (0.5 * (tt - d.a) + w / (2.0 * M_PI) * std::sin(M_PI * (tt - d.a) / w)) +
                      std::max(t - d.b, 0.0);
    return x < 0.0 ? -pr : pr;
}

}  // namespace

extern "C" ram_status ram_plan_set_density(ram_plan plan, const ram_density *dens)
{
    if (!plan) return RAM_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(plan);
    const bool shared = (p->flags & RAM_SHARED_MESH) != 0;
    std::vector<Density> table;
    std::vector<int32_t> index(p->n_rows, -1);
    if (dens) {
        for (int r = 0; r < p->n_rows; ++r) {
            const RowInfo &ri = p->rows_h[r];
            if (ri.uniform) continue;
            const ram_density &d = dens[shared ? 0 : r];
            if (!(d.a > 0.0) || !(d.b > d.a) || !(d.c > -1.0) || !std::isfinite(d.c) ||
                !(d.x_max > d.x_min) || d.x_min > -d.b || d.x_max < d.b)
                return RAM_ERR_ARG;
            const int n = ri.n;
            const double *x = shared ? p->nodes_h.data() : p->nodes_h.data() + p->row_offset[r] + r;
            const double L = d.x_max - d.x_min;
            const double inv = 1.0 / (L + d.c * (d.a + d.b));
            const double pm = bump_primitive(d, d.x_min);
            if (std::fabs(x[0] - d.x_min) > 1e-12 * L || std::fabs(x[n] - d.x_max) > 1e-12 * L)
                return RAM_ERR_MESH;
            for (int j = 0; j <= n; ++j)
                if (std::fabs(n * (bump_primitive(d, x[j]) - pm) * inv - j) > 0.25)
                    return RAM_ERR_MESH;
            if (shared && r > 0) {
                index[r] = index[0];
                continue;
            }
            Density e;
            e.x_min = (float)d.x_min;
            e.L = (float)L;
            e.a = (float)d.a;
            e.b = (float)d.b;
            e.c = (float)d.c;
            e.inv_norm = (float)inv;
            e.prim_min = (float)pm;
            e.pad = 0.f;
            index[r] = (int32_t)table.size();
            table.push_back(e);
        }
    }
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(p->device) != cudaSuccess) return RAM_ERR_CUDA;
    ram_status st = RAM_OK;
    Density *dev = nullptr;
    if (cudaDeviceSynchronize() != cudaSuccess || upload(&dev, table.data(), table.size()) != cudaSuccess)
        st = RAM_ERR_NOMEM;
    if (st == RAM_OK) {
        std::vector<RowInfo> rows = p->rows_h;
        for (int r = 0; r < p->n_rows; ++r) rows[r].density = index[r];
        if (cudaMemcpy(p->rows, rows.data(), sizeof(RowInfo) * rows.size(),
                       cudaMemcpyHostToDevice) != cudaSuccess) {
            st = RAM_ERR_CUDA;
            cudaFree(dev);
        } else {
            p->rows_h = rows;
            cudaFree(p->density);
            p->density = dev;
        }
    } else {
        cudaFree(dev);
    }
    cudaSetDevice(prev);
    return st;
}
