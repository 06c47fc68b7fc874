// Launch-shape tuning of a plan: explicit settings and a timing autotuner.
#include <cuda_runtime.h>

#include "ram_internal.h"

using namespace ram;

namespace {

bool valid_rows_v(int v)
{
    for (int i = 0; i < kRowsVCount; ++i)
        if (kRowsVCandidates[i] == v) return true;
    return false;
}

struct DeviceSwitch {
    int prev = -1;
    bool ok = false;
    explicit DeviceSwitch(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceSwitch()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" ram_status ram_plan_get_tuning(ram_plan plan, ram_tuning *out)
{
    if (!plan || !out) return RAM_ERR_ARG;
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    out->rows_cells_per_thread_f32 = p->rows_v[0];
    out->rows_cells_per_thread_f64 = p->rows_v[1];
    out->tile_cells = p->tile_cells;
    out->threads = p->threads;
    out->uniform_kernel_f32 = p->uniform_kernel[0];
    out->uniform_kernel_f64 = p->uniform_kernel[1];
    out->rows_ctas_per_sm_f32 = p->rows_cps[0];
    out->rows_ctas_per_sm_f64 = p->rows_cps[1];
    out->stream_cells_per_lane_f32 = p->stream_v;
    out->seg_variant_f32 = p->seg_variant;
    out->seg_warps = p->seg_warps;
    out->nonuniform_kernel_f32 = p->nu_kernel;
    return RAM_OK;
}

extern "C" ram_status ram_plan_set_tuning(ram_plan plan, const ram_tuning *t)
{
    if (!plan || !t) return RAM_ERR_ARG;
    if (!valid_rows_v(t->rows_cells_per_thread_f32) || !valid_rows_v(t->rows_cells_per_thread_f64))
        return RAM_ERR_ARG;
    if (t->uniform_kernel_f32 < 0 || t->uniform_kernel_f32 > 2 ||
        (t->uniform_kernel_f64 != 0 && t->uniform_kernel_f64 != 1))
        return RAM_ERR_ARG;
    bool sv = false;
    for (int i = 0; i < kStreamVCount; ++i) sv |= t->stream_cells_per_lane_f32 == kStreamVCandidates[i];
    if (!sv) return RAM_ERR_ARG;
    if (t->seg_variant_f32 < 0 || t->seg_variant_f32 > 2) return RAM_ERR_ARG;
    if (t->seg_warps < 3 || t->seg_warps > 8) return RAM_ERR_ARG;
    if (t->nonuniform_kernel_f32 != 0 && t->nonuniform_kernel_f32 != 1) return RAM_ERR_ARG;
    if (t->rows_ctas_per_sm_f32 < 1 || t->rows_ctas_per_sm_f32 > 4 || t->rows_ctas_per_sm_f64 != 1)
        return RAM_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (t->tile_cells != p->tile_cells || t->threads != p->threads) {
        ram_status st = ram_plan_set_tiling(plan, t->tile_cells, t->threads);
        if (st != RAM_OK) return st;
    }
    p->rows_v[0] = t->rows_cells_per_thread_f32;
    p->rows_v[1] = t->rows_cells_per_thread_f64;
    p->uniform_kernel[0] = t->uniform_kernel_f32;
    p->uniform_kernel[1] = t->uniform_kernel_f64;
    p->rows_cps[0] = t->rows_ctas_per_sm_f32;
    p->rows_cps[1] = t->rows_ctas_per_sm_f64;
    p->stream_v = t->stream_cells_per_lane_f32;
    p->seg_variant = t->seg_variant_f32;
    p->seg_warps = t->seg_warps;
    p->nu_kernel = t->nonuniform_kernel_f32;
    return RAM_OK;
}

extern "C" ram_status ram_plan_autotune(ram_plan plan, ram_dtype dtype, const void *q_in,
                                        void *q_out, const double *v0, double dt,
                                        const void *dv_iface, ram_scheme scheme,
                                        const int32_t *nsub, int32_t reps, void *stream)
{
    if (!plan || reps < 1 || reps > 10000) return RAM_ERR_ARG;
    Plan *p = reinterpret_cast<Plan *>(plan);
    DeviceSwitch g(p->device);
    if (!g.ok) return RAM_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return RAM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return RAM_ERR_CUDA;
    }
    ram_status st = RAM_OK;
    auto time_once = [&](float *ms) -> ram_status {
        ram_status r = ram_step(plan, dtype, q_in, q_out, nullptr, v0, dt, dv_iface, scheme,
                                nsub, stream);
        if (r != RAM_OK) return r;
        cudaEventRecord(e0, s);
        for (int i = 0; i < reps && r == RAM_OK; ++i)
            r = ram_step(plan, dtype, q_in, q_out, nullptr, v0, dt, dv_iface, scheme, nsub,
                         stream);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return RAM_ERR_CUDA;
        cudaEventElapsedTime(ms, e0, e1);
        return r;
    };
    const int d = dtype == RAM_F64 ? 1 : 0;
    bool any_rows = false, any_tiles = false;
    for (int o = 2; o <= 4; ++o) {
        any_rows |= !p->rows_fit_h[d][o].empty();
        any_tiles |= !p->tiles_rest_h[d][o].empty() || !p->tiles_general_h[o].empty();
    }
    bool any_seg = false;
    for (int o = 2; o <= 4; ++o) any_seg |= !p->rows_seg_h[d][o].empty();
    if (any_rows || any_seg) {
        // candidates: (kernel, cells per thread)
        int best_k = p->uniform_kernel[d], best_v = p->rows_v[d], best_c = p->rows_cps[d];
        int best_sv = p->stream_v, best_gv = p->seg_variant, best_gw = p->seg_warps;
        float best = 3.4e38f;
        if (any_seg)
            for (int gv = 0; gv <= (d == 0 ? 2 : 0) && st == RAM_OK; ++gv)
                for (int gw : {3, 4, 6, 8}) {
                    if (st != RAM_OK) break;
                    p->uniform_kernel[d] = 1;
                    p->seg_variant = gv;
                    p->seg_warps = gw;
                    float ms = 0;
                    st = time_once(&ms);
                    if (st == RAM_OK && ms < best) {
                        best = ms;
                        best_k = 1;
                        best_gv = gv;
                        best_gw = gw;
                    }
                }
        if (any_seg && d == 0)
            for (int i = 0; i < kStreamVCount && st == RAM_OK; ++i) {
                p->uniform_kernel[0] = 2;
                p->stream_v = kStreamVCandidates[i];
                float ms = 0;
                st = time_once(&ms);
                if (st == RAM_OK && ms < best) {
                    best = ms;
                    best_k = 2;
                    best_sv = kStreamVCandidates[i];
                }
            }
        if (any_rows)
            for (int i = 0; i < kRowsVCount && st == RAM_OK; ++i) {
                const int v = kRowsVCandidates[i];
                const int cmax = d == 1 ? 1 : (v <= 5 ? 4 : (v <= 9 ? 3 : 2));
                for (int c = (d == 1 ? 1 : 2); c <= cmax && st == RAM_OK; ++c) {
                    p->uniform_kernel[d] = 0;
                    p->rows_v[d] = v;
                    p->rows_cps[d] = c;
                    float ms = 0;
                    st = time_once(&ms);
                    if (st == RAM_OK && ms < best) {
                        best = ms;
                        best_k = 0;
                        best_v = v;
                        best_c = c;
                    }
                }
            }
        p->uniform_kernel[d] = best_k;
        p->rows_v[d] = best_v;
        p->rows_cps[d] = best_c;
        p->stream_v = best_sv;
        p->seg_variant = best_gv;
        p->seg_warps = best_gw;
    }
    if (any_tiles && st == RAM_OK) {
        const int tcs[] = {256, 512, 1024, 2048};
        const int ths[] = {128, 256, 512};
        int best_tc = p->tile_cells, best_th = p->threads;
        float best = 3.4e38f;
        for (int tc : tcs)
            for (int th : ths) {
                if (st != RAM_OK) break;
                if (ram_plan_set_tiling(plan, tc, th) != RAM_OK) continue;
                float ms = 0;
                ram_status r = time_once(&ms);
                if (r == RAM_ERR_CUDA) {
                    st = r;
                    break;
                }
                if (r == RAM_OK && ms < best) {
                    best = ms;
                    best_tc = tc;
                    best_th = th;
                }
            }
        ram_status r = ram_plan_set_tiling(plan, best_tc, best_th);
        if (st == RAM_OK) st = r;
    }
    if (d == 0 && p->nseg_rows > 0 && st == RAM_OK) {
        // FP32 rows with their own mesh: the warp-segment kernel or the per-order ones
        int best_nu = p->nu_kernel;
        float best = 3.4e38f;
        for (int nu = 1; nu >= 0 && st == RAM_OK; --nu) {
            p->nu_kernel = nu;
            float ms = 0;
            st = time_once(&ms);
            if (st == RAM_OK && ms < best) {
                best = ms;
                best_nu = nu;
            }
        }
        p->nu_kernel = best_nu;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}
