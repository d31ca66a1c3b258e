// plan.cu -- batched plans (one CUDA graph for encode + search of a fixed
// set of query batches) and the schedule autotuner.  Host code only: every
// computation is one of libhd's kernels.
#include <algorithm>
#include <chrono>
#include <functional>
#include <string>
#include <vector>

#include "hd_internal.cuh"

struct hd_plan {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t kernel_nodes = 0;
    int device = 0;
};

namespace {

struct scoped_stream {
    cudaStream_t s = nullptr;
    ~scoped_stream()
    {
        if (s) cudaStreamDestroy(s);
    }
};

void plan_release(hd_plan *p)
{
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    delete p;
}

// One eager run of `body` on a private stream (kernel attributes and lazy
// module loading happen outside capture), then its capture into a graph.
hd_status plan_capture(int dev, const std::function<hd_status(cudaStream_t)> &body, hd_plan **out)
{
    scoped_stream ss;
    HD_CUDA_TRY(cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking));
    hd_status st = body(ss.s);
    if (st != HD_OK) return st;
    HD_CUDA_TRY(cudaStreamSynchronize(ss.s));

    hd_plan *p = new hd_plan;
    p->device = dev;
    cudaError_t e = cudaStreamBeginCapture(ss.s, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        plan_release(p);
        return hd_cuda_fail(e, "hd_plan_create: begin capture");
    }
    st = body(ss.s);
    e = cudaStreamEndCapture(ss.s, &p->graph);
    if (st != HD_OK || e != cudaSuccess) {
        plan_release(p);
        return st != HD_OK ? st : hd_cuda_fail(e, "hd_plan_create: end capture");
    }
    e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) {
        plan_release(p);
        return hd_cuda_fail(e, "hd_plan_create: instantiate");
    }
    size_t n = 0;
    cudaGraphGetNodes(p->graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (n) cudaGraphGetNodes(p->graph, nodes.data(), &n);
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++p->kernel_nodes;
    }
    *out = p;
    return HD_OK;
}

// Autotuner: argument checks shared by the binary and the dot-product tuner.
hd_status tune_checks(const hd_library *lib, const void *d_q, const double *d_q_mz, const uint8_t *d_q_charge,
                      const uint8_t *d_q_class, uint32_t n_q, const hd_window *windows, uint32_t n_windows,
                      uint32_t k, hd_qwin *win, const std::string &name)
{
    if (k < 1 || k > 16) return hd_fail(HD_ERR_INVALID_ARG, name + ": k must be in [1, 16]");
    if (n_q == 0 || !d_q || !d_q_mz || !d_q_charge) return hd_fail(HD_ERR_INVALID_ARG, name + ": empty or null query set");
    hd_status st = hd_make_qwin(d_q_class, windows, n_windows, win);
    if (st != HD_OK) return st;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != lib->device)
        return hd_fail(HD_ERR_INVALID_ARG, name + ": library belongs to another device");
    return HD_OK;
}

// Candidates: popc (binary rows only), then for every prepared tensor-core
// form (tile_group, super_group) in {4, 8, 16, 32} x {2, 4, 16} on one SM and on SM
// pairs (kind::mxf4 on pairs only, and only when D is a multiple of 256, with
// one or two reference tiles per query stage).
std::vector<hd_tune_result> tc_candidates(const hd_library *lib, bool with_popc)
{
    std::vector<hd_tune_result> cand;
    if (with_popc) cand.push_back({HD_FORM_POPC, 0, 0, 0, 0, 0, 0.0});
    const uint32_t tgs[4] = {4, 8, 16, 32}, sgs[3] = {2, 4, 16};
    const uint32_t shapes[2][2] = {{1, 1}, {2, 2}};   // (cluster, cta_group): one SM, or the SM pair
    for (hd_search_form f : {HD_FORM_TC_MXF4, HD_FORM_TC_FP4, HD_FORM_TC_FP8, HD_FORM_TC_BF16}) {
        if (!hd_tc_copy(lib, f) || (f == HD_FORM_TC_MXF4 && lib->dim % 256 != 0)) continue;
        for (uint32_t tg : tgs)
            for (uint32_t sg : sgs)
                for (const auto &sh : shapes) {
                    if (f != HD_FORM_TC_MXF4) cand.push_back({f, tg, sg, sh[0], sh[1], 1, 0.0});
                    else if (sh[1] == 2)
                        for (uint32_t tps : {1u, 2u}) cand.push_back({f, tg, sg, sh[0], sh[1], tps, 0.0});
                }
    }
    return cand;
}

// Times every candidate (best of two runs after a warm-up, CUDA events on a
// private stream) through `run` and keeps the fastest as the library's
// HD_FORM_AUTO form and schedule.
hd_status tune(hd_library *lib, std::vector<hd_tune_result> cand, uint32_t n_q, uint32_t k, hd_tune_result *best,
               hd_tune_result *all, uint32_t cap, uint32_t *n_all,
               const std::function<hd_status(hd_search_form, uint32_t *, void *, cudaStream_t)> &run)
{
    scoped_stream ss;
    HD_CUDA_TRY(cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking));
    uint32_t *oi = nullptr;
    void *osc = nullptr;
    if (cudaMalloc(&oi, (size_t)n_q * k * 4) != cudaSuccess || cudaMalloc(&osc, (size_t)n_q * k * 4) != cudaSuccess) {
        cudaFree(oi);
        cudaGetLastError();
        return hd_fail(HD_ERR_OOM, "autotune: output allocation failed");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const hd_mma_tuning saved = lib->mma_tuning;
    hd_status st = HD_OK;
    for (auto &c : cand) {
        lib->mma_tuning.tile_group = c.tile_group;
        lib->mma_tuning.super_group = c.super_group;
        lib->mma_tuning.cluster = c.cluster;
        lib->mma_tuning.cta_group = c.cta_group;
        lib->mma_tuning.tiles_per_stage = c.tiles_per_stage;
        double bestms = 1e30;
        for (int rep = 0; rep < 3 && st == HD_OK; ++rep) {   // first run warms up
            cudaEventRecord(e0, ss.s);
            st = run(c.form, oi, osc, ss.s);
            cudaEventRecord(e1, ss.s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = hd_fail(HD_ERR_CUDA, "autotune: run failed");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) bestms = std::min(bestms, (double)ms);
        }
        c.ms = bestms;
        if (st != HD_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(oi);
    cudaFree(osc);
    if (st != HD_OK) {
        lib->mma_tuning = saved;
        return st;
    }
    const auto it = std::min_element(cand.begin(), cand.end(),
                                     [](const hd_tune_result &a, const hd_tune_result &b) { return a.ms < b.ms; });
    lib->mma_tuning.tile_group = it->tile_group;
    lib->mma_tuning.super_group = it->super_group;
    lib->mma_tuning.cluster = it->cluster;
    lib->mma_tuning.cta_group = it->cta_group;
    lib->mma_tuning.tiles_per_stage = it->tiles_per_stage;
    lib->auto_form = it->form;
    if (best) *best = *it;
    if (n_all) *n_all = (uint32_t)cand.size();
    if (all)
        for (uint32_t i = 0; i < cand.size() && i < cap; ++i) all[i] = cand[i];
    return HD_OK;
}

}  // namespace

extern "C" {

hd_status hd_plan_create(hd_ctx *ctx, const hd_library *lib, const uint32_t *d_offsets, const uint32_t *d_bins,
                         const uint8_t *d_levels, const double *d_q_mz, const uint8_t *d_q_charge,
                         const uint8_t *d_q_class, uint32_t n_q, const hd_window *windows, uint32_t n_windows,
                         uint32_t k, hd_search_form form, uint64_t *d_q_hv_work, uint32_t *d_out_idx,
                         uint16_t *d_out_dist, hd_plan **out)
{
    if (!out) return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create: null output");
    *out = nullptr;
    if (!ctx || !lib) return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create: null ctx or library");
    if (!hd_lib_binary(lib)) return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create: multi-bit library (use hd_plan_create_dot)");
    if (ctx->p.dim != lib->dim) return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create: ctx and library dims differ");
    if (k < 1 || k > 16) return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create: k must be in [1, 16]");
    if (n_q == 0) return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create: empty query set");
    if (!d_offsets || !d_bins || !d_levels || !d_q_mz || !d_q_charge || !d_q_hv_work || !d_out_idx || !d_out_dist)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create: null buffer");
    if (reinterpret_cast<uintptr_t>(d_q_hv_work) & 15u)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create: d_q_hv_work must be 16-byte aligned");
    hd_qwin win;
    hd_status st = hd_make_qwin(d_q_class, windows, n_windows, &win);
    if (st != HD_OK) return st;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != lib->device || dev != ctx->device)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create: objects belong to another device");
    return plan_capture(dev, [&](cudaStream_t s) -> hd_status {
        hd_encode_launch(ctx, d_offsets, d_bins, d_levels, n_q, d_q_hv_work, s);
        HD_CUDA_TRY(cudaGetLastError());
        return hd_search_dispatch(lib, d_q_hv_work, d_q_mz, d_q_charge, n_q, win, k, form, d_out_idx, d_out_dist, s);
    }, out);
}

hd_status hd_plan_create_dot(hd_ctx *ctx, const hd_library *lib, const uint32_t *d_offsets, const uint32_t *d_bins,
                             const uint8_t *d_levels, const double *d_q_mz, const uint8_t *d_q_charge,
                             const uint8_t *d_q_class, uint32_t n_q, const hd_window *windows, uint32_t n_windows,
                             uint32_t k, hd_search_form form, int8_t *d_q_comp_work, uint32_t *d_out_idx,
                             int32_t *d_out_score, hd_plan **out)
{
    if (!out) return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create_dot: null output");
    *out = nullptr;
    if (!ctx || !lib) return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create_dot: null ctx or library");
    if (hd_lib_binary(lib)) return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create_dot: binary library (use hd_plan_create)");
    if (ctx->p.dim != lib->dim) return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create_dot: ctx and library dims differ");
    if (k < 1 || k > 16) return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create_dot: k must be in [1, 16]");
    if (n_q == 0) return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create_dot: empty query set");
    if (!d_offsets || !d_bins || !d_levels || !d_q_mz || !d_q_charge || !d_q_comp_work || !d_out_idx || !d_out_score)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create_dot: null buffer");
    if (reinterpret_cast<uintptr_t>(d_q_comp_work) & 15u)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create_dot: d_q_comp_work must be 16-byte aligned");
    hd_status st0 = hd_dot_check(lib, &form, "hd_plan_create_dot");
    if (st0 != HD_OK) return st0;
    hd_qwin win;
    hd_status st = hd_make_qwin(d_q_class, windows, n_windows, &win);
    if (st != HD_OK) return st;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != lib->device || dev != ctx->device)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_create_dot: objects belong to another device");
    const uint32_t bits = lib->bits;
    return plan_capture(dev, [&](cudaStream_t s) -> hd_status {
        hd_encode_mb_launch(ctx, d_offsets, d_bins, d_levels, n_q, bits, d_q_comp_work, s);
        HD_CUDA_TRY(cudaGetLastError());
        return hd_search_dot_dispatch(lib, form, d_q_comp_work, d_q_mz, d_q_charge, n_q, win, k, d_out_idx,
                                      d_out_score, s);
    }, out);
}

hd_status hd_plan_launch(hd_plan *plan, hd_stream stream)
{
    if (!plan) return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_launch: null plan");
    HD_CUDA_TRY(cudaGraphLaunch(plan->exec, (cudaStream_t)stream));
    hd_count_launches(plan->kernel_nodes);
    return HD_OK;
}

hd_status hd_plan_info(const hd_plan *plan, uint32_t *kernel_nodes)
{
    if (!plan) return hd_fail(HD_ERR_INVALID_ARG, "hd_plan_info: null plan");
    if (kernel_nodes) *kernel_nodes = plan->kernel_nodes;
    return HD_OK;
}

void hd_plan_destroy(hd_plan *plan) { plan_release(plan); }

hd_status hd_library_autotune(hd_library *lib, const uint64_t *d_q_hv, const double *d_q_mz,
                              const uint8_t *d_q_charge, const uint8_t *d_q_class, uint32_t n_q,
                              const hd_window *windows, uint32_t n_windows, uint32_t k, hd_tune_result *best,
                              hd_tune_result *all, uint32_t cap, uint32_t *n_all)
{
    if (!lib) return hd_fail(HD_ERR_INVALID_ARG, "hd_library_autotune: null library");
    if (!hd_lib_binary(lib)) return hd_fail(HD_ERR_INVALID_ARG, "hd_library_autotune: multi-bit library (use hd_library_autotune_dot)");
    if (reinterpret_cast<uintptr_t>(d_q_hv) & 15u)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_library_autotune: d_q_hv must be 16-byte aligned");
    hd_qwin win;
    hd_status st = tune_checks(lib, d_q_hv, d_q_mz, d_q_charge, d_q_class, n_q, windows, n_windows, k, &win,
                               "hd_library_autotune");
    if (st != HD_OK) return st;
    return tune(lib, tc_candidates(lib, true), n_q, k, best, all, cap, n_all,
                [&](hd_search_form f, uint32_t *oi, void *osc, cudaStream_t s) {
                    return hd_search_dispatch(lib, d_q_hv, d_q_mz, d_q_charge, n_q, win, k, f, oi,
                                              static_cast<uint16_t *>(osc), s);
                });
}

hd_status hd_library_autotune_dot(hd_library *lib, const int8_t *d_q_comp, const double *d_q_mz,
                                  const uint8_t *d_q_charge, const uint8_t *d_q_class, uint32_t n_q,
                                  const hd_window *windows, uint32_t n_windows, uint32_t k, hd_tune_result *best,
                                  hd_tune_result *all, uint32_t cap, uint32_t *n_all)
{
    if (!lib) return hd_fail(HD_ERR_INVALID_ARG, "hd_library_autotune_dot: null library");
    if (hd_lib_binary(lib)) return hd_fail(HD_ERR_INVALID_ARG, "hd_library_autotune_dot: binary library (use hd_library_autotune)");
    if (reinterpret_cast<uintptr_t>(d_q_comp) & 15u)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_library_autotune_dot: d_q_comp must be 16-byte aligned");
    hd_qwin win;
    hd_status st = tune_checks(lib, d_q_comp, d_q_mz, d_q_charge, d_q_class, n_q, windows, n_windows, k, &win,
                               "hd_library_autotune_dot");
    if (st != HD_OK) return st;
    std::vector<hd_tune_result> cand = tc_candidates(lib, lib->x_planes != nullptr);   // popc on prepared bit planes
    if (cand.empty()) return hd_fail(HD_ERR_INVALID_ARG, "hd_library_autotune_dot: no tensor-core copy or bit planes prepared");
    return tune(lib, cand, n_q, k, best, all, cap, n_all,
                [&](hd_search_form f, uint32_t *oi, void *osc, cudaStream_t s) {
                    return hd_search_dot_dispatch(lib, f, d_q_comp, d_q_mz, d_q_charge, n_q, win, k, oi,
                                                  static_cast<int32_t *>(osc), s);
                });
}

}  // extern "C"
