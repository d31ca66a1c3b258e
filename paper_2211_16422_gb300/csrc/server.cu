// server.cu -- continuous-batching search server on a resident library.
//
// The paper batches queries to fill device memory (Section 4.1); a serving
// process sees requests arrive one by one instead.  Requests are queued on
// submit (their inputs copied, so the caller may reuse its buffers).  A
// scheduler thread owns `slots` execution slots, each with its own stream,
// page-locked staging and completion event.  Whenever a slot is free and the
// device-memory budget allows, it coalesces every pending request that fits
// (up to max_batch_queries) into one batch, copies it to the device, encodes
// it (Eq. 1) and runs the multi-window search (Section 3.4), then copies the
// top-k back.  Batches in different slots overlap on the device; a request
// that arrives while others run joins the next batch that starts.  Results
// are exactly those of searching each request alone: the top-k of a query
// depends only on that query.  On a multi-bit library (Section 4.3) the
// batch is encoded into components and scored by the dot-product search, and
// requests come through hd_server_submit_dot with score outputs.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hd_internal.cuh"

namespace {

using clock_t_ = std::chrono::steady_clock;

double now_s()
{
    return std::chrono::duration<double>(clock_t_::now().time_since_epoch()).count();
}

struct request {
    uint64_t id = 0;
    std::vector<uint32_t> off, bins;
    std::vector<uint8_t> lv, z;
    std::vector<double> mz;
    uint32_t n_q = 0;
    hd_window win{};
    uint32_t *out_idx = nullptr;
    uint16_t *out_dist = nullptr;   // binary library
    int32_t *out_score = nullptr;   // multi-bit library
    double t_submit = 0, t_start = 0, t_done = 0;
    uint32_t batch_queries = 0;
    bool done = false;
    hd_status status = HD_OK;
};
using req_ptr = std::shared_ptr<request>;

template <class T>
struct pinned {
    T *p = nullptr;
    size_t cap = 0;
    bool reserve(size_t n)
    {
        if (n <= cap) return true;
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        size_t want = n + n / 2 + 64;
        if (cudaHostAlloc((void **)&p, want * sizeof(T), cudaHostAllocDefault) != cudaSuccess) return false;
        cap = want;
        return true;
    }
    ~pinned()
    {
        if (p) cudaFreeHost(p);
    }
};

struct slot {
    uint32_t index = 0;
    uint64_t batch = 0;               // number of the batch in flight
    cudaStream_t stream = nullptr;
    cudaEvent_t start_ev = nullptr;   // recorded before the batch's first copy
    cudaEvent_t done_ev = nullptr;    // recorded after its last copy
    pinned<uint32_t> off, bins, out_idx;
    pinned<uint8_t> lv, z, cls;
    pinned<double> mz;
    pinned<uint16_t> out_dist;
    pinned<int32_t> out_score;
    std::vector<req_ptr> reqs;
    size_t bytes = 0;
    bool busy = false;
    hd_status launch_status = HD_OK;
};

}  // namespace

struct hd_server {
    hd_ctx *ctx = nullptr;
    const hd_library *lib = nullptr;
    hd_server_params p{};
    size_t budget = 0, inflight_bytes = 0, per_query_bytes = 0;
    bool multibit = false;            // lib->bits > 1: components, dot-product scores
    hd_search_form form = HD_FORM_AUTO;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<req_ptr> pending;
    std::unordered_map<uint64_t, req_ptr> reqs;
    std::vector<std::unique_ptr<slot>> slots;
    uint64_t next_id = 1;
    hd_server_stats stats{};
    uint32_t busy_slots = 0;
    cudaEvent_t ref_ev = nullptr;                 // device-time origin of the batch log
    std::deque<hd_batch_record> log;              // the last HD_SERVER_LOG_CAP finished batches
    static constexpr size_t HD_SERVER_LOG_CAP = 4096;

    // Launches the requests in `batch` on slot `s`.  Called with `mu` held.
    hd_status launch(slot &s, std::vector<req_ptr> &batch)
    {
        uint32_t nq = 0, nnz = 0;
        std::vector<hd_window> wins;
        std::vector<uint8_t> rcls(batch.size());
        for (size_t i = 0; i < batch.size(); ++i) {
            auto &r = *batch[i];
            nq += r.n_q;
            nnz += r.off[r.n_q];
            size_t c = 0;
            while (c < wins.size() && !(wins[c].tol == r.win.tol && wins[c].unit == r.win.unit)) ++c;
            if (c == wins.size()) wins.push_back(r.win);
            rcls[i] = (uint8_t)c;
        }
        if (!s.off.reserve(nq + 1) || !s.bins.reserve(nnz + 1) || !s.lv.reserve(nnz + 1) || !s.mz.reserve(nq) ||
            !s.z.reserve(nq) || !s.cls.reserve(nq) || !s.out_idx.reserve((size_t)nq * p.k) ||
            (multibit ? !s.out_score.reserve((size_t)nq * p.k) : !s.out_dist.reserve((size_t)nq * p.k)))
            return hd_fail(HD_ERR_OOM, "hd_server: page-locked staging allocation failed");
        uint32_t q0 = 0, p0 = 0;
        s.off.p[0] = 0;
        for (size_t i = 0; i < batch.size(); ++i) {
            auto &r = *batch[i];
            const uint32_t rn = r.off[r.n_q];
            for (uint32_t q = 0; q < r.n_q; ++q) s.off.p[q0 + q + 1] = p0 + r.off[q + 1];
            if (rn) {
                std::memcpy(s.bins.p + p0, r.bins.data(), rn * 4);
                std::memcpy(s.lv.p + p0, r.lv.data(), rn);
            }
            std::memcpy(s.mz.p + q0, r.mz.data(), r.n_q * 8);
            std::memcpy(s.z.p + q0, r.z.data(), r.n_q);
            std::memset(s.cls.p + q0, rcls[i], r.n_q);
            q0 += r.n_q;
            p0 += rn;
        }
        hd_qwin win;
        hd_status st = hd_make_qwin(nullptr, wins.data(), (uint32_t)wins.size(), &win);
        if (st != HD_OK) return st;
        hd_arena plan;
        // query rows: W words of HV bits, or D int8 components (D/8 words) on a multi-bit library
        const size_t row_words = multibit ? lib->dim / 8 : ctx->W;
        auto carve = [&](hd_arena &ar, uint32_t **off, uint32_t **bins, uint8_t **lv, double **mz, uint8_t **z,
                         uint8_t **cls, uint64_t **hv, uint32_t **oi, uint16_t **od, int32_t **os) {
            *off = ar.take<uint32_t>(nq + 1);
            *bins = ar.take<uint32_t>(nnz ? nnz : 1);
            *lv = ar.take<uint8_t>(nnz ? nnz : 1);
            *mz = ar.take<double>(nq);
            *z = ar.take<uint8_t>(nq);
            *cls = ar.take<uint8_t>(nq);
            *hv = ar.take<uint64_t>((size_t)nq * row_words);
            *oi = ar.take<uint32_t>((size_t)nq * p.k);
            *od = multibit ? nullptr : ar.take<uint16_t>((size_t)nq * p.k);
            *os = multibit ? ar.take<int32_t>((size_t)nq * p.k) : nullptr;
        };
        uint32_t *d_off, *d_bins, *d_oi;
        uint8_t *d_lv, *d_z, *d_cls;
        double *d_mz;
        uint64_t *d_hv;
        uint16_t *d_od;
        int32_t *d_os;
        carve(plan, &d_off, &d_bins, &d_lv, &d_mz, &d_z, &d_cls, &d_hv, &d_oi, &d_od, &d_os);
        hd_arena ar;
        if (cudaMallocAsync((void **)&ar.base, plan.used, s.stream) != cudaSuccess) {
            cudaGetLastError();
            return hd_fail(HD_ERR_OOM, "hd_server: device allocation failed");
        }
        carve(ar, &d_off, &d_bins, &d_lv, &d_mz, &d_z, &d_cls, &d_hv, &d_oi, &d_od, &d_os);
        win.cls = wins.size() > 1 ? d_cls : nullptr;
        const auto H2D = cudaMemcpyHostToDevice, D2H = cudaMemcpyDeviceToHost;
        cudaEventRecord(s.start_ev, s.stream);
        cudaError_t e = cudaMemcpyAsync(d_off, s.off.p, (size_t)(nq + 1) * 4, H2D, s.stream);
        if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(d_bins, s.bins.p, (size_t)nnz * 4, H2D, s.stream);
        if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(d_lv, s.lv.p, nnz, H2D, s.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_mz, s.mz.p, (size_t)nq * 8, H2D, s.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_z, s.z.p, nq, H2D, s.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_cls, s.cls.p, nq, H2D, s.stream);
        if (e == cudaSuccess) {
            if (multibit)
                hd_encode_mb_launch(ctx, d_off, d_bins, d_lv, nq, lib->bits, reinterpret_cast<int8_t *>(d_hv), s.stream);
            else
                hd_encode_launch(ctx, d_off, d_bins, d_lv, nq, d_hv, s.stream);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            st = multibit ? hd_search_dot_dispatch(lib, form, reinterpret_cast<const int8_t *>(d_hv), d_mz, d_z, nq, win,
                                                   p.k, d_oi, d_os, s.stream)
                          : hd_search_dispatch(lib, d_hv, d_mz, d_z, nq, win, p.k, p.form, d_oi, d_od, s.stream);
            if (st != HD_OK) e = cudaErrorUnknown;
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(s.out_idx.p, d_oi, (size_t)nq * p.k * 4, D2H, s.stream);
        if (e == cudaSuccess && multibit)
            e = cudaMemcpyAsync(s.out_score.p, d_os, (size_t)nq * p.k * 4, D2H, s.stream);
        if (e == cudaSuccess && !multibit)
            e = cudaMemcpyAsync(s.out_dist.p, d_od, (size_t)nq * p.k * 2, D2H, s.stream);
        cudaFreeAsync(ar.base, s.stream);
        cudaEventRecord(s.done_ev, s.stream);
        if (st != HD_OK) return st;
        if (e != cudaSuccess) return hd_cuda_fail(e, "hd_server: batch launch");
        return HD_OK;
    }

    // Copies a finished slot's results out to its requests.  `mu` held.
    void finish(slot &s)
    {
        const double t = now_s();
        uint32_t q0 = 0;
        hd_status st = s.launch_status;
        if (st == HD_OK && cudaEventSynchronize(s.done_ev) != cudaSuccess) st = HD_ERR_CUDA;
        if (st == HD_OK) {
            const hd_status ls = hd_library_status(const_cast<hd_library *>(lib));
            const hd_status cs = hd_ctx_status(ctx);
            st = ls != HD_OK ? ls : cs;
        }
        if (st == HD_OK) {   // the batch's device-time interval, for the overlap record
            float a = 0.f, b = 0.f;
            if (cudaEventElapsedTime(&a, ref_ev, s.start_ev) == cudaSuccess &&
                cudaEventElapsedTime(&b, ref_ev, s.done_ev) == cudaSuccess) {
                uint32_t nq = 0;
                for (auto &rp : s.reqs) nq += rp->n_q;
                log.push_back(hd_batch_record{s.batch, s.index, nq, (uint32_t)s.reqs.size(), (double)a, (double)b});
                if (log.size() > HD_SERVER_LOG_CAP) log.pop_front();
            }
        }
        for (auto &rp : s.reqs) {
            auto &r = *rp;
            if (st == HD_OK) {
                std::memcpy(r.out_idx, s.out_idx.p + (size_t)q0 * p.k, (size_t)r.n_q * p.k * 4);
                if (multibit) std::memcpy(r.out_score, s.out_score.p + (size_t)q0 * p.k, (size_t)r.n_q * p.k * 4);
                else std::memcpy(r.out_dist, s.out_dist.p + (size_t)q0 * p.k, (size_t)r.n_q * p.k * 2);
            }
            q0 += r.n_q;
            r.status = st;
            r.t_done = t;
            r.done = true;
            stats.completed += 1;
            stats.queries += r.n_q;
        }
        s.reqs.clear();
        inflight_bytes -= s.bytes;
        s.bytes = 0;
        s.busy = false;
        --busy_slots;
        cv_done.notify_all();
    }

    void loop()
    {
        cudaSetDevice(lib->device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            for (auto &sp : slots)
                if (sp->busy && (sp->launch_status != HD_OK || cudaEventQuery(sp->done_ev) != cudaErrorNotReady))
                    finish(*sp);
            bool launched = false;
            for (auto &sp : slots) {
                if (sp->busy || pending.empty()) continue;
                std::vector<req_ptr> batch;
                uint32_t nq = 0;
                size_t bytes = 0;
                std::vector<hd_window> wins;
                while (!pending.empty()) {
                    auto &r = *pending.front();
                    bool new_win = true;
                    for (auto &w : wins)
                        if (w.tol == r.win.tol && w.unit == r.win.unit) new_win = false;
                    if (new_win && wins.size() == HD_MAX_WINDOWS) break;
                    const size_t b = (size_t)r.n_q * per_query_bytes;
                    if (!batch.empty() && (nq + r.n_q > p.max_batch_queries)) break;
                    // admit by device memory; a lone request on an idle device always runs
                    const bool mem_ok = inflight_bytes + bytes + b <= budget;
                    if (!mem_ok && !(batch.empty() && busy_slots == 0)) break;
                    if (new_win) wins.push_back(r.win);
                    batch.push_back(pending.front());
                    pending.pop_front();
                    nq += r.n_q;
                    bytes += b;
                }
                if (batch.empty()) break;   // memory budget: wait for a slot to drain
                const double t = now_s();
                for (auto &r : batch) {
                    r->t_start = t;
                    r->batch_queries = nq;
                }
                sp->reqs = batch;
                sp->bytes = bytes;
                sp->batch = stats.batches;
                sp->busy = true;
                ++busy_slots;
                inflight_bytes += bytes;
                sp->launch_status = launch(*sp, batch);
                stats.batches += 1;
                if (busy_slots > stats.max_inflight) stats.max_inflight = busy_slots;
                launched = true;
            }
            if (stop && pending.empty() && busy_slots == 0) break;
            if (!launched) cv_work.wait_for(lk, std::chrono::microseconds(busy_slots ? 50 : 2000));
        }
    }
};

namespace {

hd_status submit(hd_server *s, const uint32_t *h_offsets, const uint32_t *h_bins, const uint8_t *h_levels,
                 const double *h_q_mz, const uint8_t *h_q_charge, uint32_t n_q, double tol, hd_tol_unit unit,
                 uint32_t *h_out_idx, uint16_t *h_out_dist, int32_t *h_out_score, uint64_t *request_id,
                 const char *fn)
{
    const std::string f(fn);
    if (!s || !request_id) return hd_fail(HD_ERR_INVALID_ARG, f + ": null argument");
    if (n_q == 0 || !h_offsets || !h_q_mz || !h_q_charge || !h_out_idx || (!h_out_dist && !h_out_score))
        return hd_fail(HD_ERR_INVALID_ARG, f + ": empty request or null buffer");
    if (s->multibit != (h_out_score != nullptr))
        return hd_fail(HD_ERR_INVALID_ARG, s->multibit ? f + ": multi-bit library: use hd_server_submit_dot"
                                                       : f + ": binary library: use hd_server_submit");
    if (!(tol >= 0.0) || tol > 1.7976931348623157e308 || (unit != HD_TOL_DA && unit != HD_TOL_PPM && unit != HD_TOL_MASS))
        return hd_fail(HD_ERR_INVALID_ARG, f + ": bad window");
    const uint32_t nnz = h_offsets[n_q] - h_offsets[0];
    if (nnz && (!h_bins || !h_levels)) return hd_fail(HD_ERR_INVALID_ARG, f + ": null CSR buffer");
    for (uint32_t q = 0; q < n_q; ++q)
        if (h_offsets[q + 1] < h_offsets[q]) return hd_fail(HD_ERR_INVALID_ARG, f + ": bad offsets");
    auto r = std::make_shared<request>();
    r->n_q = n_q;
    r->off.resize(n_q + 1);
    for (uint32_t q = 0; q <= n_q; ++q) r->off[q] = h_offsets[q] - h_offsets[0];
    r->bins.assign(h_bins ? h_bins + h_offsets[0] : nullptr, h_bins ? h_bins + h_offsets[n_q] : nullptr);
    r->lv.assign(h_levels ? h_levels + h_offsets[0] : nullptr, h_levels ? h_levels + h_offsets[n_q] : nullptr);
    r->mz.assign(h_q_mz, h_q_mz + n_q);
    r->z.assign(h_q_charge, h_q_charge + n_q);
    r->win = hd_window{tol, unit};
    r->out_idx = h_out_idx;
    r->out_dist = h_out_dist;
    r->out_score = h_out_score;
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stop) return hd_fail(HD_ERR_INVALID_ARG, f + ": server is stopping");
        r->id = s->next_id++;
        s->reqs[r->id] = r;
        s->pending.push_back(r);
        s->stats.submitted += 1;
    }
    s->cv_work.notify_one();
    *request_id = r->id;
    return HD_OK;
}

}  // namespace

extern "C" {

hd_status hd_server_create(hd_ctx *ctx, const hd_library *lib, const hd_server_params *params, hd_server **out)
{
    if (!out) return hd_fail(HD_ERR_INVALID_ARG, "hd_server_create: null output");
    *out = nullptr;
    if (!ctx || !lib || !params) return hd_fail(HD_ERR_INVALID_ARG, "hd_server_create: null argument");
    if (ctx->p.dim != lib->dim) return hd_fail(HD_ERR_INVALID_ARG, "hd_server_create: ctx and library dims differ");
    if (params->k < 1 || params->k > 16) return hd_fail(HD_ERR_INVALID_ARG, "hd_server_create: k must be in [1, 16]");
    if (params->slots < 1 || params->slots > 64)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_server_create: slots must be in [1, 64]");
    if (params->max_batch_queries < 1) return hd_fail(HD_ERR_INVALID_ARG, "hd_server_create: max_batch_queries >= 1");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != lib->device)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_server_create: library belongs to another device");
    auto srv = std::make_unique<hd_server>();
    srv->ctx = ctx;
    srv->lib = lib;
    srv->p = *params;
    srv->multibit = !hd_lib_binary(lib);
    srv->form = params->form;
    if (srv->multibit) {   // the dot-product search runs on a copy the library holds
        hd_status st0 = hd_dot_check(lib, &srv->form, "hd_server_create (multi-bit library)");
        if (st0 != HD_OK) return st0;
    }
    const size_t row_tc = (size_t)lib->dim * 2;
    srv->per_query_bytes = (srv->multibit ? (size_t)lib->dim : (size_t)lib->dim / 8) + row_tc + 1024 +
                           (size_t)params->k * 32;
    size_t free_b = 0, total_b = 0;
    HD_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    srv->budget = params->mem_budget_bytes ? (size_t)params->mem_budget_bytes : free_b / 2;
    for (uint32_t i = 0; i < params->slots; ++i) {
        auto sl = std::make_unique<slot>();
        sl->index = i;
        HD_CUDA_TRY(cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking));
        HD_CUDA_TRY(cudaEventCreate(&sl->start_ev));
        HD_CUDA_TRY(cudaEventCreate(&sl->done_ev));
        srv->slots.push_back(std::move(sl));
    }
    HD_CUDA_TRY(cudaEventCreate(&srv->ref_ev));
    HD_CUDA_TRY(cudaEventRecord(srv->ref_ev, srv->slots[0]->stream));
    HD_CUDA_TRY(cudaEventSynchronize(srv->ref_ev));
    hd_server *s = srv.release();
    s->th = std::thread([s] { s->loop(); });
    *out = s;
    return HD_OK;
}

hd_status hd_server_submit(hd_server *s, const uint32_t *h_offsets, const uint32_t *h_bins, const uint8_t *h_levels,
                           const double *h_q_mz, const uint8_t *h_q_charge, uint32_t n_q, double tol,
                           hd_tol_unit unit, uint32_t *h_out_idx, uint16_t *h_out_dist, uint64_t *request_id)
{
    if (!h_out_dist) return hd_fail(HD_ERR_INVALID_ARG, "hd_server_submit: null buffer");
    return submit(s, h_offsets, h_bins, h_levels, h_q_mz, h_q_charge, n_q, tol, unit, h_out_idx, h_out_dist, nullptr,
                  request_id, "hd_server_submit");
}

hd_status hd_server_submit_dot(hd_server *s, const uint32_t *h_offsets, const uint32_t *h_bins,
                               const uint8_t *h_levels, const double *h_q_mz, const uint8_t *h_q_charge, uint32_t n_q,
                               double tol, hd_tol_unit unit, uint32_t *h_out_idx, int32_t *h_out_score,
                               uint64_t *request_id)
{
    if (!h_out_score) return hd_fail(HD_ERR_INVALID_ARG, "hd_server_submit_dot: null buffer");
    return submit(s, h_offsets, h_bins, h_levels, h_q_mz, h_q_charge, n_q, tol, unit, h_out_idx, nullptr, h_out_score,
                  request_id, "hd_server_submit_dot");
}

hd_status hd_server_wait(hd_server *s, uint64_t id, double timeout_s, hd_request_info *info)
{
    if (!s) return hd_fail(HD_ERR_INVALID_ARG, "hd_server_wait: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return hd_fail(HD_ERR_INVALID_ARG, "hd_server_wait: unknown request");
    req_ptr r = it->second;
    const auto deadline = clock_t_::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9);
    while (!r->done)
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done)
            return hd_fail(HD_ERR_TIMEOUT, "hd_server_wait: request not finished in time");
    if (info) {
        info->latency_s = r->t_done - r->t_submit;
        info->queue_s = r->t_start - r->t_submit;
        info->n_queries = r->n_q;
        info->batch_queries = r->batch_queries;
    }
    s->reqs.erase(it);
    if (r->status != HD_OK) return hd_fail(r->status, "hd_server: request failed");
    return HD_OK;
}

hd_status hd_server_batch_log(hd_server *s, hd_batch_record *out, uint32_t cap, uint32_t *n)
{
    if (!s || !n || (cap && !out)) return hd_fail(HD_ERR_INVALID_ARG, "hd_server_batch_log: null argument");
    std::lock_guard<std::mutex> g(s->mu);
    const uint32_t m = (uint32_t)std::min<size_t>(cap, s->log.size());
    for (uint32_t i = 0; i < m; ++i) out[i] = s->log[s->log.size() - m + i];
    *n = m;
    return HD_OK;
}

hd_status hd_server_stats_get(hd_server *s, hd_server_stats *out)
{
    if (!s || !out) return hd_fail(HD_ERR_INVALID_ARG, "hd_server_stats_get: null argument");
    std::lock_guard<std::mutex> g(s->mu);
    *out = s->stats;
    return HD_OK;
}

void hd_server_destroy(hd_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (auto &sl : s->slots) {
        if (sl->stream) {
            cudaStreamSynchronize(sl->stream);
            cudaStreamDestroy(sl->stream);
        }
        if (sl->start_ev) cudaEventDestroy(sl->start_ev);
        if (sl->done_ev) cudaEventDestroy(sl->done_ev);
    }
    if (s->ref_ev) cudaEventDestroy(s->ref_ev);
    delete s;
}

}  // extern "C"
