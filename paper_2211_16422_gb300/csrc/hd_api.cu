// hd_api.cu -- the extern "C" boundary of libhd: argument checks, object
// life cycle and the order of launches.  Every computation runs in the
// kernels of the other translation units.
#include <cmath>
#include <cstring>
#include <cstdio>
#include <string>
#include <vector>

#include "hd_internal.cuh"

static thread_local std::string g_msg;

hd_status hd_fail(hd_status s, const std::string &msg)
{
    g_msg = msg;
    return s;
}

hd_status hd_cuda_fail(cudaError_t e, const char *what)
{
    g_msg = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return HD_ERR_OOM;
    return HD_ERR_CUDA;
}

#define HD_CHECK(cond, msg)                                                 \
    do {                                                                    \
        if (!(cond)) return hd_fail(HD_ERR_INVALID_ARG, msg);               \
    } while (0)

namespace {

hd_status status_alloc(hd_status_word &w)
{
    HD_CUDA_TRY(cudaHostAlloc((void **)&w.host, sizeof(uint32_t), cudaHostAllocMapped));
    *w.host = 0;
    HD_CUDA_TRY(cudaHostGetDevicePointer((void **)&w.dev, w.host, 0));
    return HD_OK;
}

void status_free(hd_status_word &w)
{
    if (w.host) cudaFreeHost(w.host);
    w.host = w.dev = nullptr;
}

hd_status status_take(hd_status_word &w, const char *who)
{
    if (!w.host) return HD_OK;
    const uint32_t v = __atomic_exchange_n(w.host, 0u, __ATOMIC_SEQ_CST);
    if (v & HD_DEV_TIMEOUT)
        return hd_fail(HD_ERR_TIMEOUT, std::string(who) + ": a bounded device wait expired");
    if (v & HD_DEV_TMEM)
        return hd_fail(HD_ERR_CUDA, std::string(who) + ": paired CTAs hold different tensor-memory columns");
    if (v & HD_DEV_BAD_INPUT)
        return hd_fail(HD_ERR_INVALID_ARG, std::string(who) + ": malformed input found on the device");
    return HD_OK;
}

hd_status check_device(int want)
{
    int dev = -1;
    HD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != want) return hd_fail(HD_ERR_INVALID_ARG, "object belongs to another CUDA device");
    return HD_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool form_ok(hd_search_form f)
{
    return f == HD_FORM_AUTO || f == HD_FORM_POPC || hd_is_tc_form(f);
}
bool unit_ok(hd_tol_unit u) { return u == HD_TOL_DA || u == HD_TOL_PPM || u == HD_TOL_MASS; }

bool tol_ok(double tol) { return std::isfinite(tol) && tol >= 0.0; }

// --------------------------------------------------------------- library
__global__ void k_gather_rows(const uint64_t *__restrict__ hv, const double *__restrict__ mz,
                              const uint8_t *__restrict__ z, const uint32_t *__restrict__ perm,
                              uint32_t n, uint32_t W, uint64_t *__restrict__ o_hv,
                              double *__restrict__ o_mz, uint8_t *__restrict__ o_z,
                              uint32_t *__restrict__ o_orig, uint32_t *status)
{
    const uint32_t r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const uint32_t lane = threadIdx.x & 31;
    if (r >= n) return;
    const uint32_t src = perm[r];
    const uint2 *s2 = reinterpret_cast<const uint2 *>(hv + (size_t)src * W);
    uint2 *d2 = reinterpret_cast<uint2 *>(o_hv + (size_t)r * W);
    for (uint32_t w = lane; w < W; w += 32) d2[w] = s2[w];
    if (lane == 0) {
        const double m = mz[src];
        if (!isfinite(m)) hd_flag(status, HD_DEV_BAD_INPUT);
        o_mz[r] = m;
        o_z[r] = z[src];
        o_orig[r] = src;
    }
}

// cstart[c] = first row whose charge is >= c, c = 0..256.
__global__ void k_charge_start(const uint8_t *__restrict__ z, uint32_t n, uint32_t *__restrict__ cstart)
{
    const uint32_t c = threadIdx.x;
    if (c > 256) return;
    uint32_t a = 0, b = n;
    while (a < b) {
        const uint32_t m = a + ((b - a) >> 1);
        if ((uint32_t)z[m] >= c) b = m; else a = m + 1;
    }
    cstart[c] = a;
}

void lib_release(hd_library *lib)
{
    if (!lib) return;
    cudaFree(lib->hv);
    cudaFree(lib->mz);
    cudaFree(lib->charge);
    cudaFree(lib->orig);
    cudaFree(lib->charge_start);
    cudaFree(lib->x_fp8);
    cudaFree(lib->x_bf16);
    cudaFree(lib->x_fp4);
    cudaFree(lib->decoy);
    cudaFree(lib->comp);
    cudaFree(lib->x_planes);
    cudaFree(lib->usum);
    status_free(lib->status);
    delete lib;
}

void ctx_release(hd_ctx *ctx)
{
    if (!ctx) return;
    cudaFree(ctx->F);
    cudaFree(ctx->L);
    cudaFree(ctx->rank_F);
    cudaFree(ctx->rank_L);
    status_free(ctx->status);
    delete ctx;
}

struct scoped_stream {
    cudaStream_t s = nullptr;
    ~scoped_stream()
    {
        if (s) cudaStreamDestroy(s);
    }
};

}  // namespace

hd_status hd_make_qwin(const uint8_t *cls, const hd_window *windows, uint32_t n_windows, hd_qwin *out)
{
    HD_CHECK(windows && n_windows >= 1 && n_windows <= HD_MAX_WINDOWS,
             "windows: need 1..16 window descriptions");
    hd_qwin w;
    w.cls = n_windows > 1 ? cls : nullptr;
    w.n = n_windows;
    for (uint32_t i = 0; i < n_windows; ++i) {
        HD_CHECK(tol_ok(windows[i].tol), "windows: tol must be finite and >= 0");
        HD_CHECK(unit_ok(windows[i].unit), "windows: bad unit");
        w.w[i] = hd_single_window(windows[i].tol, windows[i].unit).w[0];
    }
    *out = w;
    return HD_OK;
}

hd_status hd_dot_check(const hd_library *lib, hd_search_form *form, const std::string &name)
{
    if (*form != HD_FORM_AUTO && *form != HD_FORM_POPC && !hd_is_tc_form(*form))
        return hd_fail(HD_ERR_INVALID_ARG, name + ": form must be AUTO, POPC or a tensor-core form");
    *form = hd_dot_form(lib, *form);
    if (!hd_dot_copy(lib, *form) && lib->n > 0)
        return hd_fail(HD_ERR_INVALID_ARG, name + ": call hd_library_prepare for this form first");
    if (*form == HD_FORM_TC_MXF4 && lib->dim % 256 != 0)
        return hd_fail(HD_ERR_INVALID_ARG, name + ": the kind::mxf4 form needs D to be a multiple of 256");
    return HD_OK;
}

hd_status hd_search_dispatch(const hd_library *lib, const uint64_t *q_hv, const double *q_mz, const uint8_t *q_charge,
                             uint32_t n_q, const hd_qwin &win, uint32_t k, hd_search_form form, uint32_t *out_idx,
                             uint16_t *out_dist, cudaStream_t s)
{
    if (!hd_lib_binary(lib)) return hd_fail(HD_ERR_INVALID_ARG, "multi-bit library: search it with hd_search_dot");
    if (form == HD_FORM_AUTO) {
        form = lib->auto_form;
        const bool ok = form == HD_FORM_POPC || (form != HD_FORM_AUTO && hd_tc_copy(lib, form));
        if (!ok) {
            form = hd_fastest_tc_form(lib);
            if (form == HD_FORM_AUTO) form = HD_FORM_POPC;
        }
    }
    if (hd_is_tc_form(form)) {
        HD_CHECK(hd_tc_copy(lib, form) != nullptr || lib->n == 0,
                 "hd_search_open: call hd_library_prepare for this form first");
        HD_CHECK(form != HD_FORM_TC_MXF4 || lib->dim % 256 == 0,
                 "hd_search_open: the kind::mxf4 form needs D to be a multiple of 256");
        return hd_search_mma_run(lib, form, q_hv, q_mz, q_charge, n_q, win, k, out_idx, out_dist, s);
    }
    return hd_search_popc_run(lib, q_hv, q_mz, q_charge, n_q, win, k, out_idx, out_dist, s);
}

bool hd_take_injected_stall(const hd_library *lib)
{
    uint32_t n = __atomic_load_n(&lib->inject_stalls, __ATOMIC_SEQ_CST);
    while (n > 0)
        if (__atomic_compare_exchange_n(&lib->inject_stalls, &n, n - 1, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST))
            return true;
    return false;
}

namespace {

// Shared by the binary and multi-bit builds: sorts the references by (charge,
// precursor m/z, input index) and gathers `row_words` 64-bit words of each row
// (binary HVs: D/64; int8 components: D/8) into the library's sorted rows.
hd_status build_rows(hd_ctx *ctx, const uint64_t *d_rows, uint32_t bits, const double *d_prec_mz,
                     const uint8_t *d_charge, uint32_t n_refs, hd_library **out, const char *fn)
{
    hd_library *lib = new hd_library;
    lib->n = n_refs;
    lib->dim = ctx->p.dim;
    lib->W = ctx->W;
    lib->bits = bits;
    lib->device = ctx->device;
    lib->num_sms = ctx->num_sms;
    auto fail = [&](hd_status s) {
        lib_release(lib);
        return s;
    };
    const size_t n1 = n_refs ? n_refs : 1;
    const uint32_t row_words = bits == 1 ? lib->W : lib->dim / 8;
    uint64_t *rows = nullptr;
    if (cudaMalloc(&rows, n1 * row_words * 8) != cudaSuccess || cudaMalloc(&lib->mz, n1 * 8) != cudaSuccess ||
        cudaMalloc(&lib->charge, n1) != cudaSuccess || cudaMalloc(&lib->orig, n1 * 4) != cudaSuccess ||
        cudaMalloc(&lib->charge_start, 257 * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(rows);
        return fail(hd_fail(HD_ERR_OOM, std::string(fn) + ": allocation failed"));
    }
    if (bits == 1) lib->hv = rows;
    else lib->comp = reinterpret_cast<int8_t *>(rows);
    hd_status st = status_alloc(lib->status);
    if (st != HD_OK) return fail(st);
    scoped_stream ss;
    if (cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking) != cudaSuccess)
        return fail(hd_fail(HD_ERR_CUDA, std::string(fn) + ": stream creation failed"));
    if (n_refs > 0) {
        hd_arena plan;
        uint32_t *perm = plan.take<uint32_t>(n_refs);
        hd_sort_charge_mz(d_prec_mz, d_charge, nullptr, n_refs, nullptr, plan, ss.s);
        hd_arena ar;
        if (cudaMallocAsync((void **)&ar.base, plan.used, ss.s) != cudaSuccess) {
            cudaGetLastError();
            return fail(hd_fail(HD_ERR_OOM, std::string(fn) + ": scratch allocation failed"));
        }
        perm = ar.take<uint32_t>(n_refs);
        hd_sort_charge_mz(d_prec_mz, d_charge, nullptr, n_refs, perm, ar, ss.s);
        hd_count_launches(1), k_gather_rows<<<hd_ceil_div(n_refs, 8), 256, 0, ss.s>>>(d_rows, d_prec_mz, d_charge, perm, n_refs,
                                                                row_words, rows, lib->mz, lib->charge,
                                                                lib->orig, lib->status.dev);
        cudaFreeAsync(ar.base, ss.s);
    }
    hd_count_launches(1), k_charge_start<<<1, 288, 0, ss.s>>>(lib->charge, n_refs, lib->charge_start);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(lib->charge_start_h, lib->charge_start, 257 * 4,
                                              cudaMemcpyDeviceToHost, ss.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ss.s);
    if (e != cudaSuccess) return fail(hd_cuda_fail(e, fn));
    st = status_take(lib->status, fn);
    if (st != HD_OK) return fail(hd_fail(st, std::string(fn) + ": precursor m/z must be finite"));
    if (bits > 1) {   // the default tensor-core copy; it also checks the component range
        st = hd_library_expand(lib, bits <= 3 ? HD_FORM_TC_FP4 : HD_FORM_TC_FP8, ss.s);
        if (st != HD_OK) return fail(st);
        e = cudaStreamSynchronize(ss.s);
        if (e != cudaSuccess) return fail(hd_cuda_fail(e, fn));
        st = status_take(lib->status, fn);
        if (st != HD_OK) return fail(hd_fail(st, std::string(fn) + ": components must lie in [-m, m]"));
    }
    *out = lib;
    return HD_OK;
}

}  // namespace

extern "C" {

const char *hd_status_string(hd_status s)
{
    switch (s) {
    case HD_OK: return "HD_OK";
    case HD_ERR_INVALID_ARG: return "HD_ERR_INVALID_ARG";
    case HD_ERR_OOM: return "HD_ERR_OOM";
    case HD_ERR_CUDA: return "HD_ERR_CUDA";
    case HD_ERR_TIMEOUT: return "HD_ERR_TIMEOUT";
    case HD_ERR_UNSUPPORTED: return "HD_ERR_UNSUPPORTED";
    }
    return "HD_ERR_UNKNOWN";
}

const char *hd_last_error_message(void) { return g_msg.c_str(); }

uint32_t hd_version(void) { return 100u; }

// Scratch comes from the device's default stream-ordered pool, which by
// default returns its memory at every synchronisation, so each call ending in
// one (hd_search_host, a cascade level) would map its scratch again: 0.5 ms of
// a 36.5 ms end-to-end call at 1M x 50k, D = 8192.  The pool keeps up to
// HD_SCRATCH_RETAIN bytes mapped instead; a higher threshold the caller set
// stays.
constexpr uint64_t HD_SCRATCH_RETAIN = 4ull << 30;
static void keep_scratch_mapped(int device)
{
    cudaMemPool_t pool;
    uint64_t cur = 0;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && cur < HD_SCRATCH_RETAIN) {
        uint64_t want = HD_SCRATCH_RETAIN;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &want);
    }
    cudaGetLastError();   // a pool that cannot be tuned only costs the re-mapping
}

hd_status hd_ctx_create(const hd_params *p, hd_ctx **out)
{
    HD_CHECK(p && out, "hd_ctx_create: null argument");
    *out = nullptr;
    HD_CHECK(p->dim >= 128 && p->dim <= 32768 && p->dim % 128 == 0,
             "hd_ctx_create: dim must be a multiple of 128 in [128, 32768]");
    HD_CHECK(p->n_levels >= 2 && p->n_levels <= 256, "hd_ctx_create: n_levels must be in [2, 256]");
    HD_CHECK(p->n_bins >= 1, "hd_ctx_create: n_bins must be >= 1");
    HD_CHECK(p->alpha <= p->dim, "hd_ctx_create: alpha must be <= dim");
    HD_CHECK(p->position_mode <= HD_POS_RANDOM, "hd_ctx_create: unknown position_mode");
    HD_CHECK(p->encoder <= HD_ENC_PROJECTION, "hd_ctx_create: unknown encoder");
    HD_CHECK(p->position_mode != HD_POS_WALK || (p->alpha <= 256 && p->n_bins <= (1u << 24)),
             "hd_ctx_create: a position walk takes alpha <= 256 flips per step and n_bins <= 2^24");
    HD_CHECK(p->position_mode != HD_POS_RANDOM || (uint64_t)p->n_bins * (p->dim / 32) <= 0xFFFFFFFFull,
             "hd_ctx_create: n_bins * dim / 32 must fit 32 bits for random position HVs");
    hd_ctx *c = new hd_ctx;
    c->p = *p;
    c->W = p->dim / 64;
    auto fail = [&](hd_status s) {
        ctx_release(c);
        return s;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        return fail(hd_fail(HD_ERR_CUDA, "hd_ctx_create: no usable CUDA device"));
    keep_scratch_mapped(c->device);
    const size_t nF = (size_t)p->n_bins * c->W, nL = (size_t)p->n_levels * c->W;
    if (cudaMalloc(&c->F, nF * 8) != cudaSuccess || cudaMalloc(&c->L, nL * 8) != cudaSuccess ||
        cudaMalloc(&c->rank_F, (size_t)p->dim * 4) != cudaSuccess ||
        cudaMalloc(&c->rank_L, (size_t)p->dim * 4) != cudaSuccess) {
        cudaGetLastError();
        return fail(hd_fail(HD_ERR_OOM, "hd_ctx_create: item memory allocation failed"));
    }
    hd_status st = status_alloc(c->status);
    if (st != HD_OK) return fail(st);
    scoped_stream ss;
    if (cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking) != cudaSuccess)
        return fail(hd_fail(HD_ERR_CUDA, "hd_ctx_create: stream creation failed"));
    st = hd_item_memory_build(c, ss.s);
    if (st != HD_OK) return fail(st);
    cudaError_t e = cudaStreamSynchronize(ss.s);
    if (e != cudaSuccess) return fail(hd_cuda_fail(e, "hd_ctx_create"));
    *out = c;
    return HD_OK;
}

void hd_ctx_destroy(hd_ctx *ctx) { ctx_release(ctx); }

hd_status hd_ctx_item_memory(const hd_ctx *ctx, uint64_t *d_F, uint64_t *d_L, uint32_t *d_rank_F,
                             uint32_t *d_rank_L, hd_stream stream)
{
    HD_CHECK(ctx, "hd_ctx_item_memory: null ctx");
    hd_status st = check_device(ctx->device);
    if (st != HD_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const auto D2D = cudaMemcpyDeviceToDevice;
    if (d_F) HD_CUDA_TRY(cudaMemcpyAsync(d_F, ctx->F, (size_t)ctx->p.n_bins * ctx->W * 8, D2D, s));
    if (d_L) HD_CUDA_TRY(cudaMemcpyAsync(d_L, ctx->L, (size_t)ctx->p.n_levels * ctx->W * 8, D2D, s));
    if (d_rank_F) HD_CUDA_TRY(cudaMemcpyAsync(d_rank_F, ctx->rank_F, (size_t)ctx->p.dim * 4, D2D, s));
    if (d_rank_L) HD_CUDA_TRY(cudaMemcpyAsync(d_rank_L, ctx->rank_L, (size_t)ctx->p.dim * 4, D2D, s));
    return HD_OK;
}

hd_status hd_random_words(uint64_t seed, uint32_t stream_id, uint32_t n, uint32_t *d_out, hd_stream stream)
{
    if (n == 0) return HD_OK;
    HD_CHECK(d_out, "hd_random_words: null output");
    HD_CHECK(n <= 0xFFFFFFFCu, "hd_random_words: n too large");
    hd_random_words_launch(seed, stream_id, n, d_out, (cudaStream_t)stream);
    HD_CUDA_TRY(cudaGetLastError());
    return HD_OK;
}

hd_status hd_measure_peak(hd_peak_kind kind, uint32_t launches, hd_peak_result *out)
{
    HD_CHECK(out, "hd_measure_peak: null result");
    HD_CHECK(launches >= 1 && launches <= 1000, "hd_measure_peak: launches must be in [1, 1000]");
    switch (kind) {
    case HD_PEAK_TC_FP4: return hd_peak_mma_run(HD_FORM_TC_FP4, launches, out);
    case HD_PEAK_TC_FP8: return hd_peak_mma_run(HD_FORM_TC_FP8, launches, out);
    case HD_PEAK_TC_BF16: return hd_peak_mma_run(HD_FORM_TC_BF16, launches, out);
    case HD_PEAK_POPC: return hd_peak_alu_run(true, launches, out);
    case HD_PEAK_LOP3: return hd_peak_alu_run(false, launches, out);
    case HD_PEAK_TC_MXF4: return hd_peak_mma_run(HD_FORM_TC_MXF4, launches, out);
    }
    return hd_fail(HD_ERR_INVALID_ARG, "hd_measure_peak: unknown kind");
}

hd_status hd_ctx_status(hd_ctx *ctx)
{
    HD_CHECK(ctx, "hd_ctx_status: null ctx");
    return status_take(ctx->status, "hd_ctx");
}

hd_status hd_preprocess(hd_ctx *ctx, const hd_preprocess_params *pp, const uint32_t *d_raw_off,
                        const double *d_raw_mz, const double *d_raw_int, uint32_t n_spectra,
                        uint32_t *d_out_off, uint32_t *d_out_bins, uint8_t *d_out_levels,
                        hd_stream stream)
{
    HD_CHECK(ctx && pp, "hd_preprocess: null argument");
    HD_CHECK(std::isfinite(pp->mz_min) && std::isfinite(pp->mz_max) && pp->mz_min <= pp->mz_max,
             "hd_preprocess: mz_min/mz_max must be finite, mz_min <= mz_max");
    HD_CHECK(std::isfinite(pp->bin_width) && pp->bin_width > 0.0, "hd_preprocess: bin_width must be > 0");
    HD_CHECK(std::isfinite(pp->min_rel_intensity) && pp->min_rel_intensity >= 0.0,
             "hd_preprocess: min_rel_intensity must be finite and >= 0");
    HD_CHECK(pp->n_bins >= 1, "hd_preprocess: n_bins must be >= 1");
    HD_CHECK(pp->max_peaks >= 1 && pp->max_peaks <= 1023, "hd_preprocess: max_peaks must be in [1, 1023]");
    HD_CHECK(pp->n_levels >= 2 && pp->n_levels <= 256, "hd_preprocess: n_levels must be in [2, 256]");
    HD_CHECK(d_out_off, "hd_preprocess: null output offsets");
    HD_CHECK(n_spectra == 0 || (d_raw_off && d_raw_mz && d_raw_int && d_out_bins && d_out_levels),
             "hd_preprocess: null buffer");
    hd_status st = check_device(ctx->device);
    if (st != HD_OK) return st;
    return hd_preprocess_launch(*pp, d_raw_off, d_raw_mz, d_raw_int, n_spectra, d_out_off, d_out_bins,
                                d_out_levels, ctx->status.dev, (cudaStream_t)stream);
}

hd_status hd_encode(hd_ctx *ctx, const uint32_t *d_offsets, const uint32_t *d_bins,
                    const uint8_t *d_levels, uint32_t n_spectra, uint64_t *d_out_hv, hd_stream stream)
{
    HD_CHECK(ctx, "hd_encode: null ctx");
    if (n_spectra == 0) return HD_OK;
    HD_CHECK(d_offsets && d_bins && d_levels && d_out_hv, "hd_encode: null buffer");
    HD_CHECK(aligned16(d_out_hv), "hd_encode: d_out_hv must be 16-byte aligned");
    hd_status st = check_device(ctx->device);
    if (st != HD_OK) return st;
    hd_encode_launch(ctx, d_offsets, d_bins, d_levels, n_spectra, d_out_hv, (cudaStream_t)stream);
    HD_CUDA_TRY(cudaGetLastError());
    return HD_OK;
}


hd_status hd_build_library(hd_ctx *ctx, const uint64_t *d_hv, const double *d_prec_mz,
                           const uint8_t *d_charge, uint32_t n_refs, hd_library **out)
{
    HD_CHECK(ctx && out, "hd_build_library: null argument");
    *out = nullptr;
    HD_CHECK(n_refs == 0 || (d_hv && d_prec_mz && d_charge), "hd_build_library: null buffer");
    hd_status st = check_device(ctx->device);
    if (st != HD_OK) return st;
    return build_rows(ctx, d_hv, 1, d_prec_mz, d_charge, n_refs, out, "hd_build_library");
}

hd_status hd_encode_multibit(hd_ctx *ctx, const uint32_t *d_offsets, const uint32_t *d_bins,
                             const uint8_t *d_levels, uint32_t n_spectra, uint32_t bits, int8_t *d_out,
                             hd_stream stream)
{
    HD_CHECK(ctx, "hd_encode_multibit: null ctx");
    HD_CHECK(bits >= 2 && bits <= 5, "hd_encode_multibit: bits must be in [2, 5]");
    if (n_spectra == 0) return HD_OK;
    HD_CHECK(d_offsets && d_bins && d_levels && d_out, "hd_encode_multibit: null buffer");
    HD_CHECK(aligned16(d_out), "hd_encode_multibit: d_out must be 16-byte aligned");
    hd_status st = check_device(ctx->device);
    if (st != HD_OK) return st;
    hd_encode_mb_launch(ctx, d_offsets, d_bins, d_levels, n_spectra, bits, d_out, (cudaStream_t)stream);
    HD_CUDA_TRY(cudaGetLastError());
    return HD_OK;
}

hd_status hd_build_library_multibit(hd_ctx *ctx, const int8_t *d_comp, const double *d_prec_mz,
                                    const uint8_t *d_charge, uint32_t n_refs, uint32_t bits, hd_library **out)
{
    HD_CHECK(ctx && out, "hd_build_library_multibit: null argument");
    *out = nullptr;
    HD_CHECK(bits >= 2 && bits <= 5, "hd_build_library_multibit: bits must be in [2, 5]");
    HD_CHECK(n_refs == 0 || (d_comp && d_prec_mz && d_charge), "hd_build_library_multibit: null buffer");
    HD_CHECK(aligned16(d_comp), "hd_build_library_multibit: d_comp must be 16-byte aligned");
    hd_status st = check_device(ctx->device);
    if (st != HD_OK) return st;
    return build_rows(ctx, reinterpret_cast<const uint64_t *>(d_comp), bits, d_prec_mz, d_charge, n_refs, out,
                      "hd_build_library_multibit");
}

hd_status hd_library_component_bits(const hd_library *lib, uint32_t *bits)
{
    HD_CHECK(lib && bits, "hd_library_component_bits: null argument");
    *bits = lib->bits;
    return HD_OK;
}

hd_status hd_search_dot(const hd_library *lib, const int8_t *d_q_comp, const double *d_q_mz,
                        const uint8_t *d_q_charge, uint32_t n_q, double tol, hd_tol_unit unit, uint32_t k,
                        hd_search_form form, uint32_t *d_out_idx, int32_t *d_out_score, hd_stream stream)
{
    HD_CHECK(lib, "hd_search_dot: null library");
    HD_CHECK(lib->bits > 1, "hd_search_dot: binary library (use hd_search_open)");
    HD_CHECK(k >= 1 && k <= 16, "hd_search_dot: k must be in [1, 16]");
    HD_CHECK(tol_ok(tol), "hd_search_dot: tol must be finite and >= 0");
    HD_CHECK(unit_ok(unit), "hd_search_dot: bad unit");
    hd_status st = hd_dot_check(lib, &form, "hd_search_dot");
    if (st != HD_OK) return st;
    if (n_q == 0) return HD_OK;
    HD_CHECK(d_q_comp && d_q_mz && d_q_charge && d_out_idx && d_out_score, "hd_search_dot: null buffer");
    HD_CHECK(aligned16(d_q_comp), "hd_search_dot: d_q_comp must be 16-byte aligned");
    st = check_device(lib->device);
    if (st != HD_OK) return st;
    return hd_search_dot_dispatch(lib, form, d_q_comp, d_q_mz, d_q_charge, n_q, hd_single_window(tol, unit), k,
                                  d_out_idx, d_out_score, (cudaStream_t)stream);
}

hd_status hd_search_dot_multi(const hd_library *lib, const int8_t *d_q_comp, const double *d_q_mz,
                              const uint8_t *d_q_charge, const uint8_t *d_q_class, uint32_t n_q,
                              const hd_window *windows, uint32_t n_windows, uint32_t k, hd_search_form form,
                              uint32_t *d_out_idx, int32_t *d_out_score, hd_stream stream)
{
    HD_CHECK(lib, "hd_search_dot_multi: null library");
    HD_CHECK(lib->bits > 1, "hd_search_dot_multi: binary library (use hd_search_open_multi)");
    HD_CHECK(k >= 1 && k <= 16, "hd_search_dot_multi: k must be in [1, 16]");
    hd_qwin win;
    hd_status st = hd_make_qwin(d_q_class, windows, n_windows, &win);
    if (st != HD_OK) return st;
    st = hd_dot_check(lib, &form, "hd_search_dot_multi");
    if (st != HD_OK) return st;
    if (n_q == 0) return HD_OK;
    HD_CHECK(d_q_comp && d_q_mz && d_q_charge && d_out_idx && d_out_score, "hd_search_dot_multi: null buffer");
    HD_CHECK(aligned16(d_q_comp), "hd_search_dot_multi: d_q_comp must be 16-byte aligned");
    st = check_device(lib->device);
    if (st != HD_OK) return st;
    return hd_search_dot_dispatch(lib, form, d_q_comp, d_q_mz, d_q_charge, n_q, win, k, d_out_idx, d_out_score,
                                  (cudaStream_t)stream);
}

void hd_library_free(hd_library *lib) { lib_release(lib); }

hd_status hd_library_info(const hd_library *lib, uint32_t *n_refs, uint32_t *dim)
{
    HD_CHECK(lib, "hd_library_info: null library");
    if (n_refs) *n_refs = lib->n;
    if (dim) *dim = lib->dim;
    return HD_OK;
}

hd_status hd_library_export(const hd_library *lib, uint64_t *d_hv, double *d_mz, uint8_t *d_charge,
                            uint32_t *d_orig, hd_stream stream)
{
    HD_CHECK(lib, "hd_library_export: null library");
    HD_CHECK(hd_lib_binary(lib), "hd_library_export: multi-bit library (binary HVs only)");
    hd_status st = check_device(lib->device);
    if (st != HD_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const auto D2D = cudaMemcpyDeviceToDevice;
    if (lib->n == 0) return HD_OK;
    if (d_hv) HD_CUDA_TRY(cudaMemcpyAsync(d_hv, lib->hv, (size_t)lib->n * lib->W * 8, D2D, s));
    if (d_mz) HD_CUDA_TRY(cudaMemcpyAsync(d_mz, lib->mz, (size_t)lib->n * 8, D2D, s));
    if (d_charge) HD_CUDA_TRY(cudaMemcpyAsync(d_charge, lib->charge, lib->n, D2D, s));
    if (d_orig) HD_CUDA_TRY(cudaMemcpyAsync(d_orig, lib->orig, (size_t)lib->n * 4, D2D, s));
    return HD_OK;
}

namespace {

const char LIB_MAGIC[8] = {'H', 'D', 'L', 'I', 'B', '0', '0', '1'};

struct lib_header {
    char magic[8];
    uint32_t dim, n_levels, n_bins, alpha;
    uint64_t seed;
    uint32_t position_mode, encoder;
    uint32_t n, flags;
};

struct fnv64 {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n)
    {
        const uint8_t *b = static_cast<const uint8_t *>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    }
};

struct file_closer {
    FILE *f = nullptr;
    ~file_closer()
    {
        if (f) fclose(f);
    }
};

}  // namespace

hd_status hd_library_save(const hd_library *lib, const hd_ctx *ctx, const char *path)
{
    HD_CHECK(lib && ctx && path, "hd_library_save: null argument");
    HD_CHECK(ctx->p.dim == lib->dim, "hd_library_save: ctx and library dims differ");
    hd_status st = check_device(lib->device);
    if (st != HD_OK) return st;
    // binary rows: D/64 words; multi-bit rows: D int8 components (D/8 words)
    const size_t n = lib->n, W = hd_lib_binary(lib) ? lib->W : lib->dim / 8;
    std::vector<uint64_t> hv(n * W);
    std::vector<double> mz(n);
    std::vector<uint8_t> z(n), dec(lib->decoy ? n : 0);
    std::vector<uint32_t> orig(n);
    if (n) {
        HD_CUDA_TRY(cudaMemcpy(hv.data(), hd_lib_binary(lib) ? (const void *)lib->hv : (const void *)lib->comp, n * W * 8,
                               cudaMemcpyDeviceToHost));
        HD_CUDA_TRY(cudaMemcpy(mz.data(), lib->mz, n * 8, cudaMemcpyDeviceToHost));
        HD_CUDA_TRY(cudaMemcpy(z.data(), lib->charge, n, cudaMemcpyDeviceToHost));
        HD_CUDA_TRY(cudaMemcpy(orig.data(), lib->orig, n * 4, cudaMemcpyDeviceToHost));
        if (lib->decoy) HD_CUDA_TRY(cudaMemcpy(dec.data(), lib->decoy, n, cudaMemcpyDeviceToHost));
    }
    lib_header h{};
    std::memcpy(h.magic, LIB_MAGIC, 8);
    h.dim = ctx->p.dim;
    h.n_levels = ctx->p.n_levels;
    h.n_bins = ctx->p.n_bins;
    h.alpha = ctx->p.alpha;
    h.seed = ctx->p.seed;
    h.position_mode = ctx->p.position_mode;
    h.encoder = ctx->p.encoder;
    h.n = lib->n;
    h.flags = (lib->decoy ? 1u : 0u) | (hd_lib_binary(lib) ? 0u : (lib->bits << 8));
    file_closer fc;
    fc.f = std::fopen(path, "wb");
    if (!fc.f) return hd_fail(HD_ERR_INVALID_ARG, std::string("hd_library_save: cannot open ") + path);
    fnv64 hash;
    bool ok = true;
    auto put = [&](const void *p, size_t bytes) {
        if (!ok || bytes == 0) return;
        hash.add(p, bytes);
        ok = std::fwrite(p, 1, bytes, fc.f) == bytes;
    };
    put(&h, sizeof(h));
    put(hv.data(), hv.size() * 8);
    put(mz.data(), mz.size() * 8);
    put(z.data(), z.size());
    put(orig.data(), orig.size() * 4);
    put(dec.data(), dec.size());
    const uint64_t digest = hash.h;
    if (ok) ok = std::fwrite(&digest, 1, 8, fc.f) == 8;
    if (ok) ok = std::fclose(fc.f) == 0;
    fc.f = nullptr;
    if (!ok) return hd_fail(HD_ERR_INVALID_ARG, std::string("hd_library_save: write failed: ") + path);
    return HD_OK;
}

hd_status hd_library_load(hd_ctx *ctx, const char *path, hd_library **out)
{
    HD_CHECK(ctx && path && out, "hd_library_load: null argument");
    *out = nullptr;
    hd_status st = check_device(ctx->device);
    if (st != HD_OK) return st;
    file_closer fc;
    fc.f = std::fopen(path, "rb");
    if (!fc.f) return hd_fail(HD_ERR_INVALID_ARG, std::string("hd_library_load: cannot open ") + path);
    fnv64 hash;
    bool ok = true;
    auto get = [&](void *p, size_t bytes) {
        if (!ok || bytes == 0) return;
        ok = std::fread(p, 1, bytes, fc.f) == bytes;
        if (ok) hash.add(p, bytes);
    };
    lib_header h{};
    get(&h, sizeof(h));
    if (!ok || std::memcmp(h.magic, LIB_MAGIC, 8) != 0)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_library_load: not a library file");
    if (h.dim != ctx->p.dim || h.n_levels != ctx->p.n_levels || h.n_bins != ctx->p.n_bins ||
        h.alpha != ctx->p.alpha || h.seed != ctx->p.seed || h.position_mode != ctx->p.position_mode ||
        h.encoder != ctx->p.encoder)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_library_load: the file was encoded with other item-memory parameters");
    const uint32_t bits = (h.flags >> 8) & 0xFFu;   // 0: binary rows
    if ((h.flags & ~0xFF01u) != 0 || bits == 1 || bits > 5)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_library_load: unknown flags");
    const size_t n = h.n, W = bits ? ctx->p.dim / 8 : ctx->W;
    std::vector<uint64_t> hv(n * W);
    std::vector<double> mz(n);
    std::vector<uint8_t> z(n), dec((h.flags & 1u) ? n : 0);
    std::vector<uint32_t> orig(n);
    get(hv.data(), hv.size() * 8);
    get(mz.data(), mz.size() * 8);
    get(z.data(), z.size());
    get(orig.data(), orig.size() * 4);
    get(dec.data(), dec.size());
    uint64_t digest = 0;
    if (ok) ok = std::fread(&digest, 1, 8, fc.f) == 8;
    if (!ok || digest != hash.h) return hd_fail(HD_ERR_INVALID_ARG, "hd_library_load: truncated or corrupted file");
    std::vector<uint8_t> seen(n, 0);
    for (size_t i = 0; i < n; ++i) {
        const bool order = i == 0 || z[i] > z[i - 1] || (z[i] == z[i - 1] && mz[i] >= mz[i - 1]);
        if (!order || !std::isfinite(mz[i]) || orig[i] >= n || seen[orig[i]])
            return hd_fail(HD_ERR_INVALID_ARG, "hd_library_load: rows out of order or bad index");
        seen[orig[i]] = 1;
    }
    hd_library *lib = new hd_library;
    lib->n = h.n;
    lib->dim = ctx->p.dim;
    lib->W = ctx->W;
    lib->bits = bits ? bits : 1u;
    lib->device = ctx->device;
    lib->num_sms = ctx->num_sms;
    auto fail = [&](hd_status s) {
        lib_release(lib);
        return s;
    };
    const size_t n1 = n ? n : 1;
    uint64_t *rows = nullptr;
    if (cudaMalloc(&rows, n1 * W * 8) == cudaSuccess) {
        if (bits) lib->comp = reinterpret_cast<int8_t *>(rows);
        else lib->hv = rows;
    }
    if (!rows || cudaMalloc(&lib->mz, n1 * 8) != cudaSuccess ||
        cudaMalloc(&lib->charge, n1) != cudaSuccess || cudaMalloc(&lib->orig, n1 * 4) != cudaSuccess ||
        cudaMalloc(&lib->charge_start, 257 * 4) != cudaSuccess ||
        (!dec.empty() && cudaMalloc(&lib->decoy, n) != cudaSuccess)) {
        cudaGetLastError();
        return fail(hd_fail(HD_ERR_OOM, "hd_library_load: allocation failed"));
    }
    st = status_alloc(lib->status);
    if (st != HD_OK) return fail(st);
    cudaError_t e = cudaSuccess;
    if (n) {
        e = cudaMemcpy(rows, hv.data(), n * W * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(lib->mz, mz.data(), n * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(lib->charge, z.data(), n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(lib->orig, orig.data(), n * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !dec.empty()) e = cudaMemcpy(lib->decoy, dec.data(), n, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return fail(hd_cuda_fail(e, "hd_library_load: upload"));
    hd_count_launches(1), k_charge_start<<<1, 288>>>(lib->charge, h.n, lib->charge_start);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(lib->charge_start_h, lib->charge_start, 257 * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(hd_cuda_fail(e, "hd_library_load"));
    if (bits) {   // multi-bit rows: the default tensor-core copy, which also checks the component range
        st = hd_library_expand(lib, bits <= 3 ? HD_FORM_TC_FP4 : HD_FORM_TC_FP8, nullptr);
        if (st != HD_OK) return fail(st);
        e = cudaStreamSynchronize(nullptr);
        if (e != cudaSuccess) return fail(hd_cuda_fail(e, "hd_library_load"));
        st = status_take(lib->status, "hd_library_load");
        if (st != HD_OK) return fail(hd_fail(st, "hd_library_load: components must lie in [-m, m]"));
    }
    *out = lib;
    return HD_OK;
}

hd_status hd_library_status(hd_library *lib)
{
    HD_CHECK(lib, "hd_library_status: null library");
    return status_take(lib->status, "hd_library");
}

hd_status hd_library_prepare(hd_library *lib, hd_search_form form)
{
    HD_CHECK(lib, "hd_library_prepare: null library");
    HD_CHECK(form == HD_FORM_POPC || hd_is_tc_form(form), "hd_library_prepare: unknown form");
    HD_CHECK(form != HD_FORM_TC_MXF4 || lib->dim % 256 == 0,
             "hd_library_prepare: the kind::mxf4 form needs D to be a multiple of 256");
    hd_status st = check_device(lib->device);
    if (st != HD_OK || (form == HD_FORM_POPC && hd_lib_binary(lib))) return st;   // binary rows need no copy
    scoped_stream ss;
    if (cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking) != cudaSuccess)
        return hd_fail(HD_ERR_CUDA, "hd_library_prepare: stream creation failed");
    st = form == HD_FORM_POPC ? hd_library_planes(lib, ss.s) : hd_library_expand(lib, form, ss.s);
    if (st != HD_OK) return st;
    HD_CUDA_TRY(cudaStreamSynchronize(ss.s));
    return HD_OK;
}

hd_status hd_library_set_wait_limit(hd_library *lib, uint64_t ns)
{
    HD_CHECK(lib, "hd_library_set_wait_limit: null library");
    HD_CHECK(ns == 0 || ns >= 1000000ull, "hd_library_set_wait_limit: limit must be 0 or >= 1 ms");
    lib->wait_ns = ns;
    return HD_OK;
}

hd_status hd_library_inject_stall(hd_library *lib, uint32_t n_searches)
{
    HD_CHECK(lib, "hd_library_inject_stall: null library");
    __atomic_store_n(&lib->inject_stalls, n_searches, __ATOMIC_SEQ_CST);
    return HD_OK;
}

hd_status hd_library_set_schedule(hd_library *lib, uint32_t tile_group, uint32_t super_group, uint32_t cluster,
                                  uint32_t cta_group)
{
    HD_CHECK(lib, "hd_library_set_schedule: null library");
    HD_CHECK(tile_group <= 4096 && super_group <= 4096, "hd_library_set_schedule: values must be <= 4096");
    HD_CHECK(cluster <= 2, "hd_library_set_schedule: cluster must be 0, 1 or 2");
    HD_CHECK(cta_group <= 2, "hd_library_set_schedule: cta_group must be 0, 1 or 2");
    HD_CHECK(cluster == 0 || cta_group == 0 || cluster == cta_group,
             "hd_library_set_schedule: the cluster is the SM pair (2, 2) or one SM (1, 1)");
    const uint32_t cg = cta_group ? cta_group : (cluster == 1 ? 1u : 2u);
    lib->mma_tuning.tile_group = tile_group;
    lib->mma_tuning.super_group = super_group;
    lib->mma_tuning.cluster = cg;
    lib->mma_tuning.cta_group = cg;
    return HD_OK;
}

hd_status hd_library_set_stage_tiles(hd_library *lib, uint32_t tiles_per_stage)
{
    HD_CHECK(lib, "hd_library_set_stage_tiles: null library");
    HD_CHECK(tiles_per_stage <= 2, "hd_library_set_stage_tiles: tiles_per_stage must be 0, 1 or 2");
    lib->mma_tuning.tiles_per_stage = tiles_per_stage;
    return HD_OK;
}

hd_status hd_query_windows(const hd_library *lib, const double *d_q_mz, const uint8_t *d_q_charge,
                           uint32_t n_q, double tol, hd_tol_unit unit, uint32_t *d_lo, uint32_t *d_hi,
                           hd_stream stream)
{
    HD_CHECK(lib, "hd_query_windows: null library");
    HD_CHECK(tol_ok(tol), "hd_query_windows: tol must be finite and >= 0");
    HD_CHECK(unit_ok(unit), "hd_query_windows: bad unit");
    if (n_q == 0) return HD_OK;
    HD_CHECK(d_q_mz && d_q_charge && d_lo && d_hi, "hd_query_windows: null buffer");
    hd_status st = check_device(lib->device);
    if (st != HD_OK) return st;
    hd_windows_launch(lib, d_q_mz, d_q_charge, nullptr, n_q, hd_single_window(tol, unit), d_lo, d_hi,
                      (cudaStream_t)stream);
    HD_CUDA_TRY(cudaGetLastError());
    return HD_OK;
}

hd_status hd_search_open_ex(const hd_library *lib, const uint64_t *d_q_hv, const double *d_q_mz,
                            const uint8_t *d_q_charge, uint32_t n_q, double tol, hd_tol_unit unit,
                            uint32_t k, hd_search_form form, uint32_t *d_out_idx, uint16_t *d_out_dist,
                            hd_stream stream)
{
    HD_CHECK(lib, "hd_search_open: null library");
    HD_CHECK(k >= 1 && k <= 16, "hd_search_open: k must be in [1, 16]");
    HD_CHECK(tol_ok(tol), "hd_search_open: tol must be finite and >= 0");
    HD_CHECK(unit_ok(unit), "hd_search_open: bad unit");
    HD_CHECK(form_ok(form),
             "hd_search_open: unknown form");
    if (n_q == 0) return HD_OK;
    HD_CHECK(d_q_hv && d_q_mz && d_q_charge && d_out_idx && d_out_dist, "hd_search_open: null buffer");
    HD_CHECK(aligned16(d_q_hv), "hd_search_open: d_q_hv must be 16-byte aligned");
    hd_status st = check_device(lib->device);
    if (st != HD_OK) return st;
    return hd_search_dispatch(lib, d_q_hv, d_q_mz, d_q_charge, n_q, hd_single_window(tol, unit), k,
                              form, d_out_idx, d_out_dist, (cudaStream_t)stream);
}

hd_status hd_search_open_multi(const hd_library *lib, const uint64_t *d_q_hv, const double *d_q_mz,
                               const uint8_t *d_q_charge, const uint8_t *d_q_class, uint32_t n_q,
                               const hd_window *windows, uint32_t n_windows, uint32_t k, hd_search_form form,
                               uint32_t *d_out_idx, uint16_t *d_out_dist, hd_stream stream)
{
    HD_CHECK(lib, "hd_search_open_multi: null library");
    HD_CHECK(k >= 1 && k <= 16, "hd_search_open_multi: k must be in [1, 16]");
    HD_CHECK(form_ok(form),
             "hd_search_open_multi: unknown form");
    hd_qwin win;
    hd_status st = hd_make_qwin(d_q_class, windows, n_windows, &win);
    if (st != HD_OK) return st;
    if (n_q == 0) return HD_OK;
    HD_CHECK(d_q_hv && d_q_mz && d_q_charge && d_out_idx && d_out_dist, "hd_search_open_multi: null buffer");
    HD_CHECK(aligned16(d_q_hv), "hd_search_open_multi: d_q_hv must be 16-byte aligned");
    st = check_device(lib->device);
    if (st != HD_OK) return st;
    return hd_search_dispatch(lib, d_q_hv, d_q_mz, d_q_charge, n_q, win, k, form, d_out_idx, d_out_dist,
                              (cudaStream_t)stream);
}

hd_status hd_search_open(const hd_library *lib, const uint64_t *d_q_hv, const double *d_q_mz,
                         const uint8_t *d_q_charge, uint32_t n_q, double tol, hd_tol_unit unit, uint32_t k,
                         uint32_t *d_out_idx, uint16_t *d_out_dist, hd_stream stream)
{
    return hd_search_open_ex(lib, d_q_hv, d_q_mz, d_q_charge, n_q, tol, unit, k, HD_FORM_AUTO, d_out_idx,
                             d_out_dist, stream);
}

hd_status hd_search_host(hd_ctx *ctx, const hd_library *lib, const uint32_t *h_offsets, const uint32_t *h_bins,
                         const uint8_t *h_levels, const double *h_q_mz, const uint8_t *h_q_charge,
                         uint32_t n_q, double tol, hd_tol_unit unit, uint32_t k, uint32_t *h_out_idx,
                         uint16_t *h_out_dist, hd_stream stream)
{
    HD_CHECK(ctx && lib, "hd_search_host: null ctx or library");
    HD_CHECK(ctx->p.dim == lib->dim, "hd_search_host: ctx and library dims differ");
    HD_CHECK(k >= 1 && k <= 16, "hd_search_host: k must be in [1, 16]");
    HD_CHECK(tol_ok(tol), "hd_search_host: tol must be finite and >= 0");
    if (n_q == 0) return HD_OK;
    HD_CHECK(h_offsets && h_q_mz && h_q_charge && h_out_idx && h_out_dist, "hd_search_host: null buffer");
    const uint32_t nnz = h_offsets[n_q];
    HD_CHECK(nnz == 0 || (h_bins && h_levels), "hd_search_host: null CSR buffer");
    hd_status st = check_device(ctx->device);
    if (st != HD_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    hd_arena plan;
    auto carve = [&](hd_arena &ar, uint32_t **off, uint32_t **bins, uint8_t **lv, double **mz,
                     uint8_t **z, uint64_t **hv, uint32_t **oi, uint16_t **od) {
        *off = ar.take<uint32_t>(n_q + 1);
        *bins = ar.take<uint32_t>(nnz ? nnz : 1);
        *lv = ar.take<uint8_t>(nnz ? nnz : 1);
        *mz = ar.take<double>(n_q);
        *z = ar.take<uint8_t>(n_q);
        *hv = ar.take<uint64_t>((size_t)n_q * ctx->W);
        *oi = ar.take<uint32_t>((size_t)n_q * k);
        *od = ar.take<uint16_t>((size_t)n_q * k);
    };
    uint32_t *off, *bins, *oi;
    uint8_t *lv, *z;
    double *mz;
    uint64_t *hv;
    uint16_t *od;
    carve(plan, &off, &bins, &lv, &mz, &z, &hv, &oi, &od);
    hd_arena ar;
    if (cudaMallocAsync((void **)&ar.base, plan.used, s) != cudaSuccess) {
        cudaGetLastError();
        return hd_fail(HD_ERR_OOM, "hd_search_host: device buffer allocation failed");
    }
    carve(ar, &off, &bins, &lv, &mz, &z, &hv, &oi, &od);
    const auto H2D = cudaMemcpyHostToDevice, D2H = cudaMemcpyDeviceToHost;
    cudaError_t e = cudaMemcpyAsync(off, h_offsets, (size_t)(n_q + 1) * 4, H2D, s);
    if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(bins, h_bins, (size_t)nnz * 4, H2D, s);
    if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(lv, h_levels, nnz, H2D, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mz, h_q_mz, (size_t)n_q * 8, H2D, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(z, h_q_charge, n_q, H2D, s);
    if (e == cudaSuccess) {
        hd_encode_launch(ctx, off, bins, lv, n_q, hv, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        st = hd_search_dispatch(lib, hv, mz, z, n_q, hd_single_window(tol, unit), k, HD_FORM_AUTO,
                                oi, od, s);
        if (st != HD_OK) {
            cudaFreeAsync(ar.base, s);
            cudaStreamSynchronize(s);
            return st;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_out_idx, oi, (size_t)n_q * k * 4, D2H, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_out_dist, od, (size_t)n_q * k * 2, D2H, s);
    cudaFreeAsync(ar.base, s);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return hd_cuda_fail(e, "hd_search_host");
    if (e2 != cudaSuccess) return hd_cuda_fail(e2, "hd_search_host");
    st = status_take(ctx->status, "hd_search_host (encode)");
    if (st != HD_OK) return st;
    return status_take(const_cast<hd_library *>(lib)->status, "hd_search_host (search)");
}

}  // extern "C"
