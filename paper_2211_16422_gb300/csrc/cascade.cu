// cascade.cu -- cascade search with target-decoy FDR filtering (Section 3.4:
// narrow precursor window, FDR filter, wider window for the spectra still
// unidentified; the FDR filter is the target-decoy strategy of Section 2.1).
//
// Per level, all on the device: gather the queries still unidentified, run
// the top-1 search, histogram the scores of target and decoy SSMs, turn the
// two histograms into a q-value table over the score range, apply it to
// every SSM, and compact the queries left for the next level.  Counting over
// the score range replaces a sort of the SSMs: the FDR at threshold s needs
// only how many target and decoy SSMs score >= s.  Binary HVs score D - dist
// (0..D); multi-bit components (Section 4.3) score their dot product S in
// [-D m^2, D m^2], histogrammed at S + D m^2.
#include <cmath>
#include <limits>
#include <string>

#include "hd_internal.cuh"

void hd_exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint32_t n, hd_arena &arena, cudaStream_t s);

namespace {

constexpr uint32_t NONE_IDX = 0xFFFFFFFFu;
constexpr int QT_THREADS = 1024;

__device__ __forceinline__ double quiet_nan() { return __longlong_as_double(0x7FF8000000000000ll); }

__global__ void k_iota(uint32_t *__restrict__ a, uint32_t n)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = i;
}

template <class T>
__global__ void k_fill(T *__restrict__ a, uint32_t n, T v)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// Rows act[j] of the query set -> compact buffers, one warp per row
// (row_bytes a multiple of 16).
__global__ void k_gather_active(const uint8_t *__restrict__ rows, const double *__restrict__ mz,
                                const uint8_t *__restrict__ z, const uint32_t *__restrict__ act, uint32_t n,
                                uint32_t row_bytes, uint8_t *__restrict__ o_rows, double *__restrict__ o_mz,
                                uint8_t *__restrict__ o_z)
{
    const uint32_t r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const uint32_t lane = threadIdx.x & 31;
    if (r >= n) return;
    const uint32_t src = act[r];
    const uint4 *s4 = reinterpret_cast<const uint4 *>(rows + (size_t)src * row_bytes);
    uint4 *d4 = reinterpret_cast<uint4 *>(o_rows + (size_t)r * row_bytes);
    for (uint32_t w = lane; w < row_bytes / 16; w += 32) d4[w] = s4[w];
    if (lane == 0) {
        o_mz[r] = mz[src];
        o_z[r] = z[src];
    }
}

// Histogram slot of an SSM's score: D - dist for a Hamming distance (u16,
// 0..D), S + bias for a dot-product score (i32, |S| <= bias).  False for a
// query without a candidate (or a value outside the range).
__device__ __forceinline__ bool score_slot(uint16_t d, uint32_t D, uint32_t, uint32_t &slot)
{
    slot = D - d;
    return d <= D;
}
__device__ __forceinline__ bool score_slot(int32_t sc, uint32_t, uint32_t bias, uint32_t &slot)
{
    slot = (uint32_t)((int64_t)sc + bias);
    return sc != INT32_MIN && sc >= -(int64_t)bias && sc <= (int64_t)bias;
}

// Score histograms of one level's SSMs: hist[0..nb) targets, hist[nb..2nb) decoys.
template <class T>
__global__ void k_fdr_hist(const uint32_t *__restrict__ idx, const T *__restrict__ sc, uint32_t n,
                           const uint8_t *__restrict__ decoy, uint32_t D, uint32_t bias, uint32_t nb,
                           uint32_t *__restrict__ hist)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t r = idx[j];
    uint32_t slot;
    if (r == NONE_IDX || !score_slot(sc[j], D, bias, slot)) return;
    atomicAdd(&hist[(decoy[r] ? nb : 0) + slot], 1u);
}

// q-value table over scores 0..nb-1 (one CTA): with T(s), Dc(s) the target
// and decoy SSMs scoring >= s, FDR(s) = Dc(s) / max(1, T(s)) and
// q(s) = min over s' <= s of FDR(s').  A score no SSM has repeats the FDR of
// the next higher score that occurs, so taking the minimum over every score
// equals taking it over the thresholds the SSMs define.
__global__ void __launch_bounds__(QT_THREADS) k_fdr_qtable(const uint32_t *__restrict__ hist, uint32_t nb,
                                                           double *__restrict__ qtab)
{
    __shared__ uint32_t st[QT_THREADS], sd[QT_THREADS];
    __shared__ double sm[QT_THREADS];
    const uint32_t t = threadIdx.x;
    const uint32_t seg = (nb + QT_THREADS - 1) / QT_THREADS;
    const uint32_t b0 = min(nb, t * seg), b1 = min(nb, b0 + seg);
    uint32_t ct = 0, cd = 0;
    for (uint32_t s = b0; s < b1; ++s) {
        ct += hist[s];
        cd += hist[nb + s];
    }
    st[t] = ct;
    sd[t] = cd;
    __syncthreads();
    // inclusive suffix sums over the threads' segments
    for (uint32_t off = 1; off < QT_THREADS; off <<= 1) {
        const uint32_t at = t + off < QT_THREADS ? st[t + off] : 0u;
        const uint32_t ad = t + off < QT_THREADS ? sd[t + off] : 0u;
        __syncthreads();
        st[t] += at;
        sd[t] += ad;
        __syncthreads();
    }
    uint32_t T = t + 1 < QT_THREADS ? st[t + 1] : 0u;   // SSMs scoring above this segment
    uint32_t Dc = t + 1 < QT_THREADS ? sd[t + 1] : 0u;
    double mseg = INFINITY;
    for (uint32_t s = b1; s-- > b0;) {
        T += hist[s];
        Dc += hist[nb + s];
        const double f = (double)Dc / (double)(T ? T : 1u);
        qtab[s] = f;
        mseg = fmin(mseg, f);
    }
    sm[t] = mseg;
    __syncthreads();
    // inclusive prefix minimum over the segments (ascending scores)
    for (uint32_t off = 1; off < QT_THREADS; off <<= 1) {
        const double o = t >= off ? sm[t - off] : INFINITY;
        __syncthreads();
        sm[t] = fmin(sm[t], o);
        __syncthreads();
    }
    double run = t > 0 ? sm[t - 1] : INFINITY;
    for (uint32_t s = b0; s < b1; ++s) {
        run = fmin(run, qtab[s]);
        qtab[s] = run;
    }
}

// One level's verdicts: outputs of query act[j], and keep[j] = 1 when it is
// still unidentified.
template <class T>
__global__ void k_fdr_apply(const uint32_t *__restrict__ act, uint32_t n, const uint32_t *__restrict__ idx,
                            const T *__restrict__ sc, const uint8_t *__restrict__ decoy,
                            const double *__restrict__ qtab, uint32_t D, uint32_t bias, double fdr, uint8_t level,
                            uint32_t *__restrict__ out_idx, T *__restrict__ out_sc, double *__restrict__ out_q,
                            uint8_t *__restrict__ out_level, uint32_t *__restrict__ keep)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint32_t q = act[j], r = idx[j];
    const T v = sc[j];
    out_idx[q] = r;
    out_sc[q] = v;
    double qv = quiet_nan();
    bool hit = false;
    uint32_t slot;
    if (r != NONE_IDX && score_slot(v, D, bias, slot)) {
        qv = qtab[slot];
        hit = decoy[r] == 0 && qv <= fdr;
    }
    out_q[q] = qv;
    if (hit) out_level[q] = level;
    keep[j] = hit ? 0u : 1u;
}

__global__ void k_compact_active(const uint32_t *__restrict__ act, const uint32_t *__restrict__ keep,
                                 const uint32_t *__restrict__ pos, uint32_t n, uint32_t *__restrict__ next)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n && keep[j]) next[pos[j]] = act[j];
}

// One level's top-1 search of `n` rows (binary HVs, or int8 components for
// the dot-product form).
hd_status level_search(const hd_library *lib, const uint8_t *q, const double *qm, const uint8_t *qz, uint32_t n,
                       const hd_qwin &win, hd_search_form form, uint32_t *idx, uint16_t *dist, cudaStream_t s)
{
    return hd_search_dispatch(lib, reinterpret_cast<const uint64_t *>(q), qm, qz, n, win, 1, form, idx, dist, s);
}
hd_status level_search(const hd_library *lib, const uint8_t *q, const double *qm, const uint8_t *qz, uint32_t n,
                       const hd_qwin &win, hd_search_form form, uint32_t *idx, int32_t *score, cudaStream_t s)
{
    return hd_search_dot_dispatch(lib, form, reinterpret_cast<const int8_t *>(q), qm, qz, n, win, 1, idx, score, s);
}

// The cascade over query rows of row_bytes bytes; SSM scores of type T
// (u16 Hamming distance or i32 dot product, `none` for a query without a
// candidate) histogrammed over nb slots (see score_slot).  Arguments checked
// by the caller.
template <class T>
hd_status cascade_run(const hd_library *lib, const uint8_t *d_q, uint32_t row_bytes, const double *d_q_mz,
                      const uint8_t *d_q_charge, uint32_t n_q, const hd_window *levels, uint32_t n_levels,
                      double fdr, hd_search_form form, uint32_t bias, uint32_t nb, T none, uint32_t *d_out_idx,
                      T *d_out_sc, double *d_out_q, uint8_t *d_out_level, cudaStream_t s, const std::string &name)
{
    const uint32_t D = lib->dim;
    auto carve = [&](hd_arena &ar, uint32_t **act0, uint32_t **act1, uint32_t **keep, uint32_t **pos,
                     uint8_t **rows, double **mz, uint8_t **z, uint32_t **idx, T **sc, uint32_t **hist,
                     double **qtab) {
        *act0 = ar.take<uint32_t>(n_q);
        *act1 = ar.take<uint32_t>(n_q);
        *keep = ar.take<uint32_t>(n_q);
        *pos = ar.take<uint32_t>((size_t)n_q + 1);
        *rows = ar.take<uint8_t>((size_t)n_q * row_bytes);
        *mz = ar.take<double>(n_q);
        *z = ar.take<uint8_t>(n_q);
        *idx = ar.take<uint32_t>(n_q);
        *sc = ar.take<T>(n_q);
        *hist = ar.take<uint32_t>(2 * (size_t)nb);
        *qtab = ar.take<double>(nb);
    };
    uint32_t *act0, *act1, *keep, *pos, *idx, *hist;
    uint8_t *rows, *z;
    double *mz, *qtab;
    T *sc;
    hd_arena plan;
    carve(plan, &act0, &act1, &keep, &pos, &rows, &mz, &z, &idx, &sc, &hist, &qtab);
    hd_exclusive_scan_u32(nullptr, nullptr, n_q, plan, s);   // sizing pass
    hd_arena ar;
    if (cudaMallocAsync((void **)&ar.base, plan.used, s) != cudaSuccess) {
        cudaGetLastError();
        return hd_fail(HD_ERR_OOM, name + ": scratch allocation failed");
    }
    carve(ar, &act0, &act1, &keep, &pos, &rows, &mz, &z, &idx, &sc, &hist, &qtab);
    const size_t scan_mark = ar.used;
    auto fail = [&](hd_status st) {
        cudaFreeAsync(ar.base, s);
        return st;
    };
    const uint32_t g = hd_ceil_div(n_q, 256);
    if (cudaMemsetAsync(d_out_idx, 0xFF, (size_t)n_q * 4, s) != cudaSuccess ||
        cudaMemsetAsync(d_out_level, 0xFF, n_q, s) != cudaSuccess)
        return fail(hd_cuda_fail(cudaGetLastError(), "cascade output init"));
    hd_count_launches(3);
    k_fill<T><<<g, 256, 0, s>>>(d_out_sc, n_q, none);
    k_fill<double><<<g, 256, 0, s>>>(d_out_q, n_q, std::numeric_limits<double>::quiet_NaN());
    k_iota<<<g, 256, 0, s>>>(act0, n_q);

    uint32_t n_act = n_q;
    for (uint32_t l = 0; l < n_levels && n_act > 0; ++l) {
        const uint8_t *qr = d_q;
        const double *qm = d_q_mz;
        const uint8_t *qz = d_q_charge;
        if (l > 0) {   // level 0 searches every query in input order
            hd_count_launches(1), k_gather_active<<<hd_ceil_div(n_act, 8), 256, 0, s>>>(d_q, d_q_mz, d_q_charge, act0,
                                                                                     n_act, row_bytes, rows, mz, z);
            qr = rows;
            qm = mz;
            qz = z;
        }
        const hd_qwin win = hd_single_window(levels[l].tol, levels[l].unit);
        hd_status st = level_search(lib, qr, qm, qz, n_act, win, form, idx, sc, s);
        if (st != HD_OK) return fail(st);
        const uint32_t ga = hd_ceil_div(n_act, 256);
        if (cudaMemsetAsync(hist, 0, 2 * (size_t)nb * 4, s) != cudaSuccess)
            return fail(hd_cuda_fail(cudaGetLastError(), "cascade histogram init"));
        hd_count_launches(1), k_fdr_hist<T><<<ga, 256, 0, s>>>(idx, sc, n_act, lib->decoy, D, bias, nb, hist);
        hd_count_launches(1), k_fdr_qtable<<<1, QT_THREADS, 0, s>>>(hist, nb, qtab);
        hd_count_launches(1), k_fdr_apply<T><<<ga, 256, 0, s>>>(act0, n_act, idx, sc, lib->decoy, qtab, D, bias, fdr,
                                                                (uint8_t)l, d_out_idx, d_out_sc, d_out_q,
                                                                d_out_level, keep);
        if (l + 1 == n_levels) break;
        ar.used = scan_mark;   // the scan's scratch is reused level after level (stream order)
        hd_exclusive_scan_u32(keep, pos, n_act, ar, s);
        hd_count_launches(1), k_compact_active<<<ga, 256, 0, s>>>(act0, keep, pos, n_act, act1);
        uint32_t n_next = 0;
        cudaError_t e = cudaMemcpyAsync(&n_next, pos + n_act, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(hd_cuda_fail(e, "cascade level count"));
        n_act = n_next;
        uint32_t *t = act0;
        act0 = act1;
        act1 = t;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(hd_cuda_fail(e, "cascade"));
    HD_CUDA_TRY(cudaFreeAsync(ar.base, s));
    return HD_OK;
}

// Checks shared by both entry points.
hd_status check_levels(const hd_library *lib, const hd_window *levels, uint32_t n_levels, double fdr,
                       const std::string &name)
{
    if (!levels || n_levels < 1 || n_levels > HD_MAX_WINDOWS) return hd_fail(HD_ERR_INVALID_ARG, name + ": 1 <= n_levels <= 16");
    if (std::isnan(fdr)) return hd_fail(HD_ERR_INVALID_ARG, name + ": fdr is NaN");
    for (uint32_t l = 0; l < n_levels; ++l) {
        hd_qwin w;
        hd_status st = hd_make_qwin(nullptr, &levels[l], 1, &w);
        if (st != HD_OK) return st;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != lib->device)
        return hd_fail(HD_ERR_INVALID_ARG, name + ": library belongs to another device");
    if (lib->n > 0 && !lib->decoy) return hd_fail(HD_ERR_INVALID_ARG, name + ": the library has no decoy flags");
    return HD_OK;
}

}  // namespace

extern "C" {


hd_status hd_library_set_decoys(hd_library *lib, const uint8_t *d_is_decoy)
{
    if (!lib || !d_is_decoy) return hd_fail(HD_ERR_INVALID_ARG, "hd_library_set_decoys: null argument");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != lib->device)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_library_set_decoys: library belongs to another device");
    if (lib->n == 0) return HD_OK;
    if (!lib->decoy) {
        if (cudaMalloc(&lib->decoy, lib->n) != cudaSuccess) {
            cudaGetLastError();
            lib->decoy = nullptr;
            return hd_fail(HD_ERR_OOM, "hd_library_set_decoys: allocation failed");
        }
    }
    HD_CUDA_TRY(cudaMemcpy(lib->decoy, d_is_decoy, lib->n, cudaMemcpyDeviceToDevice));
    return HD_OK;
}

hd_status hd_cascade_search(const hd_library *lib, const uint64_t *d_q_hv, const double *d_q_mz,
                            const uint8_t *d_q_charge, uint32_t n_q, const hd_window *levels, uint32_t n_levels,
                            double fdr, hd_search_form form, uint32_t *d_out_idx, uint16_t *d_out_dist,
                            double *d_out_q, uint8_t *d_out_level, hd_stream stream)
{
    const std::string name = "hd_cascade_search";
    if (!lib) return hd_fail(HD_ERR_INVALID_ARG, name + ": null library");
    if (!hd_lib_binary(lib)) return hd_fail(HD_ERR_INVALID_ARG, name + ": multi-bit library (use hd_cascade_search_dot)");
    if (n_q == 0) return HD_OK;
    if (!d_q_hv || !d_q_mz || !d_q_charge || !d_out_idx || !d_out_dist || !d_out_q || !d_out_level)
        return hd_fail(HD_ERR_INVALID_ARG, name + ": null buffer");
    if (reinterpret_cast<uintptr_t>(d_q_hv) & 15u)
        return hd_fail(HD_ERR_INVALID_ARG, name + ": d_q_hv must be 16-byte aligned");
    if (form != HD_FORM_AUTO && form != HD_FORM_POPC && !hd_is_tc_form(form))
        return hd_fail(HD_ERR_INVALID_ARG, name + ": unknown form");
    hd_status st = check_levels(lib, levels, n_levels, fdr, name);
    if (st != HD_OK) return st;
    return cascade_run<uint16_t>(lib, reinterpret_cast<const uint8_t *>(d_q_hv), lib->W * 8, d_q_mz, d_q_charge, n_q,
                                 levels, n_levels, fdr, form, 0, lib->dim + 1, (uint16_t)0xFFFF, d_out_idx,
                                 d_out_dist, d_out_q, d_out_level, (cudaStream_t)stream, name);
}

hd_status hd_cascade_search_dot(const hd_library *lib, const int8_t *d_q_comp, const double *d_q_mz,
                                const uint8_t *d_q_charge, uint32_t n_q, const hd_window *levels, uint32_t n_levels,
                                double fdr, hd_search_form form, uint32_t *d_out_idx, int32_t *d_out_score,
                                double *d_out_q, uint8_t *d_out_level, hd_stream stream)
{
    const std::string name = "hd_cascade_search_dot";
    if (!lib) return hd_fail(HD_ERR_INVALID_ARG, name + ": null library");
    if (hd_lib_binary(lib)) return hd_fail(HD_ERR_INVALID_ARG, name + ": binary library (use hd_cascade_search)");
    hd_status st0 = hd_dot_check(lib, &form, name);
    if (st0 != HD_OK) return st0;
    if (n_q == 0) return HD_OK;
    if (!d_q_comp || !d_q_mz || !d_q_charge || !d_out_idx || !d_out_score || !d_out_q || !d_out_level)
        return hd_fail(HD_ERR_INVALID_ARG, name + ": null buffer");
    if (reinterpret_cast<uintptr_t>(d_q_comp) & 15u)
        return hd_fail(HD_ERR_INVALID_ARG, name + ": d_q_comp must be 16-byte aligned");
    hd_status st = check_levels(lib, levels, n_levels, fdr, name);
    if (st != HD_OK) return st;
    const uint32_t m = hd_comp_max(lib->bits), bias = lib->dim * m * m;
    return cascade_run<int32_t>(lib, reinterpret_cast<const uint8_t *>(d_q_comp), lib->dim, d_q_mz, d_q_charge, n_q,
                                levels, n_levels, fdr, form, bias, 2 * bias + 1, INT32_MIN, d_out_idx, d_out_score,
                                d_out_q, d_out_level, (cudaStream_t)stream, name);
}

}  // extern "C"
