// preprocess.cu -- raw peaks -> CSR spectrum vectors (Section 3.2, Table 1).
//
// One CTA per spectrum.  Peak selection is by rank counting (each kept peak
// counts the peaks that beat it), so no sort is needed and the order of the
// kept peaks is fixed by the keys alone.  All floating point is IEEE double
// with explicit round-to-nearest intrinsics, so no contraction can change a
// bin or a level.
#include "hd_internal.cuh"

void hd_exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint32_t n, hd_arena &arena,
                           cudaStream_t s);

namespace {

constexpr int PP_THREADS = 128;
constexpr uint32_t PP_MAX_RAW = 8192;
constexpr uint32_t PP_MAX_KEEP = 1023;

struct pp_args {
    double mz_min, mz_max, bin_width, min_rel;
    uint32_t n_bins, max_peaks, n_levels;
};

__device__ __forceinline__ bool pk_valid(double mz, double it, const pp_args &a)
{
    return isfinite(mz) && isfinite(it) && it > 0.0 && mz >= a.mz_min && mz <= a.mz_max;
}

// (it_j, mz_j, j) ranks ahead of (it_i, mz_i, i): more intense, then lower m/z,
// then lower input position.
__device__ __forceinline__ bool beats(double itj, double mzj, uint32_t j, double iti, double mzi,
                                      uint32_t i)
{
    if (itj != iti) return itj > iti;
    if (mzj != mzi) return mzj < mzi;
    return j < i;
}

__device__ double block_max(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = red[0];
    for (int i = 1; i < PP_THREADS / 32; ++i) r = fmax(r, red[i]);
    return r;
}

__global__ void __launch_bounds__(PP_THREADS)
k_preprocess(pp_args a, const uint32_t *__restrict__ raw_off, const double *__restrict__ raw_mz,
             const double *__restrict__ raw_it, uint32_t n_spec, uint32_t *__restrict__ tmp_bins,
             uint8_t *__restrict__ tmp_lv, uint32_t *__restrict__ count, uint32_t *status)
{
    __shared__ uint32_t keep_bits[PP_MAX_RAW / 32];
    __shared__ uint32_t sel_bits[PP_MAX_RAW / 32];
    __shared__ double s_mz[PP_MAX_KEEP + 1], s_it[PP_MAX_KEEP + 1], s_sum[PP_MAX_KEEP + 1];
    __shared__ uint32_t s_bin[PP_MAX_KEEP + 1];
    __shared__ uint32_t s_head[PP_MAX_KEEP + 1];
    __shared__ double red[PP_THREADS / 32];
    __shared__ uint32_t s_cnt;

    const uint32_t sp = blockIdx.x;
    if (sp >= n_spec) return;
    const uint32_t beg = raw_off[sp], end = raw_off[sp + 1];
    if (end < beg || end - beg > PP_MAX_RAW) {
        if (threadIdx.x == 0) {
            count[sp] = 0;
            hd_flag(status, HD_DEV_BAD_INPUT);
        }
        return;
    }
    const uint32_t n = end - beg;
    const double *mz = raw_mz + beg, *it = raw_it + beg;

    // steps 0-1: finite, positive, inside the m/z range; then the top intensity
    double top = 0.0;
    for (uint32_t i = threadIdx.x; i < n; i += PP_THREADS)
        if (pk_valid(mz[i], it[i], a)) top = fmax(top, it[i]);
    top = block_max(top, red);
    const double floor_it = __dmul_rn(a.min_rel, top);

    // step 2: drop peaks below the relative floor
    for (uint32_t w = threadIdx.x; w < (n + 31) / 32; w += PP_THREADS) {
        uint32_t bits = 0;
        for (uint32_t b = 0; b < 32 && w * 32 + b < n; ++b) {
            const uint32_t i = w * 32 + b;
            bits |= (uint32_t)(pk_valid(mz[i], it[i], a) && !(it[i] < floor_it)) << b;
        }
        keep_bits[w] = bits;
        sel_bits[w] = 0;
    }
    __syncthreads();

    // step 3: keep the max_peaks most intense (rank among kept peaks)
    for (uint32_t i = threadIdx.x; i < n; i += PP_THREADS) {
        if (!((keep_bits[i >> 5] >> (i & 31)) & 1u)) continue;
        const double iti = it[i], mzi = mz[i];
        uint32_t r = 0;
        for (uint32_t j = 0; j < n && r < a.max_peaks; ++j)
            if (((keep_bits[j >> 5] >> (j & 31)) & 1u) && beats(it[j], mz[j], j, iti, mzi, i)) ++r;
        if (r < a.max_peaks) atomicOr(&sel_bits[i >> 5], 1u << (i & 31));
    }
    __syncthreads();

    // order the selected peaks by (m/z, input position)
    uint32_t m_local = 0;
    for (uint32_t i = threadIdx.x; i < n; i += PP_THREADS) {
        if (!((sel_bits[i >> 5] >> (i & 31)) & 1u)) continue;
        ++m_local;
        const double mzi = mz[i];
        uint32_t p = 0;
        for (uint32_t j = 0; j < n; ++j)
            if (((sel_bits[j >> 5] >> (j & 31)) & 1u) && (mz[j] < mzi || (mz[j] == mzi && j < i))) ++p;
        s_mz[p] = mzi;
        s_it[p] = it[i];
    }
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    if (m_local) atomicAdd(&s_cnt, m_local);
    __syncthreads();
    const uint32_t m = s_cnt;

    // step 4: bins; run heads mark the first peak of each bin
    for (uint32_t t = threadIdx.x; t < m; t += PP_THREADS) {
        const double x = floor(__ddiv_rn(__dsub_rn(s_mz[t], a.mz_min), a.bin_width));
        s_bin[t] = x < 0.0 ? 0u : (x > (double)(a.n_bins - 1) ? a.n_bins - 1 : (uint32_t)x);
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < m; t += PP_THREADS) s_head[t] = (t == 0 || s_bin[t] != s_bin[t - 1]);
    __syncthreads();
    // step 5: each run head sums its run in ascending m/z order
    for (uint32_t t = threadIdx.x; t < m; t += PP_THREADS) {
        if (!s_head[t]) continue;
        double v = s_it[t];
        for (uint32_t u = t + 1; u < m && s_bin[u] == s_bin[t]; ++u) v = __dadd_rn(v, s_it[u]);
        s_sum[t] = v;
    }
    __syncthreads();
    double vmax = 0.0;
    for (uint32_t t = threadIdx.x; t < m; t += PP_THREADS)
        if (s_head[t]) vmax = fmax(vmax, s_sum[t]);
    vmax = block_max(vmax, red);
    // step 6: quantise and write the rows (output slot = heads before t)
    const double q = (double)a.n_levels;
    for (uint32_t t = threadIdx.x; t < m; t += PP_THREADS) {
        if (!s_head[t]) continue;
        uint32_t slot = 0;
        for (uint32_t u = 0; u < t; ++u) slot += s_head[u];
        const double lv = floor(__ddiv_rn(__dmul_rn(q, s_sum[t]), vmax));
        const uint32_t l = lv >= (double)(a.n_levels - 1) ? a.n_levels - 1 : (uint32_t)lv;
        tmp_bins[(size_t)sp * a.max_peaks + slot] = s_bin[t];
        tmp_lv[(size_t)sp * a.max_peaks + slot] = (uint8_t)l;
    }
    if (threadIdx.x == 0) {
        uint32_t nb = 0;
        for (uint32_t u = 0; u < m; ++u) nb += s_head[u];
        count[sp] = nb;
    }
}

// Packs the padded rows into CSR: one warp per spectrum.
__global__ void k_compact(const uint32_t *__restrict__ tmp_bins, const uint8_t *__restrict__ tmp_lv,
                          const uint32_t *__restrict__ off, uint32_t n_spec, uint32_t max_peaks,
                          uint32_t *__restrict__ bins, uint8_t *__restrict__ lv)
{
    const uint32_t sp = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (sp >= n_spec) return;
    const uint32_t o = off[sp], c = off[sp + 1] - o;
    for (uint32_t t = threadIdx.x & 31; t < c; t += 32) {
        bins[o + t] = tmp_bins[(size_t)sp * max_peaks + t];
        lv[o + t] = tmp_lv[(size_t)sp * max_peaks + t];
    }
}

}  // namespace

hd_status hd_preprocess_launch(const hd_preprocess_params &pp, const uint32_t *raw_off,
                               const double *raw_mz, const double *raw_int, uint32_t n,
                               uint32_t *out_off, uint32_t *out_bins, uint8_t *out_levels,
                               uint32_t *status, cudaStream_t s)
{
    if (n == 0) {
        HD_CUDA_TRY(cudaMemsetAsync(out_off, 0, sizeof(uint32_t), s));
        return HD_OK;
    }
    hd_arena plan;
    auto carve = [&](hd_arena &ar, uint32_t **tb, uint8_t **tl, uint32_t **cnt) {
        *tb = ar.take<uint32_t>((size_t)n * pp.max_peaks);
        *tl = ar.take<uint8_t>((size_t)n * pp.max_peaks);
        *cnt = ar.take<uint32_t>(n);
    };
    uint32_t *tb, *cnt;
    uint8_t *tl;
    carve(plan, &tb, &tl, &cnt);
    hd_exclusive_scan_u32(nullptr, nullptr, n, plan, s);   // sizing pass
    hd_arena ar;
    HD_CUDA_TRY(cudaMallocAsync((void **)&ar.base, plan.used, s));
    carve(ar, &tb, &tl, &cnt);
    pp_args a{pp.mz_min, pp.mz_max, pp.bin_width, pp.min_rel_intensity, pp.n_bins, pp.max_peaks,
              pp.n_levels};
    hd_count_launches(1), k_preprocess<<<n, PP_THREADS, 0, s>>>(a, raw_off, raw_mz, raw_int, n, tb, tl, cnt, status);
    hd_exclusive_scan_u32(cnt, out_off, n, ar, s);
    hd_count_launches(1), k_compact<<<hd_ceil_div(n, 8), 256, 0, s>>>(tb, tl, out_off, n, pp.max_peaks, out_bins, out_levels);
    HD_CUDA_TRY(cudaGetLastError());
    HD_CUDA_TRY(cudaFreeAsync(ar.base, s));
    return HD_OK;
}
