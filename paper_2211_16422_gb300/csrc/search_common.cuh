// search_common.cuh -- pieces shared by the two search forms (Section 3.4):
// candidate windows, the work list over query blocks and reference tiles,
// mbarrier / bulk-copy PTX, per-query top-k lists and the final merge.
#pragma once

#include "hd_internal.cuh"

namespace hd_search {

// Non-template kernels and functions are static: every translation unit that
// includes this header gets its own copy.

constexpr uint64_t KEY_NONE = ~0ull;

// ----------------------------------------------------------------- windows
static __global__ void k_windows(const double *__restrict__ lib_mz, const uint32_t *__restrict__ cstart,
                          const double *__restrict__ q_mz, const uint8_t *__restrict__ q_z,
                          const uint32_t *__restrict__ perm, uint32_t n_q, hd_qwin win,
                          uint32_t *__restrict__ lo, uint32_t *__restrict__ hi)
{
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_q) return;
    const uint32_t q = perm ? perm[s] : s;
    const double m = q_mz[q];
    const uint32_t c = q_z[q];
    const uint32_t wc = win.cls ? min((uint32_t)win.cls[q], win.n - 1) : 0u;
    const hd_win w = win.w[wc];
    const uint32_t p0 = cstart[c], p1 = cstart[c + 1];
    // Within one charge the compared quantity is non-decreasing in the row's
    // m/z (IEEE subtraction and multiplication by a charge >= 0 are monotone),
    // so each bound is the first row where a monotone predicate turns true.
    auto delta = [&](uint32_t r) -> double {
        if (w.unit == HD_TOL_MASS)   // neutral masses (mz - 1.007276) * z
            return __dsub_rn(__dmul_rn(__dsub_rn(lib_mz[r], 1.007276), (double)c),
                             __dmul_rn(__dsub_rn(m, 1.007276), (double)c));
        return __dsub_rn(lib_mz[r], m);
    };
    const double t = w.unit == HD_TOL_PPM ? __dmul_rn(m, w.tol) : w.tol;   // tol holds tol*1e-6 for ppm
    const double nt = -t;
    // first row with delta >= -t
    uint32_t a = p0, b = p1;
    while (a < b) {
        const uint32_t mid = a + ((b - a) >> 1);
        if (delta(mid) >= nt) b = mid; else a = mid + 1;
    }
    const uint32_t l = a;
    // first row with delta > t
    b = p1;
    while (a < b) {
        const uint32_t mid = a + ((b - a) >> 1);
        if (delta(mid) > t) b = mid; else a = mid + 1;
    }
    lo[s] = l;
    hi[s] = a;
}

// --------------------------------------------------------------- work list
static __device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total, uint32_t *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t y = lane < nw ? sh[lane] : 0u, yi = y;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t z = __shfl_up_sync(0xffffffffu, yi, o);
            if (lane >= o) yi += z;
        }
        if (lane < nw) sh[lane] = yi - y;
        if (lane == 31) sh[32] = yi;
    }
    __syncthreads();
    *total = sh[32];
    return sh[w] + x - v;
}

static __global__ void __launch_bounds__(1024)
k_worklist(const uint32_t *__restrict__ lo, const uint32_t *__restrict__ hi, uint32_t n_q,
           uint32_t bq, uint32_t br, uint32_t n_blocks, uint32_t target_items, uint32_t *__restrict__ blk_lo,
           uint32_t *__restrict__ blk_hi, uint32_t *__restrict__ blk_nt, uint32_t *__restrict__ item_start,
           uint32_t *__restrict__ meta)
{
    __shared__ uint32_t sh[33];
    __shared__ unsigned long long s_tot;
    if (threadIdx.x == 0) s_tot = 0;
    __syncthreads();
    unsigned long long mine = 0;
    for (uint32_t b = threadIdx.x; b < n_blocks; b += blockDim.x) {
        uint32_t l = 0xFFFFFFFFu, h = 0;
        const uint32_t e = min(n_q, (b + 1) * bq);
        for (uint32_t s = b * bq; s < e; ++s)
            if (hi[s] > lo[s]) {
                l = min(l, lo[s]);
                h = max(h, hi[s]);
            }
        const uint32_t nt = h > l ? (h - l + br - 1) / br : 0u;
        blk_lo[b] = nt ? l : 0u;
        blk_hi[b] = nt ? h : 0u;
        blk_nt[b] = nt;
        mine += nt;
    }
    atomicAdd(&s_tot, mine);
    __syncthreads();
    const unsigned long long T = s_tot;
    uint32_t tpi = (uint32_t)((T + target_items - 1) / target_items);
    tpi = max(tpi, 4u);
    if (threadIdx.x == 0) {
        meta[0] = tpi;
        meta[1] = 0;   // work counter
    }
    uint32_t carry = 0;
    for (uint32_t base = 0; base < n_blocks; base += blockDim.x) {
        const uint32_t b = base + threadIdx.x;
        const uint32_t v = b < n_blocks ? (blk_nt[b] + tpi - 1) / tpi : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, &tot, sh);
        if (b < n_blocks) item_start[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) item_start[n_blocks] = carry;
}

// ------------------------------------------------- mbarrier / bulk copy PTX
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false once `limit_ns` of wall time passed without the phase.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns = HD_WAIT_NS)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = hd_globaltimer_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 0 && hd_globaltimer_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// -------------------------------------------------------------- top-k lists
template <int K>
__device__ __forceinline__ void topk_insert(uint64_t (&best)[K], uint64_t key)
{
#pragma unroll
    for (int t = K - 1; t > 0; --t) {
        const uint64_t prev = best[t - 1];
        best[t] = key < prev ? prev : (key < best[t] ? key : best[t]);
    }
    best[0] = key < best[0] ? key : best[0];
}

// best <- the K smallest of best U other (both ascending): bitonic merge.
template <int K>
__device__ __forceinline__ void topk_merge(uint64_t (&best)[K], const uint64_t (&other)[K])
{
#pragma unroll
    for (int t = 0; t < K; ++t) {
        const uint64_t o = other[K - 1 - t];
        best[t] = o < best[t] ? o : best[t];
    }
#pragma unroll
    for (int len = K / 2; len >= 1; len >>= 1)
#pragma unroll
        for (int t = 0; t < K; ++t)
            if ((t & len) == 0) {
                const uint64_t a = best[t], b = best[t + len];
                best[t] = a < b ? a : b;
                best[t + len] = a < b ? b : a;
            }
}


// ------------------------------------------------------------ final merge
template <int K>
__global__ void k_merge(const uint64_t *__restrict__ partial, const uint32_t *__restrict__ item_start, uint32_t bq,
                        const uint32_t *__restrict__ perm, uint32_t n_q, uint32_t k,
                        uint32_t *__restrict__ out_idx, uint16_t *__restrict__ out_dist)
{
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_q) return;
    const uint32_t b = s / bq, ql = s % bq;
    uint64_t best[K];
#pragma unroll
    for (int t = 0; t < K; ++t) best[t] = KEY_NONE;
    for (uint32_t it = item_start[b]; it < item_start[b + 1]; ++it) {
        const uint64_t *p = partial + ((size_t)it * bq + ql) * K;
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const uint64_t key = p[t];
            if (key >= best[K - 1]) break;
            topk_insert<K>(best, key);
        }
    }
    const uint32_t q = perm[s];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        if ((uint32_t)t < k) {
            const bool none = best[t] == KEY_NONE;
            out_idx[(size_t)q * k + t] = none ? 0xFFFFFFFFu : (uint32_t)best[t];
            out_dist[(size_t)q * k + t] = none ? (uint16_t)0xFFFF : (uint16_t)(best[t] >> 32);
        }
    }
}


}  // namespace hd_search
