// search_popc.cu -- open-modification Hamming search (Section 3.4), popcount
// form.
//
// Pipeline of one hd_search_open call (all on the caller's stream):
//   1. sort the queries by (charge, precursor m/z) so that consecutive
//      queries share most of their candidate window;
//   2. per query, its window [lo, hi) of library rows (same charge,
//      |mz_r - mz_q| <= tol_q in IEEE double) by binary search;
//   3. work list: blocks of BQ sorted queries; a block's tiles cover the
//      union of its windows in BR-row tiles; a work item is a run of tiles;
//   4. persistent search kernel: each CTA takes items from an atomic
//      counter, stages query and reference rows into shared memory with
//      1-D bulk copies (TMA engine, mbarrier completion), scores every pair
//      with XOR + popc, masks pairs outside the query's own window and keeps
//      a per-query top-k of (distance, input index) keys, merged across the
//      warp with shuffles;
//   5. merge the items of each block and scatter to the caller's order.
#include "hd_internal.cuh"

void hd_exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint32_t n, hd_arena &arena,
                           cudaStream_t s);

namespace {

constexpr int BQ = 64;                  // queries per block
constexpr int BR = 64;                  // reference rows per tile
constexpr int THREADS = 256;
constexpr uint32_t CHUNK_W32 = 128;     // 4096 bits of a row staged per step
constexpr uint32_t PITCH32 = CHUNK_W32 + 4;   // padded row pitch (conflict-free LDS.128)
constexpr uint32_t PITCH_B = PITCH32 * 4;
constexpr uint32_t STAGE_B = (BQ + BR) * PITCH_B;
constexpr uint32_t SMEM_B = 2 * STAGE_B + 64;
constexpr uint64_t KEY_NONE = ~0ull;

// ----------------------------------------------------------------- windows
__global__ void k_windows(const double *__restrict__ lib_mz, const uint32_t *__restrict__ cstart,
                          const double *__restrict__ q_mz, const uint8_t *__restrict__ q_z,
                          const uint32_t *__restrict__ perm, uint32_t n_q, double tol, int ppm,
                          uint32_t *__restrict__ lo, uint32_t *__restrict__ hi)
{
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_q) return;
    const uint32_t q = perm ? perm[s] : s;
    const double m = q_mz[q];
    const uint32_t c = q_z[q];
    const double t = ppm ? __dmul_rn(m, tol) : tol;   // tol holds tol*1e-6 for ppm
    const double nt = -t;
    const uint32_t p0 = cstart[c], p1 = cstart[c + 1];
    // first row with (mz_r - m) >= -t
    uint32_t a = p0, b = p1;
    while (a < b) {
        const uint32_t mid = a + ((b - a) >> 1);
        if (__dsub_rn(lib_mz[mid], m) >= nt) b = mid; else a = mid + 1;
    }
    const uint32_t l = a;
    // first row with (mz_r - m) > t
    b = p1;
    while (a < b) {
        const uint32_t mid = a + ((b - a) >> 1);
        if (__dsub_rn(lib_mz[mid], m) > t) b = mid; else a = mid + 1;
    }
    lo[s] = l;
    hi[s] = a;
}

// --------------------------------------------------------------- work list
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total, uint32_t *sh)
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

__global__ void __launch_bounds__(1024)
k_worklist(const uint32_t *__restrict__ lo, const uint32_t *__restrict__ hi, uint32_t n_q,
           uint32_t n_blocks, uint32_t target_items, uint32_t *__restrict__ blk_lo,
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
        const uint32_t e = min(n_q, (b + 1) * (uint32_t)BQ);
        for (uint32_t s = b * BQ; s < e; ++s)
            if (hi[s] > lo[s]) {
                l = min(l, lo[s]);
                h = max(h, hi[s]);
            }
        const uint32_t nt = h > l ? (h - l + BR - 1) / BR : 0u;
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

// Bounded wait: false once HD_WAIT_NS of wall time passed without the phase.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = hd_globaltimer_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 0 && hd_globaltimer_ns() - t0 > HD_WAIT_NS) return false;
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

struct search_args {
    const uint64_t *lib_hv;
    const uint32_t *lib_orig;
    const uint64_t *q_hv;
    const uint32_t *perm;
    const uint32_t *lo, *hi;
    const uint32_t *blk_lo, *blk_hi, *blk_nt, *item_start;
    uint32_t *meta;            // [0] tiles per item, [1] work counter
    uint64_t *partial;         // [items][BQ][K]
    uint32_t *status;
    uint32_t n_q, n_blocks, W64;
};

// ------------------------------------------------------------ search kernel
template <int K>
__global__ void __launch_bounds__(THREADS, 1) k_search_popc(search_args a)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * STAGE_B);
    __shared__ uint32_t s_item;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int qg = 2 * warp + (lane >> 4);   // query group 0..15
    const int rg = lane & 15;                // reference group 0..15
    const uint32_t W32 = a.W64 * 2;
    const uint32_t nchunks = (W32 + CHUNK_W32 - 1) / CHUNK_W32;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const uint32_t total_items = a.item_start[a.n_blocks];
    const uint32_t tpi = a.meta[0];
    uint32_t parity = 0;   // bit st: phase parity expected next on stage st

    for (;;) {
        if (tid == 0) s_item = atomicAdd(&a.meta[1], 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= total_items) break;

        // block of this item: last b with item_start[b] <= item
        uint32_t lo_b = 0, hi_b = a.n_blocks;
        while (hi_b - lo_b > 1) {
            const uint32_t mid = (lo_b + hi_b) >> 1;
            if (a.item_start[mid] <= item) lo_b = mid; else hi_b = mid;
        }
        const uint32_t b = lo_b;
        const uint32_t nt = a.blk_nt[b];
        const uint32_t row_base = a.blk_lo[b];
        const uint32_t t0 = (item - a.item_start[b]) * tpi;
        const uint32_t t1 = min(nt, t0 + tpi);
        const uint32_t steps = (t1 - t0) * nchunks;
        const uint32_t q0 = b * BQ;
        const uint32_t nq = min((uint32_t)BQ, a.n_q - q0);
        const uint32_t row_end = a.blk_hi[b];   // one past the last row the block wants

        uint32_t qlo[4], qhi[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t s = q0 + qg + 16 * i;
            qlo[i] = s < a.n_q ? a.lo[s] : 0u;
            qhi[i] = s < a.n_q ? a.hi[s] : 0u;
        }
        uint64_t best[4][K];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int t = 0; t < K; ++t) best[i][t] = KEY_NONE;
        uint32_t acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0;

        // warp 0 stages step `st_step` (tile, chunk) into buffer st_step & 1
        auto issue = [&](uint32_t st_step) {
            const uint32_t tile = t0 + st_step / nchunks, ch = st_step % nchunks;
            const uint32_t cw = min(CHUNK_W32, W32 - ch * CHUNK_W32);
            const uint32_t rb = cw * 4;
            const uint32_t r0 = row_base + tile * BR;
            const uint32_t nr = min((uint32_t)BR, row_end - r0);
            uint8_t *stage = smem + (st_step & 1) * STAGE_B;
            if (lane == 0) mbar_expect_tx(&bar[st_step & 1], (nq + nr) * rb);
            __syncwarp();
            for (uint32_t x = lane; x < nq; x += 32)
                bulk_load(stage + x * PITCH_B,
                          a.q_hv + (size_t)a.perm[q0 + x] * a.W64 + ch * (CHUNK_W32 / 2), rb,
                          &bar[st_step & 1]);
            for (uint32_t x = lane; x < nr; x += 32)
                bulk_load(stage + (BQ + x) * PITCH_B,
                          a.lib_hv + (size_t)(r0 + x) * a.W64 + ch * (CHUNK_W32 / 2), rb,
                          &bar[st_step & 1]);
        };

        if (warp == 0 && steps > 0) {
            issue(0);
            if (steps > 1) issue(1);
        }
        uint32_t waited = 0;
        bool aborted = false;
        for (uint32_t s = 0; s < steps; ++s) {
            const uint32_t st = s & 1;
            const bool ok = mbar_wait(&bar[st], (parity >> st) & 1u);
            parity ^= 1u << st;
            ++waited;
            if (__syncthreads_or(!ok)) {
                aborted = true;
                break;
            }
            const uint32_t tile = t0 + s / nchunks, ch = s % nchunks;
            const uint32_t cw = min(CHUNK_W32, W32 - ch * CHUNK_W32);
            const uint32_t *qs = reinterpret_cast<const uint32_t *>(smem + st * STAGE_B);
            const uint32_t *rs = qs + BQ * PITCH32;
#pragma unroll 2
            for (uint32_t w = 0; w < cw; w += 4) {
                uint4 qv[4], rv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    qv[i] = *reinterpret_cast<const uint4 *>(qs + (qg + 16 * i) * PITCH32 + w);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    rv[j] = *reinterpret_cast<const uint4 *>(rs + (rg + 16 * j) * PITCH32 + w);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        acc[i][j] += __popc(qv[i].x ^ rv[j].x) + __popc(qv[i].y ^ rv[j].y) +
                                     __popc(qv[i].z ^ rv[j].z) + __popc(qv[i].w ^ rv[j].w);
            }
            if (ch == nchunks - 1) {
                const uint32_t r0 = row_base + tile * BR;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t row = r0 + rg + 16 * j;
                    const uint32_t o = row < row_end ? __ldg(a.lib_orig + row) : 0u;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (row >= qlo[i] && row < qhi[i]) {
                            const uint64_t key = ((uint64_t)acc[i][j] << 32) | o;
                            if (key < best[i][K - 1]) topk_insert<K>(best[i], key);
                        }
                        acc[i][j] = 0;
                    }
                }
            }
            __syncthreads();
            if (warp == 0 && s + 2 < steps) issue(s + 2);
        }
        if (aborted) {
            if (tid == 0) hd_flag(a.status, HD_DEV_TIMEOUT);
            // let copies still in flight land before the CTA's memory is released
            const uint32_t issued = min(steps, waited + 1);
            for (uint32_t s = waited; s < issued; ++s) {
                mbar_wait(&bar[s & 1], (parity >> (s & 1)) & 1u);
                parity ^= 1u << (s & 1);
            }
            return;
        }

        // merge the 16 lanes holding each query (xor butterfly within half-warps)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int off = 1; off < 16; off <<= 1) {
                uint64_t other[K];
#pragma unroll
                for (int t = 0; t < K; ++t) other[t] = __shfl_xor_sync(0xffffffffu, best[i][t], off);
                topk_merge<K>(best[i], other);
            }
            if (rg == 0) {
                uint64_t *dst = a.partial + ((size_t)item * BQ + qg + 16 * i) * K;
#pragma unroll
                for (int t = 0; t < K; ++t) dst[t] = best[i][t];
            }
        }
    }
}

// ------------------------------------------------------------ final merge
template <int K>
__global__ void k_merge(const uint64_t *__restrict__ partial, const uint32_t *__restrict__ item_start,
                        const uint32_t *__restrict__ perm, uint32_t n_q, uint32_t k,
                        uint32_t *__restrict__ out_idx, uint16_t *__restrict__ out_dist)
{
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_q) return;
    const uint32_t b = s / BQ, ql = s % BQ;
    uint64_t best[K];
#pragma unroll
    for (int t = 0; t < K; ++t) best[t] = KEY_NONE;
    for (uint32_t it = item_start[b]; it < item_start[b + 1]; ++it) {
        const uint64_t *p = partial + ((size_t)it * BQ + ql) * K;
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

template <int K>
hd_status run_k(const hd_library *lib, const uint64_t *q_hv, const double *q_mz,
                const uint8_t *q_z, uint32_t n_q, double tol, int ppm, uint32_t k,
                uint32_t *out_idx, uint16_t *out_dist, cudaStream_t s, char *ext = nullptr,
                size_t ext_cap = 0)
{
    const uint32_t n_blocks = (n_q + BQ - 1) / BQ;
    int occ = 0;
    HD_CUDA_TRY(cudaFuncSetAttribute(k_search_popc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SMEM_B));
    HD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_search_popc<K>, THREADS, SMEM_B));
    if (occ < 1) return hd_fail(HD_ERR_UNSUPPORTED, "search kernel does not fit on this GPU");
    const uint32_t grid = (uint32_t)(lib->num_sms * occ);
    const uint32_t target_items = 8 * grid;

    auto carve = [&](hd_arena &ar, uint32_t **perm, uint32_t **lo, uint32_t **hi, uint32_t **blo,
                     uint32_t **bhi, uint32_t **bnt, uint32_t **ist, uint32_t **meta, uint64_t **part) {
        *perm = ar.take<uint32_t>(n_q);
        *lo = ar.take<uint32_t>(n_q);
        *hi = ar.take<uint32_t>(n_q);
        *blo = ar.take<uint32_t>(n_blocks);
        *bhi = ar.take<uint32_t>(n_blocks);
        *bnt = ar.take<uint32_t>(n_blocks);
        *ist = ar.take<uint32_t>(n_blocks + 1);
        *meta = ar.take<uint32_t>(4);
        *part = ar.take<uint64_t>((size_t)(target_items + n_blocks) * BQ * K);
    };
    uint32_t *perm, *lo, *hi, *blo, *bhi, *bnt, *ist, *meta;
    uint64_t *part;
    hd_arena plan;
    carve(plan, &perm, &lo, &hi, &blo, &bhi, &bnt, &ist, &meta, &part);
    hd_sort_charge_mz(q_mz, q_z, n_q, nullptr, plan, s);
    hd_arena ar;
    if (ext) {   // caller-provided scratch: nothing is allocated
        if (plan.used > ext_cap)
            return hd_fail(HD_ERR_INVALID_ARG, "search needs " + std::to_string(plan.used) +
                                                   " bytes of scratch, more than the fixed " +
                                                   std::to_string(ext_cap));
        ar.base = ext;
    } else {
        cudaError_t e = cudaMallocAsync((void **)&ar.base, plan.used, s);
        if (e != cudaSuccess) return hd_fail(HD_ERR_OOM, "search scratch allocation failed");
    }
    carve(ar, &perm, &lo, &hi, &blo, &bhi, &bnt, &ist, &meta, &part);
    hd_sort_charge_mz(q_mz, q_z, n_q, perm, ar, s);
    const double tq = ppm ? tol * 1e-6 : tol;
    hd_count_launches(1), k_windows<<<hd_ceil_div(n_q, 256), 256, 0, s>>>(lib->mz, lib->charge_start, q_mz, q_z, perm, n_q,
                                                    tq, ppm, lo, hi);
    hd_count_launches(1), k_worklist<<<1, 1024, 0, s>>>(lo, hi, n_q, n_blocks, target_items, blo, bhi, bnt, ist, meta);
    search_args sa{lib->hv, lib->orig, q_hv, perm, lo, hi, blo, bhi, bnt, ist, meta, part,
                   lib->status.dev, n_q, n_blocks, lib->W};
    {
        hd_prof_scope timed(HD_KERNEL_SEARCH, s);
        hd_count_launches(1), k_search_popc<K><<<grid, THREADS, SMEM_B, s>>>(sa);
    }
    hd_count_launches(1), k_merge<K><<<hd_ceil_div(n_q, 128), 128, 0, s>>>(part, ist, perm, n_q, k, out_idx, out_dist);
    HD_CUDA_TRY(cudaGetLastError());
    if (!ext) HD_CUDA_TRY(cudaFreeAsync(ar.base, s));
    return HD_OK;
}

}  // namespace

void hd_windows_launch(const hd_library *lib, const double *q_mz, const uint8_t *q_charge,
                       const uint32_t *perm, uint32_t n_q, double tol, int ppm, uint32_t *lo,
                       uint32_t *hi, cudaStream_t s)
{
    const double tq = ppm ? tol * 1e-6 : tol;
    hd_count_launches(1), k_windows<<<hd_ceil_div(n_q, 256), 256, 0, s>>>(lib->mz, lib->charge_start, q_mz, q_charge, perm,
                                                    n_q, tq, ppm, lo, hi);
}

hd_status hd_search_popc_run(const hd_library *lib, const uint64_t *q_hv, const double *q_mz,
                             const uint8_t *q_charge, uint32_t n_q, double tol, int ppm,
                             uint32_t k, uint32_t *out_idx, uint16_t *out_dist, cudaStream_t s)
{
    if (k <= 1) return run_k<1>(lib, q_hv, q_mz, q_charge, n_q, tol, ppm, k, out_idx, out_dist, s);
    if (k <= 2) return run_k<2>(lib, q_hv, q_mz, q_charge, n_q, tol, ppm, k, out_idx, out_dist, s);
    if (k <= 4) return run_k<4>(lib, q_hv, q_mz, q_charge, n_q, tol, ppm, k, out_idx, out_dist, s);
    if (k <= 8) return run_k<8>(lib, q_hv, q_mz, q_charge, n_q, tol, ppm, k, out_idx, out_dist, s);
    return run_k<16>(lib, q_hv, q_mz, q_charge, n_q, tol, ppm, k, out_idx, out_dist, s);
}

hd_status hd_search_popc_run_scratch(const hd_library *lib, const uint64_t *q_hv, const double *q_mz,
                                     const uint8_t *q_charge, uint32_t n_q, double tol, int ppm,
                                     uint32_t k, uint32_t *out_idx, uint16_t *out_dist, cudaStream_t s,
                                     void *scratch, size_t scratch_bytes)
{
    char *x = static_cast<char *>(scratch);
#define HD_RUN_K(KK) run_k<KK>(lib, q_hv, q_mz, q_charge, n_q, tol, ppm, k, out_idx, out_dist, s, x, scratch_bytes)
    if (k <= 1) return HD_RUN_K(1);
    if (k <= 2) return HD_RUN_K(2);
    if (k <= 4) return HD_RUN_K(4);
    if (k <= 8) return HD_RUN_K(8);
    return HD_RUN_K(16);
#undef HD_RUN_K
}
