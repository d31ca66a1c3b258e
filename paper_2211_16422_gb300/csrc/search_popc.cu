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
#include <vector>
#include <algorithm>
#include "hd_internal.cuh"
#include "search_common.cuh"

void hd_exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint32_t n, hd_arena &arena,
                           cudaStream_t s);

namespace {

using namespace hd_search;

constexpr int BQ = 64;                  // queries per block
constexpr int BR = 64;                  // reference rows per tile
constexpr int THREADS = 256;
constexpr uint32_t CHUNK_W32 = 128;     // 4096 bits of a row staged per step
constexpr uint32_t PITCH32 = CHUNK_W32 + 4;   // padded row pitch (conflict-free LDS.128)
constexpr uint32_t PITCH_B = PITCH32 * 4;
constexpr uint32_t STAGE_B = (BQ + BR) * PITCH_B;
// Stage ring: the loads of step s + NST - 1 are issued at the start of step
// s, once the CTA barrier that opens the step has shown every warp done with
// step s - 1, so each step needs one barrier.  At "full": 3 stages 831 ms
// against 943 ms for 2 stages with a second barrier at the end of each step.
#ifndef HD_POPC_STAGES
#define HD_POPC_STAGES 3
#endif
constexpr uint32_t NST = HD_POPC_STAGES;
static_assert(NST >= 2 && NST <= 3, "two or three stages fit in shared memory");
constexpr uint32_t SMEM_B = NST * STAGE_B + 64;

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
    uint64_t wait_ns;      // bound of every device wait
    uint32_t stall;        // test hook: drop the first stage copies
};

// Carry-save step: ones + a + b = ones' + 2 * carry bitwise (a full adder per
// bit position), and the carries are counted at once: acc += 2 * popc(carry).
__device__ __forceinline__ void csa2(uint32_t &ones, uint32_t &acc, uint32_t a, uint32_t b)
{
    const uint32_t carry = (ones & a) | (ones & b) | (a & b);
    ones ^= a ^ b;
    acc += __popc(carry) << 1;
}

// ------------------------------------------------------------ search kernel
template <int K>
__global__ void __launch_bounds__(THREADS, 1) k_search_popc(search_args a)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + NST * STAGE_B);
    __shared__ uint32_t s_item;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int qg = 2 * warp + (lane >> 4);   // query group 0..15
    const int rg = lane & 15;                // reference group 0..15
    const uint32_t W32 = a.W64 * 2;
    const uint32_t nchunks = (W32 + CHUNK_W32 - 1) / CHUNK_W32;

    if (tid == 0) {
        for (uint32_t i = 0; i < NST; ++i) mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const uint32_t total_items = a.item_start[a.n_blocks];
    const uint32_t tpi = a.meta[0];
    uint32_t parity = 0;   // bit st: phase parity expected next on stage st
    bool first_item = true;

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
        // distance of pair (i, j) = acc + popcount(ones): `ones` is a carry-save
        // word (Harley and Seal's full adder) that absorbs two XOR words per
        // step, so one popcount of the carries counts two words
        uint32_t acc[4][4], ones[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = ones[i][j] = 0;

        // warp 0 stages step `st_step` (tile, chunk) into buffer st_step % NST
        auto issue = [&](uint32_t st_step) {
            const uint32_t tile = t0 + st_step / nchunks, ch = st_step % nchunks;
            const uint32_t cw = min(CHUNK_W32, W32 - ch * CHUNK_W32);
            const uint32_t rb = cw * 4;
            const uint32_t r0 = row_base + tile * BR;
            const uint32_t nr = min((uint32_t)BR, row_end - r0);
            const uint32_t sb = st_step % NST;
            uint8_t *stage = smem + sb * STAGE_B;
            if (lane == 0) mbar_expect_tx(&bar[sb], (nq + nr) * rb);
            __syncwarp();
            if (a.stall && first_item && st_step == 0) return;   // nothing completes this stage
            for (uint32_t x = lane; x < nq; x += 32)
                bulk_load(stage + x * PITCH_B,
                          a.q_hv + (size_t)a.perm[q0 + x] * a.W64 + ch * (CHUNK_W32 / 2), rb,
                          &bar[sb]);
            for (uint32_t x = lane; x < nr; x += 32)
                bulk_load(stage + (BQ + x) * PITCH_B,
                          a.lib_hv + (size_t)(r0 + x) * a.W64 + ch * (CHUNK_W32 / 2), rb,
                          &bar[sb]);
        };

        if (warp == 0)
            for (uint32_t p = 0; p + 1 < NST && p < steps; ++p) issue(p);
        uint32_t waited = 0;
        bool aborted = false;
        for (uint32_t s = 0; s < steps; ++s) {
            const uint32_t st = s % NST;
            const bool ok = mbar_wait(&bar[st], (parity >> st) & 1u, a.wait_ns);
            parity ^= 1u << st;
            ++waited;
            if (__syncthreads_or(!ok)) {
                aborted = true;
                break;
            }
            // every warp is done with step s - 1: its buffer takes step s + NST - 1
            if (warp == 0 && s + NST - 1 < steps) issue(s + NST - 1);
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
                    for (int j = 0; j < 4; ++j) {
                        csa2(ones[i][j], acc[i][j], qv[i].x ^ rv[j].x, qv[i].y ^ rv[j].y);
                        csa2(ones[i][j], acc[i][j], qv[i].z ^ rv[j].z, qv[i].w ^ rv[j].w);
                    }
            }
            if (ch == nchunks - 1) {
                const uint32_t r0 = row_base + tile * BR;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t row = r0 + rg + 16 * j;
                    const uint32_t o = row < row_end ? __ldg(a.lib_orig + row) : 0u;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        acc[i][j] += __popc(ones[i][j]);
                        ones[i][j] = 0;
                        if (row >= qlo[i] && row < qhi[i]) {
                            const uint64_t key = ((uint64_t)acc[i][j] << 32) | o;
                            if (key < best[i][K - 1]) topk_insert<K>(best[i], key);
                        }
                        acc[i][j] = 0;
                    }
                }
            }
        }
        if (aborted) {
            if (tid == 0) hd_flag(a.status, HD_DEV_TIMEOUT);
            // let copies still in flight land before the CTA's memory is released
            const uint32_t issued = min(steps, waited + NST - 2);
            for (uint32_t s = waited; s < issued; ++s) {
                mbar_wait(&bar[s % NST], (parity >> (s % NST)) & 1u, a.wait_ns);
                parity ^= 1u << (s % NST);
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
        first_item = false;
    }
}

template <int K>
hd_status run_k(const hd_library *lib, const uint64_t *q_hv, const double *q_mz,
                const uint8_t *q_z, uint32_t n_q, const hd_qwin &win, uint32_t k,
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
    hd_sort_charge_mz(q_mz, q_z, win.cls, n_q, nullptr, plan, s);
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
    hd_sort_charge_mz(q_mz, q_z, win.cls, n_q, perm, ar, s);
    hd_count_launches(1), k_windows<<<hd_ceil_div(n_q, 256), 256, 0, s>>>(lib->mz, lib->charge_start, q_mz, q_z, perm, n_q,
                                                    win, lo, hi);
    hd_count_launches(1), k_worklist<<<1, 1024, 0, s>>>(lo, hi, n_q, BQ, BR, n_blocks, target_items, blo, bhi, bnt, ist, meta);
    search_args sa{lib->hv, lib->orig, q_hv, perm, lo, hi, blo, bhi, bnt, ist, meta, part,
                   lib->status.dev, n_q, n_blocks, lib->W, hd_wait_limit(lib),
                   hd_take_injected_stall(lib) ? 1u : 0u};
    {
        hd_prof_scope timed(HD_KERNEL_SEARCH, s);
        hd_count_launches(1), k_search_popc<K><<<grid, THREADS, SMEM_B, s>>>(sa);
    }
    hd_count_launches(1), k_merge<K><<<hd_ceil_div(n_q, 128), 128, 0, s>>>(part, ist, BQ, perm, n_q, k, out_idx, out_dist);
    HD_CUDA_TRY(cudaGetLastError());
    if (!ext) HD_CUDA_TRY(cudaFreeAsync(ar.base, s));
    return HD_OK;
}

}  // namespace

void hd_windows_launch(const hd_library *lib, const double *q_mz, const uint8_t *q_charge,
                       const uint32_t *perm, uint32_t n_q, const hd_qwin &win, uint32_t *lo,
                       uint32_t *hi, cudaStream_t s)
{
    hd_count_launches(1), hd_search::k_windows<<<hd_ceil_div(n_q, 256), 256, 0, s>>>(lib->mz, lib->charge_start, q_mz, q_charge, perm,
                                                    n_q, win, lo, hi);
}

hd_qwin hd_single_window(double tol, hd_tol_unit unit)
{
    hd_qwin w;
    w.n = 1;
    w.w[0].tol = unit == HD_TOL_PPM ? tol * 1e-6 : tol;
    w.w[0].unit = (int)unit;
    return w;
}

hd_status hd_search_popc_run(const hd_library *lib, const uint64_t *q_hv, const double *q_mz,
                             const uint8_t *q_charge, uint32_t n_q, const hd_qwin &win,
                             uint32_t k, uint32_t *out_idx, uint16_t *out_dist, cudaStream_t s)
{
    if (k <= 1) return run_k<1>(lib, q_hv, q_mz, q_charge, n_q, win, k, out_idx, out_dist, s);
    if (k <= 2) return run_k<2>(lib, q_hv, q_mz, q_charge, n_q, win, k, out_idx, out_dist, s);
    if (k <= 4) return run_k<4>(lib, q_hv, q_mz, q_charge, n_q, win, k, out_idx, out_dist, s);
    if (k <= 8) return run_k<8>(lib, q_hv, q_mz, q_charge, n_q, win, k, out_idx, out_dist, s);
    return run_k<16>(lib, q_hv, q_mz, q_charge, n_q, win, k, out_idx, out_dist, s);
}

hd_status hd_search_popc_run_scratch(const hd_library *lib, const uint64_t *q_hv, const double *q_mz,
                                     const uint8_t *q_charge, uint32_t n_q, const hd_qwin &win,
                                     uint32_t k, uint32_t *out_idx, uint16_t *out_dist, cudaStream_t s,
                                     void *scratch, size_t scratch_bytes)
{
    char *x = static_cast<char *>(scratch);
#define HD_RUN_K(KK) run_k<KK>(lib, q_hv, q_mz, q_charge, n_q, win, k, out_idx, out_dist, s, x, scratch_bytes)
    if (k <= 1) return HD_RUN_K(1);
    if (k <= 2) return HD_RUN_K(2);
    if (k <= 4) return HD_RUN_K(4);
    if (k <= 8) return HD_RUN_K(8);
    return HD_RUN_K(16);
#undef HD_RUN_K
}

// ------------------------------------- popcount form of multi-bit components
// Components h in [-m, m] (Section 4.3) as offset values u = h + m in b bit
// planes; with P = sum over d of u_q,d u_r,d = sum over plane pairs (i, j) of
// 2^(i+j) popc(Q_i & R_j), the dot product is S = P - m (U_q + U_r) + D m^2
// (U the row sums of u).  Keys carry D m^2 - S = m (U_q + U_r) - P, the
// multi-bit key distance of the tensor-core form, so the same top-k lists and
// ties serve both.  Plane layout of a row: chunks of 1024 components, each
// chunk the b planes' 32-bit words one plane after the other (the last chunk
// holds the row's remaining words), so a row's chunk is one bulk copy.
namespace {

constexpr uint32_t MB_CW = 32;   // 32-bit words of one plane in a chunk

__host__ __device__ inline uint32_t mb_pitch(uint32_t bits) { return bits * MB_CW + 4; }   // words, conflict-free LDS.128
__host__ __device__ inline uint32_t mb_stage_bytes(uint32_t bits) { return (BQ + BR) * mb_pitch(bits) * 4; }

// int8 components [n][D] -> planes [n][bits * D/32] and row sums; one warp
// per row, one ballot per plane and 32-component word.  A component outside
// [-m, m] flags the status word and counts as 0.
__global__ void k_comp_planes(const int8_t *__restrict__ comp, uint32_t n, uint32_t D, uint32_t bits, int32_t m,
                              uint32_t *__restrict__ planes, uint32_t *__restrict__ usum, uint32_t *status)
{
    const uint32_t row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const uint32_t lane = threadIdx.x & 31;
    if (row >= n) return;
    const uint32_t W32 = D / 32;
    const int8_t *c = comp + (size_t)row * D;
    uint32_t *dst = planes + (size_t)row * bits * W32;
    uint32_t sum = 0;
    bool bad = false;
    for (uint32_t w = 0; w < W32; ++w) {
        int32_t h = c[32 * w + lane];
        if (h < -m || h > m) {
            bad = true;
            h = 0;
        }
        const uint32_t u = (uint32_t)(h + m);
        sum += u;
        const uint32_t ch = w / MB_CW, cw = min(MB_CW, W32 - ch * MB_CW);
        for (uint32_t i = 0; i < bits; ++i) {
            const uint32_t word = __ballot_sync(0xFFFFFFFFu, (u >> i) & 1u);
            if (lane == i) dst[bits * MB_CW * ch + i * cw + (w - ch * MB_CW)] = word;
        }
    }
    sum = __reduce_add_sync(0xFFFFFFFFu, sum);
    if (lane == 0) usum[row] = sum;
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) hd_flag(status, HD_DEV_BAD_INPUT);
}

struct mb_args {
    const uint32_t *lib_planes, *lib_usum, *lib_orig;
    const uint32_t *q_planes, *q_usum;   // queries in input order
    const uint32_t *perm;
    const uint32_t *lo, *hi;
    const uint32_t *blk_lo, *blk_hi, *blk_nt, *item_start;
    uint32_t *meta;
    uint64_t *partial;
    uint32_t *status;
    uint32_t n_q, n_blocks, W32, bits, m, nst;
    uint64_t wait_ns;
    uint32_t stall;
};

// The popcount search of k_search_popc on bit planes: the same persistent
// work list, stage ring (nst buffers, one CTA barrier per step) and 4 x 4
// pairs per thread; per pair, b^2 plane pairs whose AND words are counted by
// the carry-save adder (one popcount per two words), weighted 2^(i+j).
template <int K>
__global__ void __launch_bounds__(THREADS, 1) k_search_popc_mb(mb_args a)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t bits = a.bits, pitch = mb_pitch(bits), stage_b = mb_stage_bytes(bits), nst = a.nst;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + nst * stage_b);
    __shared__ uint32_t s_item;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int qg = 2 * warp + (lane >> 4);
    const int rg = lane & 15;
    const uint32_t nchunks = (a.W32 + MB_CW - 1) / MB_CW;
    const uint32_t row_words = bits * a.W32;

    if (tid == 0) {
        for (uint32_t i = 0; i < nst; ++i) mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const uint32_t total_items = a.item_start[a.n_blocks];
    const uint32_t tpi = a.meta[0];
    uint32_t parity = 0;
    bool first_item = true;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(&a.meta[1], 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= total_items) break;

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
        const uint32_t row_end = a.blk_hi[b];

        uint32_t qlo[4], qhi[4], uq[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t s = q0 + qg + 16 * i;
            qlo[i] = s < a.n_q ? a.lo[s] : 0u;
            qhi[i] = s < a.n_q ? a.hi[s] : 0u;
            uq[i] = s < a.n_q ? a.q_usum[a.perm[s]] : 0u;
        }
        uint64_t best[4][K];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int t = 0; t < K; ++t) best[i][t] = KEY_NONE;
        uint32_t acc[4][4];   // P of pair (i, j) so far
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0;

        auto issue = [&](uint32_t st_step) {
            const uint32_t tile = t0 + st_step / nchunks, ch = st_step % nchunks;
            const uint32_t cw = min(MB_CW, a.W32 - ch * MB_CW);
            const uint32_t rb = bits * cw * 4;
            const uint32_t r0 = row_base + tile * BR;
            const uint32_t nr = min((uint32_t)BR, row_end - r0);
            const uint32_t sb = st_step % nst;
            uint8_t *stage = smem + sb * stage_b;
            if (lane == 0) mbar_expect_tx(&bar[sb], (nq + nr) * rb);
            __syncwarp();
            if (a.stall && first_item && st_step == 0) return;   // nothing completes this stage
            for (uint32_t x = lane; x < nq; x += 32)
                bulk_load(stage + x * pitch * 4, a.q_planes + (size_t)a.perm[q0 + x] * row_words + bits * MB_CW * ch,
                          rb, &bar[sb]);
            for (uint32_t x = lane; x < nr; x += 32)
                bulk_load(stage + (BQ + x) * pitch * 4, a.lib_planes + (size_t)(r0 + x) * row_words + bits * MB_CW * ch,
                          rb, &bar[sb]);
        };

        if (warp == 0)
            for (uint32_t p = 0; p + 1 < nst && p < steps; ++p) issue(p);
        uint32_t waited = 0;
        bool aborted = false;
        for (uint32_t s = 0; s < steps; ++s) {
            const uint32_t st = s % nst;
            const bool ok = mbar_wait(&bar[st], (parity >> st) & 1u, a.wait_ns);
            parity ^= 1u << st;
            ++waited;
            if (__syncthreads_or(!ok)) {
                aborted = true;
                break;
            }
            if (warp == 0 && s + nst - 1 < steps) issue(s + nst - 1);
            const uint32_t tile = t0 + s / nchunks, ch = s % nchunks;
            const uint32_t cw = min(MB_CW, a.W32 - ch * MB_CW);
            const uint32_t *qs = reinterpret_cast<const uint32_t *>(smem + st * stage_b);
            const uint32_t *rs = qs + BQ * pitch;
            // per plane pair, the chunk's AND words go through the carry-save
            // adder of k_search_popc (one popcount per two words), and the
            // pair's count enters P with weight 2^(pi + pj)
#pragma unroll 1
            for (uint32_t pi = 0; pi < bits; ++pi) {
#pragma unroll 1
                for (uint32_t pj = 0; pj < bits; ++pj) {
                    uint32_t ones[4][4], cnt[4][4];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) ones[i][j] = cnt[i][j] = 0;
                    for (uint32_t w = 0; w < cw; w += 4) {
                        uint4 qv[4], rv[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            qv[i] = *reinterpret_cast<const uint4 *>(qs + (qg + 16 * i) * pitch + pi * cw + w);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            rv[j] = *reinterpret_cast<const uint4 *>(rs + (rg + 16 * j) * pitch + pj * cw + w);
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                csa2(ones[i][j], cnt[i][j], qv[i].x & rv[j].x, qv[i].y & rv[j].y);
                                csa2(ones[i][j], cnt[i][j], qv[i].z & rv[j].z, qv[i].w & rv[j].w);
                            }
                    }
                    const uint32_t sh = pi + pj;
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] += (cnt[i][j] + (uint32_t)__popc(ones[i][j])) << sh;
                }
            }
            if (ch == nchunks - 1) {
                const uint32_t r0 = row_base + tile * BR;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t row = r0 + rg + 16 * j;
                    const bool in = row < row_end;
                    const uint32_t o = in ? __ldg(a.lib_orig + row) : 0u;
                    const uint32_t ur = in ? __ldg(a.lib_usum + row) : 0u;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const uint32_t kd = a.m * (uq[i] + ur) - acc[i][j];   // D m^2 - S >= 0
                        acc[i][j] = 0;
                        if (row >= qlo[i] && row < qhi[i]) {
                            const uint64_t key = ((uint64_t)kd << 32) | o;
                            if (key < best[i][K - 1]) topk_insert<K>(best[i], key);
                        }
                    }
                }
            }
        }
        if (aborted) {
            if (tid == 0) hd_flag(a.status, HD_DEV_TIMEOUT);
            const uint32_t in_flight = min(steps, waited + nst - 2);
            for (uint32_t s = waited; s < in_flight; ++s) {
                mbar_wait(&bar[s % nst], (parity >> (s % nst)) & 1u, a.wait_ns);
                parity ^= 1u << (s % nst);
            }
            return;
        }
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
        first_item = false;
    }
}

// Final merge of the items' lists into the caller's order, as k_merge, with
// the dot-product score S = bias - key distance (INT32_MIN for a missing slot).
template <int K>
__global__ void k_merge_score(const uint64_t *__restrict__ partial, const uint32_t *__restrict__ item_start,
                              uint32_t bq, const uint32_t *__restrict__ perm, uint32_t n_q, uint32_t k, uint32_t bias,
                              uint32_t *__restrict__ out_idx, int32_t *__restrict__ out_score)
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
            out_score[(size_t)q * k + t] = none ? INT32_MIN : (int32_t)(bias - (uint32_t)(best[t] >> 32));
        }
    }
}

template <int K>
hd_status run_mb(const hd_library *lib, const int8_t *q_comp, const double *q_mz, const uint8_t *q_z, uint32_t n_q,
                 const hd_qwin &win, uint32_t k, uint32_t *out_idx, int32_t *out_score, cudaStream_t s)
{
    const uint32_t bits = lib->bits, W32 = lib->dim / 32, m = hd_comp_max(bits);
    const uint32_t stage_b = mb_stage_bytes(bits);
    const uint32_t nst = 3 * stage_b + 64 <= 227u * 1024u ? 3u : 2u;
    const uint32_t smem_b = nst * stage_b + 64;
    const uint32_t n_blocks = (n_q + BQ - 1) / BQ;
    int occ = 0;
    HD_CUDA_TRY(cudaFuncSetAttribute(k_search_popc_mb<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
    HD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_search_popc_mb<K>, THREADS, smem_b));
    if (occ < 1) return hd_fail(HD_ERR_UNSUPPORTED, "multi-bit popcount kernel does not fit on this GPU");
    const uint32_t grid = (uint32_t)(lib->num_sms * occ);
    const uint32_t target_items = 8 * grid;

    auto carve = [&](hd_arena &ar, uint32_t **perm, uint32_t **lo, uint32_t **hi, uint32_t **blo, uint32_t **bhi,
                     uint32_t **bnt, uint32_t **ist, uint32_t **meta, uint64_t **part, uint32_t **qp,
                     uint32_t **qu) {
        *perm = ar.take<uint32_t>(n_q);
        *lo = ar.take<uint32_t>(n_q);
        *hi = ar.take<uint32_t>(n_q);
        *blo = ar.take<uint32_t>(n_blocks);
        *bhi = ar.take<uint32_t>(n_blocks);
        *bnt = ar.take<uint32_t>(n_blocks);
        *ist = ar.take<uint32_t>(n_blocks + 1);
        *meta = ar.take<uint32_t>(4);
        *part = ar.take<uint64_t>((size_t)(target_items + n_blocks) * BQ * K);
        *qp = ar.take<uint32_t>((size_t)n_q * bits * W32);
        *qu = ar.take<uint32_t>(n_q);
    };
    uint32_t *perm, *lo, *hi, *blo, *bhi, *bnt, *ist, *meta, *qp, *qu;
    uint64_t *part;
    hd_arena plan;
    carve(plan, &perm, &lo, &hi, &blo, &bhi, &bnt, &ist, &meta, &part, &qp, &qu);
    hd_sort_charge_mz(q_mz, q_z, win.cls, n_q, nullptr, plan, s);
    hd_arena ar;
    if (cudaMallocAsync((void **)&ar.base, plan.used, s) != cudaSuccess) {
        cudaGetLastError();
        return hd_fail(HD_ERR_OOM, "multi-bit popcount search: scratch allocation failed");
    }
    carve(ar, &perm, &lo, &hi, &blo, &bhi, &bnt, &ist, &meta, &part, &qp, &qu);
    hd_count_launches(1), k_comp_planes<<<hd_ceil_div(n_q, 8), 256, 0, s>>>(q_comp, n_q, lib->dim, bits, (int32_t)m, qp,
                                                                             qu, lib->status.dev);
    hd_sort_charge_mz(q_mz, q_z, win.cls, n_q, perm, ar, s);
    hd_count_launches(1), k_windows<<<hd_ceil_div(n_q, 256), 256, 0, s>>>(lib->mz, lib->charge_start, q_mz, q_z, perm,
                                                                        n_q, win, lo, hi);
    hd_count_launches(1), k_worklist<<<1, 1024, 0, s>>>(lo, hi, n_q, BQ, BR, n_blocks, target_items, blo, bhi, bnt,
                                                        ist, meta);
    mb_args ma{lib->x_planes, lib->usum, lib->orig, qp, qu, perm, lo, hi, blo, bhi, bnt, ist, meta, part,
               lib->status.dev, n_q, n_blocks, W32, bits, m, nst, hd_wait_limit(lib),
               hd_take_injected_stall(lib) ? 1u : 0u};
    {
        hd_prof_scope timed(HD_KERNEL_SEARCH, s);
        hd_count_launches(1), k_search_popc_mb<K><<<grid, THREADS, smem_b, s>>>(ma);
    }
    hd_count_launches(1), k_merge_score<K><<<hd_ceil_div(n_q, 128), 128, 0, s>>>(part, ist, BQ, perm, n_q, k,
                                                                             lib->dim * m * m, out_idx, out_score);
    HD_CUDA_TRY(cudaGetLastError());
    HD_CUDA_TRY(cudaFreeAsync(ar.base, s));
    return HD_OK;
}

}  // namespace

hd_status hd_library_planes(hd_library *lib, cudaStream_t s)
{
    if (lib->x_planes || lib->n == 0) return HD_OK;
    const uint32_t W32 = lib->dim / 32;
    if (cudaMalloc(&lib->x_planes, (size_t)lib->n * lib->bits * W32 * 4) != cudaSuccess ||
        cudaMalloc(&lib->usum, (size_t)lib->n * 4) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(lib->x_planes);
        cudaFree(lib->usum);
        lib->x_planes = nullptr;
        lib->usum = nullptr;
        return hd_fail(HD_ERR_OOM, "hd_library_prepare: bit-plane allocation failed");
    }
    hd_count_launches(1), k_comp_planes<<<hd_ceil_div(lib->n, 8), 256, 0, s>>>(
        lib->comp, lib->n, lib->dim, lib->bits, (int32_t)hd_comp_max(lib->bits), lib->x_planes, lib->usum,
        lib->status.dev);
    HD_CUDA_TRY(cudaGetLastError());
    return HD_OK;
}

hd_status hd_search_popc_dot_run(const hd_library *lib, const int8_t *q_comp, const double *q_mz,
                                 const uint8_t *q_charge, uint32_t n_q, const hd_qwin &win, uint32_t k,
                                 uint32_t *out_idx, int32_t *out_score, cudaStream_t s)
{
    if (k <= 1) return run_mb<1>(lib, q_comp, q_mz, q_charge, n_q, win, k, out_idx, out_score, s);
    if (k <= 8) return run_mb<8>(lib, q_comp, q_mz, q_charge, n_q, win, k, out_idx, out_score, s);
    return run_mb<16>(lib, q_comp, q_mz, q_charge, n_q, win, k, out_idx, out_score, s);
}

// ----------------------------------------------- integer-pipe microbenchmarks
// Sixteen independent chains per thread, 32 warps per SM.  k_peak_popc: one
// population count of a 32-bit word per step (plus the XOR that makes the
// word and the add that keeps the count, both on the ALU pipes, which issue
// four times as many per clock): the popcount unit's rate.  k_peak_lop3: one
// three-input LOP3 per step: the integer logic pipe's rate.
namespace {
constexpr uint32_t PEAK_ALU_THREADS = 256;
__global__ void __launch_bounds__(PEAK_ALU_THREADS) k_peak_popc(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    uint32_t v[16], acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        v[i] = (seed + (blockIdx.x * blockDim.x + threadIdx.x) * 16u + (uint32_t)i) * 0x9E3779B9u;
        acc[i] = 0u;
    }
#pragma unroll 4
    for (uint32_t it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] += __popc(v[i] ^ it);
    uint32_t t = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) t += acc[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = t;
}
__global__ void __launch_bounds__(PEAK_ALU_THREADS) k_peak_lop3(uint32_t iters, uint32_t seed, uint32_t *sink)
{
    uint32_t v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = (seed + (blockIdx.x * blockDim.x + threadIdx.x) * 16u + (uint32_t)i) * 0x9E3779B9u;
#pragma unroll 4
    for (uint32_t it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < 16; ++i)
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(v[i]) : "r"(v[(i + 1) & 15]), "r"(v[(i + 5) & 15]));
    uint32_t t = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) t ^= v[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = t;
}
}  // namespace

hd_status hd_peak_alu_run(bool popc, uint32_t launches, hd_peak_result *out)
{
    int dev = 0, n_sms = 0;
    HD_CUDA_TRY(cudaGetDevice(&dev));
    HD_CUDA_TRY(cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev));
    const uint32_t grid = (uint32_t)n_sms * 4u;   // 4 CTAs of 8 warps per SM
    const uint32_t iters = popc ? 8192u : 16384u;
    const uint64_t ops = (uint64_t)grid * PEAK_ALU_THREADS * iters * 16u;
    uint32_t *sink = nullptr;
    HD_CUDA_TRY(cudaMalloc(&sink, (size_t)grid * PEAK_ALU_THREADS * sizeof(uint32_t)));
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<double> ms;
    hd_status st = HD_OK;
    for (uint32_t r = 0; r <= launches; ++r) {   // launch 0 warms up
        cudaEventRecord(e0, s);
        hd_count_launches(1);
        if (popc) k_peak_popc<<<grid, PEAK_ALU_THREADS, 0, s>>>(iters, r, sink);
        else k_peak_lop3<<<grid, PEAK_ALU_THREADS, 0, s>>>(iters, r, sink);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            st = hd_cuda_fail(e, "integer peak kernel");
            break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (r > 0) ms.push_back(t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(sink);
    if (st != HD_OK) return st;
    std::sort(ms.begin(), ms.end());
    out->ops_per_launch = ops;
    out->ms_best = ms.front();
    out->best_per_s = (double)ops / (ms.front() * 1e-3);
    out->median_per_s = (double)ops / (ms[ms.size() / 2] * 1e-3);
    out->sms = (uint32_t)n_sms;
    out->launches = (uint32_t)ms.size();
    return HD_OK;
}
