// search_mma.cu -- open-modification Hamming search (Section 3.4) on the
// 5th-generation tensor cores (tcgen05), exact.
//
// Bits become bipolar values (bit 0 -> +1, bit 1 -> -1) stored as e2m1 (4 bits,
// 0x2 / 0xA, two per byte), e4m3 (0x38 / 0xB8) or bf16 (0x3F80 / 0xBF80).  For
// a query x and a reference y the tensor core computes S = sum_d x_d y_d =
// D - 2 dist(x, y) with fp32 accumulation in tensor memory.  Every product is
// +-1 and every partial sum an integer of magnitude <= D <= 32768 < 2^24, so
// the sum is exact and dist = (D - S) / 2 matches the popcount form bit for
// bit.  Multi-bit components (integers in [-m, m], Section 4.3) use the same
// kernels with the key distance D m^2 - S; their partial sums stay below
// D m^2 < 2^24.
//
// Two kernels share the warp roles (one persistent CTA per SM):
//   warp 0      TMA producer: 2-D tensor loads of 128-component K-slices of a
//               query block (A: 128 rows) and a reference tile into a ring of
//               stages, 128B-swizzled for the MMA descriptors;
//   warp 1      allocates 512 TMEM columns and issues tcgen05.mma (32
//               components of K per instruction) into one of two accumulator
//               buffers, committing stages and tiles to mbarriers;
//   warps 2..5  epilogue: tcgen05.ld of the finished accumulator, one query
//               row per thread; per 32 columns a candidate mask (window bits
//               and one float compare per column against the score that could
//               still enter the row's top-k, bounded by the query's running
//               top-k at the work item's start), then a rolled loop over the
//               candidates into the top-k of (dist, input index) keys; the
//               buffer is handed back while the next tile is accumulated in
//               the other one.
// k_search_mma: 192 threads (4 epilogue warps), M = 128, N = 256 per CTA, 4
// stages of 48 KB, one CTA per SM with no cluster; every load goes to the
// issuing CTA's own shared memory.
// k_search_mma2 (default): 192 threads (HD_MMA2_EPI_WARPS = 8 splits each
// quarter's columns over two warps), SM pairs, tcgen05.mma.cta_group::2 with
// M = 256, N = 256 issued by the even CTA; each CTA stages its own query block
// and half of the tile, 6 stages of 32 KB.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "hd_internal.cuh"
#include "search_common.cuh"

void hd_exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint32_t n, hd_arena &arena,
                           cudaStream_t s);

namespace {

using namespace hd_search;

#ifndef HD_MMA_TN
#define HD_MMA_TN 256
#endif
#ifndef HD_MMA_STAGES
#define HD_MMA_STAGES 4
#endif
// Operand formats of +-1: FMT_BF16 (kind::f16, 2 bytes), FMT_E4M3 (kind::f8f6f4,
// 1 byte), FMT_E2M1 (kind::f8f6f4, 4 bits packed in HBM and unpacked by the TMA
// into 16-byte shared-memory containers of 16 values, so the shared-memory
// image of a K-chunk is that of e4m3 while HBM and L2 carry half the bytes).
// FMT_MXF4: the e2m1 rows of FMT_E2M1, kept packed in shared memory and
// scored by the block-scaled kind::mxf4 (SM-pair form only).
constexpr int FMT_BF16 = 0, FMT_E4M3 = 1, FMT_E2M1 = 2, FMT_MXF4 = 3;
// instruction-descriptor A/B format code of each operand format
__host__ __device__ constexpr uint32_t fmt_code(int fmt) { return fmt == FMT_BF16 ? 1u : (fmt == FMT_E4M3 ? 0u : 5u); }
// Transaction bytes a load of `smem_bytes` of operand counts on its mbarrier:
// the bytes read from global memory, half the unpacked footprint for e2m1.
__host__ __device__ constexpr uint32_t tx_bytes(int fmt, uint32_t smem_bytes)
{
    return fmt == FMT_E2M1 ? smem_bytes / 2 : smem_bytes;
}
constexpr int TM = 128;                 // queries per block (MMA M)
constexpr int TN = HD_MMA_TN;           // reference rows per tile (MMA N)
constexpr int KB = 128;                 // bytes of K per stage (one 128B swizzle atom)
constexpr int STAGES = HD_MMA_STAGES;
constexpr int THREADS = 192;
constexpr uint32_t A_BYTES = TM * KB;
constexpr uint32_t B_BYTES = TN * KB;
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /* align */ + 256 /* barriers */;
constexpr uint32_t TMEM_COLS = 2 * TN;
// Epilogue warps of the pair kernel: EPI2_SPLIT per tensor-memory lane
// quarter, each scoring 1/EPI2_SPLIT of the 256 columns of its 32 query rows.
// With the compact group scoring one warp per quarter keeps up with the MMAs
// at D = 4096 and leaves the issue slots to the producer and MMA warps.
#ifndef HD_MMA2_EPI_WARPS
#define HD_MMA2_EPI_WARPS 4
#endif
constexpr int EPI2_WARPS = HD_MMA2_EPI_WARPS;
constexpr int EPI2_SPLIT = EPI2_WARPS / 4;
static_assert(EPI2_WARPS % 4 == 0 && (TN / 32) % EPI2_SPLIT == 0, "epilogue split");
static_assert(TN % 32 == 0 && TN <= 256 && (TMEM_COLS & (TMEM_COLS - 1)) == 0, "tile shape");
static_assert(STAGES * STAGE_BYTES + 1280 <= 232448, "shared memory");

// ------------------------------------------------------------ tcgen05 PTX
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int FMT>
__device__ __forceinline__ void mma_issue(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate)
{
    if (FMT != FMT_BF16)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
            : "memory");
}

// Arrives on `bar` once every tcgen05.mma issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// 32 lanes x 32 consecutive fp32 columns: thread i of the warp gets lane
// (warp % 4) * 32 + i, columns [col, col + 32).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int32_t x, int32_t y,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;               // version
    d |= (uint64_t)2 << 61;               // 128B swizzle
    return d;
}

// Instruction descriptor: fp32 accumulator, A/B e4m3 or e2m1 (kind::f8f6f4) or
// bf16 (kind::f16), both K-major, M = 128, N = 256.
template <int FMT>
__host__ __device__ constexpr uint32_t instr_desc()
{
    return (1u << 4) | (fmt_code(FMT) << 7) | (fmt_code(FMT) << 10) | ((uint32_t)(TN >> 3) << 17) |
           ((uint32_t)(TM >> 4) << 24);
}

struct mma_args {
    const uint32_t *lib_orig;
    const uint32_t *lo, *hi;                    // windows, sorted query order
    const uint32_t *blk_t0, *blk_t1;            // absolute tile range of each query block
    const uint32_t *pair_start;                 // [n_pairs + 1] first item of (super-group, block)
    uint64_t *top;                              // [n_q][K] running top-k, sorted query order
    uint32_t *locks;                            // [n_blocks] merge locks
    uint32_t *status;
    uint32_t n_q, n_blocks, n_pairs, tg, sg, dim, row_bytes;
    uint64_t wait_ns;      // bound of every device wait
    uint32_t stall;        // test hook: drop the first stage load
    // key distance (bias - S) >> shift of a score S: binary rows (D - S) / 2,
    // the Hamming distance; multi-bit rows D m^2 - S
    uint32_t bias, shift;
};

// Work item -> (query block, absolute tile range [t0, t1)).  Items are
// numbered super-group-major: pair p = G * n_blocks + b holds the groups of
// TG tiles of block b that fall in super-group G (SG groups), so the CTAs
// running at any moment share one slice of the library through L2.
__device__ __forceinline__ void item_range(const mma_args &a, uint32_t item, uint32_t &b, uint32_t &t0,
                                           uint32_t &t1)
{
    uint32_t lo = 0, hi = a.n_pairs;
    while (hi - lo > 1) {
        const uint32_t m = (lo + hi) >> 1;
        if (a.pair_start[m] <= item) lo = m; else hi = m;
    }
    const uint32_t G = lo / a.n_blocks;
    b = lo % a.n_blocks;
    const uint32_t g = max(a.blk_t0[b] / a.tg, G * a.sg) + (item - a.pair_start[lo]);
    t0 = max(a.blk_t0[b], g * a.tg);
    t1 = min(a.blk_t1[b], (g + 1) * a.tg);
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Bit e set for the columns e of a 32-column group starting at reference row
// c0 that lie in the row window [lo, lo + span).
__device__ __forceinline__ uint32_t window_bits(uint32_t lo, uint32_t span, uint32_t c0)
{
    const int64_t b0 = max((int64_t)0, min((int64_t)32, (int64_t)lo - (int64_t)c0));
    const int64_t b1 = max((int64_t)0, min((int64_t)32, (int64_t)lo + (int64_t)span - (int64_t)c0));
    if (b1 <= b0) return 0u;
    const uint32_t hi = b1 == 32 ? 0xFFFFFFFFu : (1u << b1) - 1u;
    return hi & ~((1u << b0) - 1u);
}

// v[e] for a run-time e in 0..G-1 (G = 32 or 16), by a tree of selects on
// the bits of e (keeps v in registers).
template <int G>
__device__ __forceinline__ uint32_t pick(const uint32_t (&v)[G], uint32_t e)
{
    uint32_t w16[16], w8[8], w4[4], w2[2];
#pragma unroll
    for (int i = 0; i < 16; ++i) w16[i] = G == 32 ? ((e & 16u) ? v[(i + 16) % G] : v[i]) : v[i % G];
#pragma unroll
    for (int i = 0; i < 8; ++i) w8[i] = (e & 8u) ? w16[i + 8] : w16[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) w4[i] = (e & 4u) ? w8[i + 4] : w8[i];
#pragma unroll
    for (int i = 0; i < 2; ++i) w2[i] = (e & 2u) ? w4[i + 2] : w4[i];
    return (e & 1u) ? w2[1] : w2[0];
}

// Scores one group of G (32, or 16 for the last columns of a 240-column
// tile) columns of a query row's accumulator (S in fp32, exact integers)
// into its running top-k: key distance (bias - S) >> shift, window [lo, lo +
// span) of library rows, column e = reference row c0 + e.  One float compare
// per column builds the candidate mask, and the candidates go through a loop
// that is not unrolled, which keeps the code small.
template <int K, int G = 32>
__device__ __forceinline__ void score_group(const uint32_t (&v)[G], uint32_t c0, uint32_t lo, uint32_t span,
                                            uint32_t bias, uint32_t shift, const uint32_t *__restrict__ lib_orig,
                                            uint64_t seed, uint64_t (&best)[K])
{
    const uint32_t wm = window_bits(lo, span, c0) & (G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u));
    if (!wm) return;
    // a key enters only below the list's last key and below `seed`, the last
    // key of the query's running top-k when the work item started (that list
    // only improves, so nothing at or above it can reach the result).
    // (bias - S) >> shift <= thr  <=>  S >= bias - (((thr + 1) << shift) - 1); an
    // empty list (thr = ~0) admits every column
    const uint32_t thr = (uint32_t)(min(best[K - 1], seed) >> 32);
    const float smin = thr == 0xFFFFFFFFu ? -INFINITY : (float)((int)bias - (int)(((thr + 1u) << shift) - 1u));
    // once the list is seeded almost no group holds a candidate: one maximum over
    // the group decides before any per-column mask is built
    float mx = __uint_as_float(v[0]);
#pragma unroll
    for (int e = 1; e < G; ++e) mx = fmaxf(mx, __uint_as_float(v[e]));
    if (mx < smin) return;
    uint32_t cand = 0;
#pragma unroll
    for (int e = 0; e < G; ++e) cand |= (uint32_t)(__uint_as_float(v[e]) >= smin) << e;
    cand &= wm;
    while (cand) {
        const int e = __ffs(cand) - 1;
        cand &= cand - 1u;
        const int sc = __float2int_rn(__uint_as_float(pick<G>(v, (uint32_t)e)));
        const uint32_t x = (uint32_t)((int)bias - sc);
        const uint64_t key = ((uint64_t)(x >> shift) << 32) | __ldg(lib_orig + c0 + e);
        if (key < min(best[K - 1], seed)) topk_insert<K>(best, key);
    }
}
__device__ __forceinline__ void epi_bar_n(uint32_t n) { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }

// One CTA per SM: each CTA stages its own query block and whole reference
// tiles, and its MMAs commit to its own barriers.
template <int K, int FMT>
__global__ void __launch_bounds__(THREADS, 1)
k_search_mma(const __grid_constant__ CUtensorMap qmap, const __grid_constant__ CUtensorMap lmap, mma_args a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *acc_full = empty + STAGES;
    uint64_t *acc_empty = acc_full + 2;
    uint64_t *drain = acc_empty + 2;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort, s_lock_ok;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], 128);
        }
        mbar_init(drain, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(&s_tmem, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t cid = blockIdx.x, ncl = gridDim.x;

    const uint32_t total = a.pair_start[a.n_pairs];
    const uint32_t nchunks = a.row_bytes / KB;
    volatile int *abort_flag = &s_abort;
    auto give_up = [&]() {
        *abort_flag = 1;
        hd_flag(a.status, HD_DEV_TIMEOUT);
    };

    if (warp == 0) {
        // ------------------------------------------------------- producer
        if (lane == 0) {
            uint32_t it = 0;
            for (uint32_t item = cid; item < total && !*abort_flag; item += ncl) {
                uint32_t b, t0, t1;
                item_range(a, item, b, t0, t1);
                for (uint32_t t = t0; t < t1 && !*abort_flag; ++t) {
                    const int32_t r0 = (int32_t)(t * TN);
                    for (uint32_t c = 0; c < nchunks; ++c, ++it) {
                        const uint32_t s = it % STAGES, ph = (it / STAGES) & 1u;
                        if (!mbar_wait(&empty[s], ph ^ 1u, a.wait_ns)) { give_up(); break; }
                        uint8_t *sa = smem + s * STAGE_BYTES, *sb = sa + A_BYTES;
                        mbar_expect_tx(&full[s], tx_bytes(FMT, STAGE_BYTES));
                        if (a.stall && it == 0) continue;   // nothing ever completes this stage
                        tma_load_2d(sa, &qmap, (int32_t)(c * KB), (int32_t)(b * TM), &full[s]);
                        tma_load_2d(sb, &lmap, (int32_t)(c * KB), r0, &full[s]);
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ----------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = instr_desc<FMT>();
            uint32_t it = 0, acc_it = 0;
            for (uint32_t item = cid; item < total && !*abort_flag; item += ncl) {
                uint32_t b, t0, t1;
                item_range(a, item, b, t0, t1);
                for (uint32_t t = t0; t < t1 && !*abort_flag; ++t, ++acc_it) {
                    const uint32_t buf = acc_it & 1u, aph = (acc_it >> 1) & 1u;
                    if (!mbar_wait(&acc_empty[buf], aph ^ 1u, a.wait_ns)) { give_up(); break; }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem + buf * TN;
                    bool ok = true;
                    for (uint32_t c = 0; c < nchunks; ++c, ++it) {
                        const uint32_t s = it % STAGES, ph = (it / STAGES) & 1u;
                        if (!mbar_wait(&full[s], ph, a.wait_ns)) { give_up(); ok = false; break; }
                        tc_fence_after();
                        const uint32_t sa = smem_addr(smem + s * STAGE_BYTES), sb = sa + A_BYTES;
                        const uint64_t da = sw128_desc(sa), db = sw128_desc(sb);
#pragma unroll
                        for (uint32_t j = 0; j < KB / 32; ++j)   // 32 bytes of K per instruction
                            mma_issue<FMT>(d_tmem, da + 2 * j, db + 2 * j, idesc, (c | j) != 0);
                        mma_commit(&empty[s]);
                    }
                    if (!ok) break;
                    mma_commit(&acc_full[buf]);
                }
            }
            // every issued MMA has finished before TMEM is released
            mma_commit(drain);
            mbar_wait(drain, 0, a.wait_ns);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------- epilogue
        const uint32_t quarter = warp & 3;              // TMEM lanes this warp may read
        const uint32_t row = quarter * 32 + lane;       // query row within the block
        const uint32_t lane_addr = (quarter * 32) << 16;
        const bool leader = threadIdx.x == 64;
        uint32_t acc_it = 0;
        for (uint32_t item = cid; item < total && !*abort_flag; item += ncl) {
            uint32_t b, t0, t1;
            item_range(a, item, b, t0, t1);
            const uint32_t sb_ = b;                  // this CTA's query block
            const uint32_t sq = sb_ * TM + row;
            const uint32_t lo = sq < a.n_q ? a.lo[sq] : 0u, hi = sq < a.n_q ? a.hi[sq] : 0u;
            // last key of the query's running top-k (merged from its finished items)
            const uint64_t seed = sq < a.n_q ? (uint64_t)__ldcg(reinterpret_cast<const unsigned long long *>(
                                                   a.top + (size_t)sq * K + (K - 1)))
                                             : KEY_NONE;
            const uint32_t span = hi > lo ? hi - lo : 0u;
            uint64_t best[K];
#pragma unroll
            for (int i = 0; i < K; ++i) best[i] = KEY_NONE;
            bool ok = true;
            for (uint32_t t = t0; t < t1; ++t, ++acc_it) {
                const uint32_t buf = acc_it & 1u, aph = (acc_it >> 1) & 1u;
                if (!mbar_wait(&acc_full[buf], aph, a.wait_ns)) { give_up(); ok = false; break; }
                tc_fence_after();
                const uint32_t r0 = t * TN;
#pragma unroll 1
                for (uint32_t cg = 0; cg < TN / 32; ++cg) {
                    uint32_t v[32];
                    tmem_ld32(tmem + lane_addr + buf * TN + cg * 32, v);
                    tmem_ld_wait();
                    score_group<K>(v, r0 + cg * 32, lo, span, a.bias, a.shift, a.lib_orig, seed, best);
                }
                tc_fence_before();
                mbar_arrive(&acc_empty[buf]);
            }
            // merge into the block's running top-k under its lock (bounded spin)
            epi_bar();
            if (leader) {
                int got = 0;
                if (ok && !*abort_flag) {
                    const uint64_t w0 = hd_globaltimer_ns();
                    for (uint32_t i = 0;; ++i) {
                        if (atomicCAS(&a.locks[sb_], 0u, 1u) == 0u) { got = 1; break; }
                        if ((i & 63u) == 0 && hd_globaltimer_ns() - w0 > a.wait_ns) { give_up(); break; }
                    }
                    __threadfence();
                }
                s_lock_ok = got;
            }
            epi_bar();
            const bool locked = s_lock_ok != 0;
            if (locked) {
                if (sq < a.n_q) {
                    unsigned long long *g = reinterpret_cast<unsigned long long *>(a.top + (size_t)sq * K);
                    uint64_t cur[K];
#pragma unroll
                    for (int i = 0; i < K; ++i) cur[i] = __ldcg(g + i);
                    topk_merge<K>(cur, best);
#pragma unroll
                    for (int i = 0; i < K; ++i) __stcg(g + i, (unsigned long long)cur[i]);
                }
                __threadfence();
            }
            epi_bar();
            if (leader && locked) atomicExch(&a.locks[sb_], 0u);
            if (!locked) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    // after a give-up, loads this CTA issued before it stopped may still be
    // landing in its shared memory: a bounded pause (200 us) lets them complete
    if (threadIdx.x == 0 && *abort_flag) {
        const uint64_t w0 = hd_globaltimer_ns();
        while (hd_globaltimer_ns() - w0 < 200000ull) __nanosleep(1000);
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// ------------------------------------------------------------- 2-SM form
// A cluster of two CTAs on an SM pair (cluster ranks 0 and 1) issues one
// tcgen05.mma.cta_group::2 of M = 256, N = 256 from rank 0: each CTA holds
// the 128 query rows of its own block (A) and 128 of the tile's 256
// reference rows (B; rank 0 rows 0..127, rank 1 rows 128..255) in every
// stage, and its tensor memory receives the 128 x 256 scores of its queries.
// Per SM the tensor core reads half as many B bytes from shared memory as in
// the 1-SM form, and the TMA writes half as many: at M = 128, N = 256 the two
// together exceed what shared memory delivers per clock.
constexpr uint32_t B2_BYTES = (TN / 2) * KB;
constexpr uint32_t STAGE2_BYTES = A_BYTES + B2_BYTES;
#ifndef HD_MMA2_STAGES
#define HD_MMA2_STAGES 6
#endif
#ifndef HD_MMA2_BUFS
#define HD_MMA2_BUFS 2
#endif
constexpr int STAGES2 = HD_MMA2_STAGES;
constexpr int BUFS2 = HD_MMA2_BUFS;                 // accumulator buffers in tensor memory
constexpr uint32_t TMEM2_COLS = BUFS2 * TN;
// Optional B2_BYTES of slack after the ring (HD_MMA2_PAD=1) would keep a
// 256-row B read of the last stage inside the allocation.  Off: each CTA of
// the pair supplies 128 rows of B, which exact parity of both tensor-core
// forms against the popcount form confirms.
#ifndef HD_MMA2_PAD
#define HD_MMA2_PAD 0
#endif
constexpr uint32_t PAD2_BYTES = HD_MMA2_PAD ? B2_BYTES : 0u;
constexpr uint32_t SMEM2_BYTES = STAGES2 * STAGE2_BYTES + PAD2_BYTES + 1024 + 256;
static_assert(SMEM2_BYTES <= 232448, "shared memory (2-SM form)");
static_assert((BUFS2 == 1 || BUFS2 == 2) && TN == 256, "2-SM form: N = 256, one or two accumulators");

__device__ __forceinline__ void tmem_alloc2(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish2()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc2(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

template <int FMT>
__device__ __forceinline__ void mma_issue2(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                           uint32_t accumulate)
{
    if (FMT != FMT_BF16)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
            : "memory");
}

// Arrives on `bar` (same offset in every CTA of `mask`) once the pair's
// tcgen05.mma issued so far by this thread are done.
__device__ __forceinline__ void mma_commit2_mc(uint64_t *bar, uint16_t mask)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_addr(bar)),
        "h"(mask)
        : "memory");
}
__device__ __forceinline__ void mma_commit2(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// Address of this CTA's shared variable `p` in the shared memory of cluster CTA `rank`.
__device__ __forceinline__ uint32_t cluster_addr(const void *p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t caddr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}
__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t caddr)
{
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(caddr) : "memory");
    return v;
}

// 2-D tensor load into this CTA's shared memory whose bytes are counted on
// an mbarrier of either CTA of the pair (`bar` is a cluster address).
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, int32_t x, int32_t y,
                                                 uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// L2 eviction priority of the pair's operand loads: 0 default, 1 evict-first,
// 2 evict-last.  A query block is re-read for every reference tile of its
// work item and the running pairs' blocks nearly fill L2; a reference tile is
// read by the few pairs on the same tile group at about the same time.  Query
// blocks evict-last and reference tiles evict-first keep the blocks resident
// (full workload: 83 -> 77 ms).
#ifndef HD_MMA2_HINT_A
#define HD_MMA2_HINT_A 2
#endif
#ifndef HD_MMA2_HINT_B
#define HD_MMA2_HINT_B 1
#endif
#ifndef HD_MMA2_HINT_FRAC
#define HD_MMA2_HINT_FRAC 1.0
#endif
__device__ __forceinline__ uint64_t l2_policy(int kind)
{
    uint64_t p = 0;
    const float frac = HD_MMA2_HINT_FRAC;
    if (kind == 1) asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, %1;" : "=l"(p) : "f"(frac));
    if (kind == 2) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, %1;" : "=l"(p) : "f"(frac));
    return p;
}
__device__ __forceinline__ void tma_load_2d_pair_hint(void *dst, const CUtensorMap *map, int32_t x, int32_t y,
                                                      uint32_t bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(bar), "l"(policy)
        : "memory");
}

// M = 256 (the pair), N = 256.
template <int FMT>
__host__ __device__ constexpr uint32_t instr_desc2()
{
    return (1u << 4) | (fmt_code(FMT) << 7) | (fmt_code(FMT) << 10) | ((uint32_t)(TN >> 3) << 17) |
           ((uint32_t)((2 * TM) >> 4) << 24);
}

// ------------------------------------------------ block-scaled fp4 (kind::mxf4)
// e2m1 operands packed two per byte in shared memory as in HBM, scored by the
// block-scaled tcgen05.mma kind::mxf4: 64 components of K per instruction and
// one ue8m0 scale factor per 32 components of a row, every one 1.0 (0x7F), so
// S = sum_d x_d y_d as before.  N = 240 lets two accumulators and the
// scale factors share the 512 tensor-memory columns:
//   [0, 240) accumulator 0, [240, 256) the scale factors of A and B (every
//   one 1.0, so both operands read the same columns),
//   [256, 496) accumulator 1, [496, 512) unused (also filled with 1.0).
// Accumulators and tensor-memory loads stay on 32-column boundaries.
constexpr int TN_MX = 240;
constexpr uint32_t MX_SF_COL = 240, MX_BUF1_COL = 256, MX_SPARE_COL = 496;
constexpr uint32_t B2MX_BYTES = (TN_MX / 2) * KB;   // 120 reference rows of 128 bytes (256 components)

// Block-scaled instruction descriptor: B scale-factor id 0 (bits 4-5), A and
// B e2m1 (code 1 of kind::mxf4, bits 7 and 10), both K-major, N >> 3 at bit
// 17, ue8m0 scale factors (bit 23), M >> 4 at bit 24, A scale-factor id 0
// (bits 29-30), dense K = 64 (bit 31 clear).
__host__ __device__ constexpr uint32_t instr_desc_mxf4()
{
    return (1u << 7) | (1u << 10) | ((uint32_t)(TN_MX >> 3) << 17) | (1u << 23) | ((uint32_t)((2 * TM) >> 4) << 24);
}

__device__ __forceinline__ void mma_issue2_mxf4(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                                uint32_t sfa, uint32_t sfb, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(
            d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate)
        : "memory");
}

// 32 lanes x 16 consecutive columns of this warp's lane quarter, all set to v.
__device__ __forceinline__ void tmem_fill16(uint32_t taddr, uint32_t v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr), "r"(v) : "memory");
}
// 32 lanes x 16 consecutive fp32 columns of this warp's lane quarter.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
}
// 32 lanes x 32 consecutive columns of this warp's lane quarter, all set to v.
__device__ __forceinline__ void tmem_fill32(uint32_t taddr, uint32_t v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr), "r"(v) : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Every scale factor 1.0: the warp fills its lane quarter of the scale
// columns (and of the spare columns).
__device__ __forceinline__ void mxf4_unit_scales(uint32_t tmem, uint32_t quarter)
{
    const uint32_t lanes = (quarter * 32u) << 16;
    tmem_fill16(tmem + lanes + MX_SF_COL, 0x7F7F7F7Fu);
    tmem_fill16(tmem + lanes + MX_SPARE_COL, 0x7F7F7F7Fu);
    tmem_st_wait();
}

// Query stages shared by two reference tiles (kind::mxf4, a schedule
// choice: hd_mma_tuning::tiles_per_stage = 2).  Each stage holds one K-chunk
// of the query block (A) and the same K-chunk of two consecutive reference
// tiles (B0, B1); the MMA thread scores A x B0 into accumulator 0 and A x B1
// into accumulator 1, so every query byte staged serves 480 reference rows
// instead of 240: 28% fewer bytes cross from L2 to the SM and are written
// into shared memory per product.  The two accumulators then fill and drain
// together, so eight epilogue warps (four per accumulator) shorten the drain
// the tensor pipe waits for (four stages of 46 KB).  At 1M x 50k, D = 8192:
// 34.9 -> 34.2 ms; with 10k queries (40 query blocks) 12% slower, as the
// reference tiles' L2 hit rate falls: the autotuner decides.
#ifndef HD_MXF4_AP_STAGES
#define HD_MXF4_AP_STAGES 4
#endif

// Per-format shape of the pair kernel (AP: two reference tiles per query
// stage): reference rows per tile (the MMA's N), tiles per stage, stages,
// bytes of one stage, shared memory, epilogue warps and threads, and the
// tensor-memory column of each accumulator.
template <int FMT> __host__ __device__ constexpr uint32_t pair_tn() { return FMT == FMT_MXF4 ? (uint32_t)TN_MX : (uint32_t)TN; }
template <bool AP> __host__ __device__ constexpr uint32_t pair_nt() { return AP ? 2u : 1u; }
template <bool AP> __host__ __device__ constexpr uint32_t pair_stages()
{
    return AP ? (uint32_t)HD_MXF4_AP_STAGES : (uint32_t)STAGES2;
}
template <int FMT> __host__ __device__ constexpr uint32_t pair_b_bytes() { return (pair_tn<FMT>() / 2) * KB; }
template <int FMT, bool AP> __host__ __device__ constexpr uint32_t pair_stage_bytes()
{
    return A_BYTES + pair_nt<AP>() * pair_b_bytes<FMT>();
}
template <int FMT, bool AP> __host__ __device__ constexpr uint32_t pair_smem_bytes()
{
    return pair_stages<AP>() * pair_stage_bytes<FMT, AP>() + PAD2_BYTES + 1024 + 256;
}
template <bool AP> __host__ __device__ constexpr uint32_t pair_epi_warps() { return AP ? 8u : (uint32_t)EPI2_WARPS; }
template <bool AP> __host__ __device__ constexpr uint32_t pair_threads() { return 64u + 32u * pair_epi_warps<AP>(); }
template <int FMT> __device__ __forceinline__ uint32_t pair_acc_col(uint32_t buf)
{
    return FMT == FMT_MXF4 ? (buf ? MX_BUF1_COL : 0u) : buf * TN;
}
static_assert(pair_smem_bytes<FMT_MXF4, false>() <= 232448 && pair_smem_bytes<FMT_MXF4, true>() <= 232448 &&
                  (EPI2_SPLIT == 1 || TN_MX % (32 * EPI2_SPLIT) == 0),
              "mxf4 pair shape");
static_assert(pair_b_bytes<FMT_MXF4>() % 1024 == 0 && pair_stage_bytes<FMT_MXF4, true>() % 1024 == 0,
              "128B-swizzled operands start on 1024-byte boundaries");
static_assert(2 * pair_stages<true>() + 5 <= 32 && 2 * pair_stages<false>() + 5 <= 32,
              "barriers fit in their 256 bytes");

// A cluster of two CTAs on an SM pair (cluster ranks 0 and 1; rank 0 issues
// the pair's MMAs).  Each CTA holds its own block of 128 queries (A) and its
// half of the pair's reference tile (B; of two tiles when a query stage serves
// two); all loads complete on rank 0's stage barrier.
template <int K, int FMT, bool AP>
__global__ void __launch_bounds__(pair_threads<AP>(), 1)
k_search_mma2(const __grid_constant__ CUtensorMap qmap, const __grid_constant__ CUtensorMap lmap, mma_args a)
{
    static_assert(!AP || FMT == FMT_MXF4, "two tiles per query stage: kind::mxf4 only");
    constexpr uint32_t CS = 2;
    constexpr uint32_t NT = pair_nt<AP>();                  // reference tiles per query stage
    constexpr uint32_t NST = pair_stages<AP>();
    constexpr uint32_t TNF = pair_tn<FMT>();                // reference rows per tile
    constexpr uint32_t BHF = pair_b_bytes<FMT>();           // this CTA's half of one tile, one K-chunk
    constexpr uint32_t STAGE2F = pair_stage_bytes<FMT, AP>();   // A block slice + this CTA's half of NT tiles
    constexpr uint32_t EPT = 32u * pair_epi_warps<AP>();    // epilogue threads per CTA
    // the epilogue warps form SPLITF groups of four (one warp per lane quarter):
    // with shared query stages group g drains accumulator g, otherwise group g
    // scores columns [g, g + 1) * TNF / SPLITF of the accumulator of the tile
    constexpr uint32_t SPLITF = AP ? 2u : (uint32_t)EPI2_SPLIT;
    constexpr uint32_t EPI2_COLS_F = AP ? TNF : TNF / SPLITF;   // accumulator columns per epilogue warp
    // arrivals that free one accumulator: its epilogue threads in both CTAs
    constexpr uint32_t ACC_RELEASE = 2u * (AP ? EPT / 2u : EPT);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + NST * STAGE2F + PAD2_BYTES);
    uint64_t *empty = full + NST;
    uint64_t *acc_full = empty + NST;
    uint64_t *acc_empty = acc_full + 2;
    uint64_t *drain = acc_empty + 2;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort, s_lock_ok;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t crank = cluster_rank();   // 0: issues the pair's MMAs
    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < NST; ++i) {
            mbar_init(&full[i], 1);    // rank 0's producer arms it for both CTAs' bytes
            mbar_init(&empty[i], 1);   // one commit arrive (sent to both CTAs) per use
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], ACC_RELEASE);
        }
        mbar_init(drain, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc2(&s_tmem, TMEM2_COLS);
        tmem_relinquish2();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    volatile int *abort_flag = &s_abort;
    auto give_up = [&]() {
        *abort_flag = 1;
        hd_flag(a.status, HD_DEV_TIMEOUT);
    };
    // both CTAs must hold the same tensor-memory columns; otherwise do nothing
    if (threadIdx.x == 0 && ld_cluster_u32(cluster_addr(&s_tmem, crank ^ 1u)) != tmem) {
        *abort_flag = 1;
        hd_flag(a.status, HD_DEV_TMEM);
    }
    if (FMT == FMT_MXF4) {   // unit scale factors in both CTAs before the first MMA
        if (warp >= 2 && warp < 6) mxf4_unit_scales(tmem, (uint32_t)warp & 3u);
        tc_fence_before();
        __syncthreads();
        cluster_sync();
        tc_fence_after();
    }
    __syncthreads();
    const uint32_t cid = blockIdx.x / CS, ncl = gridDim.x / CS;
    const uint32_t total = a.pair_start[a.n_pairs];
    const uint32_t nchunks = a.row_bytes / KB;

    if (warp == 0) {
        // ------------------------------------------------------- producers
        if (lane == 0) {
            const uint32_t full0 = cluster_addr(&full[0], 0);   // rank 0's stage barriers
            const uint64_t pol_a = l2_policy(HD_MMA2_HINT_A), pol_b = l2_policy(HD_MMA2_HINT_B);
            uint32_t it = 0;
            for (uint32_t item = cid; item < total && !*abort_flag; item += ncl) {
                uint32_t b, t0, t1;
                item_range(a, item, b, t0, t1);
                const int32_t ya = (int32_t)((b * CS + crank) * TM);
                for (uint32_t t = t0; t < t1 && !*abort_flag; t += NT) {
                    const uint32_t nt = min(NT, t1 - t);   // tiles this stage run carries
                    for (uint32_t c = 0; c < nchunks; ++c, ++it) {
                        const uint32_t s = it % NST, ph = (it / NST) & 1u;
                        if (!mbar_wait(&empty[s], ph ^ 1u, a.wait_ns)) { give_up(); break; }
                        if (crank == 0) mbar_expect_tx(&full[s], tx_bytes(FMT, 2 * (A_BYTES + nt * BHF)));
                        if (a.stall && it == 0) continue;   // nothing ever completes this stage
                        uint8_t *sa = smem + s * STAGE2F, *sb = sa + A_BYTES;
                        const uint32_t bar = full0 + s * 8u;
                        const int32_t x = (int32_t)(c * KB);
                        if (HD_MMA2_HINT_A) tma_load_2d_pair_hint(sa, &qmap, x, ya, bar, pol_a);
                        else tma_load_2d_pair(sa, &qmap, x, ya, bar);
                        for (uint32_t u = 0; u < nt; ++u) {
                            const int32_t rb = (int32_t)((t + u) * TNF + crank * (TNF / 2));
                            if (HD_MMA2_HINT_B) tma_load_2d_pair_hint(sb + u * BHF, &lmap, x, rb, bar, pol_b);
                            else tma_load_2d_pair(sb + u * BHF, &lmap, x, rb, bar);
                        }
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (crank == 0) {
            // ------------------------------------------- MMA issuer (rank 0)
            if (lane == 0) {
                constexpr uint32_t idesc = FMT == FMT_MXF4 ? instr_desc_mxf4() : instr_desc2<FMT>();
                uint32_t it = 0, acc_it = 0;
                for (uint32_t item = cid; item < total && !*abort_flag; item += ncl) {
                    uint32_t b, t0, t1;
                    item_range(a, item, b, t0, t1);
                    for (uint32_t t = t0; t < t1 && !*abort_flag; t += NT, ++acc_it) {
                        const uint32_t nt = min(NT, t1 - t);
                        // one tile per stage: the tiles alternate between the two
                        // accumulators; two tiles per stage: both are in use, once
                        // per stage run
                        const uint32_t buf = (!AP && BUFS2 == 2) ? (acc_it & 1u) : 0u;
                        const uint32_t aph = ((!AP && BUFS2 == 2) ? (acc_it >> 1) : acc_it) & 1u;
                        if (!mbar_wait(&acc_empty[buf], aph ^ 1u, a.wait_ns)) { give_up(); break; }
                        if (AP && !mbar_wait(&acc_empty[1], aph ^ 1u, a.wait_ns)) { give_up(); break; }
                        tc_fence_after();
                        const uint32_t d_tmem = tmem + pair_acc_col<FMT>(buf);
                        bool ok = true;
                        for (uint32_t c = 0; c < nchunks; ++c, ++it) {
                            const uint32_t s = it % NST, ph = (it / NST) & 1u;
                            if (!mbar_wait(&full[s], ph, a.wait_ns)) { give_up(); ok = false; break; }
                            tc_fence_after();
                            const uint32_t sa = smem_addr(smem + s * STAGE2F), sb = sa + A_BYTES;
                            const uint64_t da = sw128_desc(sa), db = sw128_desc(sb);
#pragma unroll
                            for (uint32_t j = 0; j < KB / 32; ++j) {   // 32 bytes of K per instruction
                                if (FMT == FMT_MXF4)
                                    mma_issue2_mxf4(d_tmem, da + 2 * j, db + 2 * j, idesc, tmem + MX_SF_COL,
                                                    tmem + MX_SF_COL, (c | j) != 0);
                                else
                                    mma_issue2<FMT>(d_tmem, da + 2 * j, db + 2 * j, idesc, (c | j) != 0);
                            }
                            if (AP && nt > 1) {   // the second tile of the stage into accumulator 1
                                const uint64_t db1 = sw128_desc(sb + BHF);
#pragma unroll
                                for (uint32_t j = 0; j < KB / 32; ++j)
                                    mma_issue2_mxf4(tmem + pair_acc_col<FMT>(1), da + 2 * j, db1 + 2 * j, idesc,
                                                    tmem + MX_SF_COL, tmem + MX_SF_COL, (c | j) != 0);
                            }
                            mma_commit2_mc(&empty[s], 0x3);
                        }
                        if (!ok) break;
                        mma_commit2_mc(&acc_full[buf], 0x3);
                        if (AP) mma_commit2_mc(&acc_full[1], 0x3);
                    }
                }
                // every issued MMA has finished before either CTA releases its memory
                mma_commit2(drain);
                mbar_wait(drain, 0, a.wait_ns);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------- epilogue
        const uint32_t quarter = warp & 3;              // TMEM lanes this warp may read
        const uint32_t slice = (uint32_t)(warp - 2) >> 2;  // its group of four warps
        const uint32_t row = quarter * 32 + lane;       // query row within the block
        const uint32_t lane_addr = (quarter * 32) << 16;
        const bool leader = threadIdx.x == 64;
        const uint32_t acc_empty0 = cluster_addr(&acc_empty[0], 0);
        uint32_t acc_it = 0;
        for (uint32_t item = cid; item < total && !*abort_flag; item += ncl) {
            uint32_t b, t0, t1;
            item_range(a, item, b, t0, t1);
            const uint32_t sb_ = b * CS + crank;     // this CTA's query block
            const uint32_t sq = sb_ * TM + row;
            const uint32_t lo = sq < a.n_q ? a.lo[sq] : 0u, hi = sq < a.n_q ? a.hi[sq] : 0u;
            // last key of the query's running top-k (merged from its finished items)
            const uint64_t seed = sq < a.n_q ? (uint64_t)__ldcg(reinterpret_cast<const unsigned long long *>(
                                                   a.top + (size_t)sq * K + (K - 1)))
                                             : KEY_NONE;
            const uint32_t span = hi > lo ? hi - lo : 0u;
            uint64_t best[K];
#pragma unroll
            for (int i = 0; i < K; ++i) best[i] = KEY_NONE;
            bool ok = true;
            for (uint32_t t = t0; t < t1; t += NT, ++acc_it) {
                // this warp's accumulator and its tile
                const uint32_t buf = AP ? slice : ((BUFS2 == 2) ? (acc_it & 1u) : 0u);
                const uint32_t aph = ((!AP && BUFS2 == 2) ? (acc_it >> 1) : acc_it) & 1u;
                const uint32_t tt = AP ? t + slice : t;
                const uint32_t r0 = tt * TNF;
                if (!mbar_wait(&acc_full[buf], aph, a.wait_ns)) { give_up(); ok = false; break; }
                tc_fence_after();
                if (tt < t1) {
                    const uint32_t cg0 = AP ? 0u : slice * (EPI2_COLS_F / 32);
#pragma unroll 1
                    for (uint32_t cg = cg0; cg < cg0 + EPI2_COLS_F / 32; ++cg) {
                        uint32_t v[32];
                        tmem_ld32(tmem + lane_addr + pair_acc_col<FMT>(buf) + cg * 32, v);
                        tmem_ld_wait();
                        score_group<K>(v, r0 + cg * 32, lo, span, a.bias, a.shift, a.lib_orig, seed, best);
                    }
                    if (TNF % 32 != 0) {   // the last 16 columns of a 240-column tile
                        constexpr uint32_t c16 = TNF / 32 * 32;
                        uint32_t v[16];
                        tmem_ld16(tmem + lane_addr + pair_acc_col<FMT>(buf) + c16, v);
                        tmem_ld_wait();
                        score_group<K, 16>(v, r0 + c16, lo, span, a.bias, a.shift, a.lib_orig, seed, best);
                    }
                }
                tc_fence_before();
                mbar_arrive_remote(acc_empty0 + buf * 8u);
            }
            // merge into the block's running top-k under its lock (bounded spin),
            // the SPLITF partial lists of each row one after the other
            epi_bar_n(EPT);
            if (leader) {
                int got = 0;
                if (ok && !*abort_flag) {
                    const uint64_t w0 = hd_globaltimer_ns();
                    for (uint32_t i = 0;; ++i) {
                        if (atomicCAS(&a.locks[sb_], 0u, 1u) == 0u) { got = 1; break; }
                        if ((i & 63u) == 0 && hd_globaltimer_ns() - w0 > a.wait_ns) { give_up(); break; }
                    }
                    __threadfence();
                }
                s_lock_ok = got;
            }
            epi_bar_n(EPT);
            const bool locked = s_lock_ok != 0;
            for (uint32_t ph = 0; ph < SPLITF; ++ph) {
                if (locked && slice == ph) {
                    if (sq < a.n_q) {
                        unsigned long long *g = reinterpret_cast<unsigned long long *>(a.top + (size_t)sq * K);
                        uint64_t cur[K];
#pragma unroll
                        for (int i = 0; i < K; ++i) cur[i] = __ldcg(g + i);
                        topk_merge<K>(cur, best);
#pragma unroll
                        for (int i = 0; i < K; ++i) __stcg(g + i, (unsigned long long)cur[i]);
                    }
                    __threadfence();
                }
                epi_bar_n(EPT);
            }
            if (leader && locked) atomicExch(&a.locks[sb_], 0u);
            if (!locked) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();   // rank 0's MMAs have drained; neither CTA issues loads any more
    // after a give-up anywhere, loads issued before the barrier may still be
    // landing in this CTA's shared memory: a bounded pause lets them complete
    if (threadIdx.x == 0 && (*abort_flag || (a.status && (atomicOr_system(a.status, 0u) & HD_DEV_TIMEOUT) != 0u))) {
        const uint64_t w0 = hd_globaltimer_ns();
        while (hd_globaltimer_ns() - w0 < 200000ull) __nanosleep(1000);
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc2(tmem, TMEM2_COLS);
}

// ------------------------------------------------- tensor-pipe microbenchmark
// The pair form's tensor-core instruction alone, as the roofline of the
// search: tcgen05.mma.cta_group::2 with M = 256, N = 256 and 32 bytes of K per
// instruction (the search's shape, descriptors and instruction descriptor),
// on +-1 operands already resident in shared memory (no global traffic),
// issued back to back by rank 0 of every SM pair.  As in the search at
// D = 8192, 256 instructions accumulate into one of two 256-column
// accumulators before the other one is used.  160 KB of dynamic shared memory
// keep one CTA per SM.
constexpr uint32_t PEAK_SMEM_BYTES = 160u * 1024u;
constexpr int PEAK_THREADS = 128;
template <int FMT>
__global__ void __launch_bounds__(PEAK_THREADS, 1) k_peak_mma2(uint32_t iters, uint64_t wait_ns, uint32_t *status)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *done = reinterpret_cast<uint64_t *>(smem + A_BYTES + B2_BYTES);
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t crank = cluster_rank();
    // +-1 in the operand format: e4m3 0x38 / 0xB8, e2m1 codes 0x2 / 0xA, bf16 0x3F80 / 0xBF80
    uint32_t *w = reinterpret_cast<uint32_t *>(smem);
    for (uint32_t i = threadIdx.x; i < (A_BYTES + B2_BYTES) / 4; i += blockDim.x) {
        const bool neg = ((i * 2654435761u) >> 31) != 0u;
        w[i] = FMT == FMT_BF16 ? (neg ? 0xBF80BF80u : 0x3F803F80u)
             : FMT == FMT_E4M3 ? (neg ? 0xB8B8B8B8u : 0x38383838u)
                               : (neg ? 0x0A0A0A0Au : 0x02020202u);
    }
    if (threadIdx.x == 0) {
        mbar_init(done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc2(&s_tmem, TMEM2_COLS);
        tmem_relinquish2();
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // operands visible to the tensor core
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (threadIdx.x == 0 && ld_cluster_u32(cluster_addr(&s_tmem, crank ^ 1u)) != tmem) {
        s_abort = 1;
        hd_flag(status, HD_DEV_TMEM);
    }
    __syncthreads();
    const bool run = s_abort == 0;
    if (warp == 1 && lane == 0 && run) {
        if (crank == 0) {
            constexpr uint32_t idesc = instr_desc2<FMT>();
            const uint32_t sa = smem_addr(smem), sb = sa + A_BYTES;
            const uint64_t da = sw128_desc(sa), db = sw128_desc(sb);
            for (uint32_t it = 0; it < iters; ++it) {
                const uint32_t d_tmem = tmem + ((it >> 6) & 1u) * TN;
#pragma unroll
                for (uint32_t j = 0; j < KB / 32; ++j)
                    mma_issue2<FMT>(d_tmem, da + 2 * j, db + 2 * j, idesc, ((it & 63u) | j) != 0);
            }
            mma_commit2_mc(done, 0x3);
        }
        // every MMA of the pair has finished before either CTA frees its tensor memory
        if (!mbar_wait(done, 0, wait_ns)) hd_flag(status, HD_DEV_TIMEOUT);
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    if (warp == 1) tmem_dealloc2(tmem, TMEM2_COLS);
}

// The kind::mxf4 instruction alone (the mxf4 search's roofline), as
// k_peak_mma2 for the other kinds.  With `check`, every operand is +1 and
// the accumulators start cleared: the last accumulator then holds 64
// instructions-groups x 4 x 64 products = 16384 in every element, which the
// kernel verifies (HD_DEV_BAD_INPUT in the status word otherwise).
__global__ void __launch_bounds__(PEAK_THREADS, 1)
k_peak_mxf4(uint32_t iters, uint32_t check, uint64_t wait_ns, uint32_t *status)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *done = reinterpret_cast<uint64_t *>(smem + A_BYTES + B2MX_BYTES);
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t crank = cluster_rank();
    uint32_t *w = reinterpret_cast<uint32_t *>(smem);
    for (uint32_t i = threadIdx.x; i < (A_BYTES + B2MX_BYTES) / 4; i += blockDim.x) {
        const bool neg = !check && ((i * 2654435761u) >> 31) != 0u;
        w[i] = neg ? 0xAAAAAAAAu : 0x22222222u;   // e2m1 -1 / +1 in both nibbles
    }
    if (threadIdx.x == 0) {
        mbar_init(done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc2(&s_tmem, TMEM2_COLS);
        tmem_relinquish2();
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (threadIdx.x == 0 && ld_cluster_u32(cluster_addr(&s_tmem, crank ^ 1u)) != tmem) {
        s_abort = 1;
        hd_flag(status, HD_DEV_TMEM);
    }
    const uint32_t quarter = (uint32_t)warp & 3u, lanes = (quarter * 32u) << 16;
    mxf4_unit_scales(tmem, quarter);
    if (check) {
        for (uint32_t c = 0; c + 32 <= (uint32_t)TN_MX; c += 32) {
            tmem_fill32(tmem + lanes + c, 0u);
            tmem_fill32(tmem + lanes + MX_BUF1_COL + c, 0u);
        }
        if (TN_MX % 32) {
            tmem_fill16(tmem + lanes + TN_MX / 32 * 32, 0u);
            tmem_fill16(tmem + lanes + MX_BUF1_COL + TN_MX / 32 * 32, 0u);
        }
        tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    const bool run = s_abort == 0;
    if (warp == 1 && lane == 0 && run) {
        if (crank == 0) {
            constexpr uint32_t idesc = instr_desc_mxf4();
            const uint32_t sa = smem_addr(smem), sb = sa + A_BYTES;
            const uint64_t da = sw128_desc(sa), db = sw128_desc(sb);
            for (uint32_t it = 0; it < iters; ++it) {
                const uint32_t d_tmem = tmem + (((it >> 6) & 1u) ? MX_BUF1_COL : 0u);
#pragma unroll
                for (uint32_t j = 0; j < KB / 32; ++j)   // 32 bytes = 64 components of K per instruction
                    mma_issue2_mxf4(d_tmem, da + 2 * j, db + 2 * j, idesc, tmem + MX_SF_COL, tmem + MX_SF_COL,
                                    ((it & 63u) | j) != 0);
            }
            mma_commit2_mc(done, 0x3);
        }
        if (!mbar_wait(done, 0, wait_ns)) hd_flag(status, HD_DEV_TIMEOUT);
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    if (check && run && iters >= 64) {
        const uint32_t col0 = ((iters - 1) >> 6) & 1u ? MX_BUF1_COL : 0u;
        bool bad = false;
#pragma unroll 1
        for (uint32_t cg = 0; cg < (uint32_t)TN_MX / 32; ++cg) {
            uint32_t v[32];
            tmem_ld32(tmem + lanes + col0 + cg * 32, v);
            tmem_ld_wait();
#pragma unroll
            for (int e = 0; e < 32; ++e) bad |= __uint_as_float(v[e]) != 16384.0f;
        }
        if (TN_MX % 32) {
            uint32_t v[16];
            tmem_ld16(tmem + lanes + col0 + TN_MX / 32 * 32, v);
            tmem_ld_wait();
#pragma unroll
            for (int e = 0; e < 16; ++e) bad |= __uint_as_float(v[e]) != 16384.0f;
        }
        if (bad) hd_flag(status, HD_DEV_BAD_INPUT);
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    if (warp == 1) tmem_dealloc2(tmem, TMEM2_COLS);
}

// Work list of the L2-blocked schedule (one CTA of 1024 threads): per query
// block the absolute tile range covering the union of its windows, then the
// item count of every (super-group, block) pair and its exclusive scan.
__global__ void __launch_bounds__(1024)
k_worklist_l2(const uint32_t *__restrict__ lo, const uint32_t *__restrict__ hi, uint32_t n_q, uint32_t bq,
              uint32_t tn, uint32_t n_blocks, uint32_t tg, uint32_t sg, uint32_t n_super,
              uint32_t *__restrict__ blk_t0, uint32_t *__restrict__ blk_t1, uint32_t *__restrict__ pair_start)
{
    __shared__ uint32_t sh[33];
    for (uint32_t b = threadIdx.x; b < n_blocks; b += blockDim.x) {
        uint32_t l = 0xFFFFFFFFu, h = 0;
        const uint32_t e = min(n_q, (b + 1) * bq);
        for (uint32_t s = b * bq; s < e; ++s)
            if (hi[s] > lo[s]) {
                l = min(l, lo[s]);
                h = max(h, hi[s]);
            }
        blk_t0[b] = h > l ? l / tn : 0u;
        blk_t1[b] = h > l ? (h + tn - 1) / tn : 0u;
    }
    __syncthreads();
    const uint32_t n_pairs = n_super * n_blocks;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < n_pairs; base += blockDim.x) {
        const uint32_t p = base + threadIdx.x;
        uint32_t v = 0;
        if (p < n_pairs) {
            const uint32_t G = p / n_blocks, b = p % n_blocks;
            const uint32_t t0 = blk_t0[b], t1 = blk_t1[b];
            if (t1 > t0) {
                const uint32_t g0 = max(t0 / tg, G * sg), g1 = min((t1 - 1) / tg, G * sg + sg - 1);
                v = g1 >= g0 ? g1 - g0 + 1 : 0u;
            }
        }
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, &tot, sh);
        if (p < n_pairs) pair_start[p] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) pair_start[n_pairs] = carry;
}

// Running top-k (sorted query order) -> the caller's order.
template <int K>
__global__ void k_emit(const uint64_t *__restrict__ top, const uint32_t *__restrict__ perm, uint32_t n_q,
                       uint32_t k, uint32_t *__restrict__ out_idx, uint16_t *__restrict__ out_dist)
{
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_q) return;
    const uint32_t q = perm[s];
    for (uint32_t t = 0; t < k; ++t) {
        const uint64_t key = top[(size_t)s * K + t];
        const bool none = key == KEY_NONE;
        out_idx[(size_t)q * k + t] = none ? 0xFFFFFFFFu : (uint32_t)key;
        out_dist[(size_t)q * k + t] = none ? (uint16_t)0xFFFF : (uint16_t)(key >> 32);
    }
}

// Multi-bit form: scores S = bias - key distance, in the caller's order.
template <int K>
__global__ void k_emit_score(const uint64_t *__restrict__ top, const uint32_t *__restrict__ perm, uint32_t n_q,
                             uint32_t k, uint32_t bias, uint32_t *__restrict__ out_idx,
                             int32_t *__restrict__ out_score)
{
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_q) return;
    const uint32_t q = perm[s];
    for (uint32_t t = 0; t < k; ++t) {
        const uint64_t key = top[(size_t)s * K + t];
        const bool none = key == KEY_NONE;
        out_idx[(size_t)q * k + t] = none ? 0xFFFFFFFFu : (uint32_t)key;
        out_score[(size_t)q * k + t] = none ? INT32_MIN : (int32_t)((int64_t)bias - (int64_t)(key >> 32));
    }
}

__global__ void k_fill_none(uint32_t *__restrict__ out_idx, int32_t *__restrict__ out_score, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        out_idx[i] = 0xFFFFFFFFu;
        out_score[i] = INT32_MIN;
    }
}

// Operand codes of small integers, from the IEEE single bits of the value:
// an integer of at most four significant bits (|v| <= 15) is exact in e4m3
// (sign, 4-bit exponent of bias 7, top 3 mantissa bits), |v| <= 3 in e2m1
// (sign, 2-bit exponent of bias 1, top mantissa bit), and bf16 is the
// single's upper half.
__device__ __forceinline__ uint32_t int_to_e4m3(int v)
{
    if (v == 0) return 0u;
    const uint32_t f = __float_as_uint((float)v);
    return ((f >> 31) << 7) | ((((f >> 23) & 0xFFu) - 120u) << 3) | ((f >> 20) & 7u);
}
__device__ __forceinline__ uint32_t int_to_e2m1(int v)
{
    if (v == 0) return 0u;
    const uint32_t f = __float_as_uint((float)v);
    return ((f >> 31) << 3) | ((((f >> 23) & 0xFFu) - 126u) << 1) | ((f >> 22) & 1u);
}
__device__ __forceinline__ uint32_t int_to_bf16(int v) { return __float_as_uint((float)v) >> 16; }

// One row of int8 components in [-m, m] per warp -> the operand format (e4m3
// bytes, bf16 halves, or e2m1 nibbles with element 2i in the low nibble of
// byte i).  A component outside [-m, m] is written as 0 and flags the
// status word.  `perm` (optional) picks the source row of output row r.
template <int FMT>
__global__ void k_expand_comp(const int8_t *__restrict__ comp, const uint32_t *__restrict__ perm, uint32_t n,
                              uint32_t D, int m, uint8_t *__restrict__ out, uint32_t *status)
{
    const uint32_t r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const uint32_t lane = threadIdx.x & 31;
    if (r >= n) return;
    const int8_t *src = comp + (size_t)(perm ? perm[r] : r) * D;
    bool bad = false;
    for (uint32_t c = lane; c < D / 16; c += 32) {
        const uint4 in = *reinterpret_cast<const uint4 *>(src + (size_t)c * 16);
        const uint32_t wv[4] = {in.x, in.y, in.z, in.w};
        int v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            v[i] = (int)(int8_t)(uint8_t)(wv[i >> 2] >> (8 * (i & 3)));
            if (v[i] < -m || v[i] > m) {
                bad = true;
                v[i] = 0;
            }
        }
        if (FMT == FMT_E4M3) {
            uint32_t p[4] = {0, 0, 0, 0};
#pragma unroll
            for (int i = 0; i < 16; ++i) p[i >> 2] |= int_to_e4m3(v[i]) << (8 * (i & 3));
            *reinterpret_cast<uint4 *>(out + (size_t)r * D + (size_t)c * 16) = make_uint4(p[0], p[1], p[2], p[3]);
        } else if (FMT == FMT_BF16) {
            uint32_t p[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) p[i] = int_to_bf16(v[2 * i]) | (int_to_bf16(v[2 * i + 1]) << 16);
            uint4 *o = reinterpret_cast<uint4 *>(out + (size_t)r * 2 * D + (size_t)c * 32);
            o[0] = make_uint4(p[0], p[1], p[2], p[3]);
            o[1] = make_uint4(p[4], p[5], p[6], p[7]);
        } else {
            uint32_t p[2] = {0, 0};
#pragma unroll
            for (int i = 0; i < 16; ++i) p[i >> 3] |= int_to_e2m1(v[i]) << (4 * (i & 7));
            *reinterpret_cast<uint2 *>(out + (size_t)r * (D / 2) + (size_t)c * 8) = make_uint2(p[0], p[1]);
        }
    }
    if (bad) hd_flag(status, HD_DEV_BAD_INPUT);
}

// One row of packed bits per warp -> +-1 in the operand format: bytes (e4m3:
// 0x38 / 0xB8), halves (bf16: 0x3F80 / 0xBF80) or nibbles (e2m1: 0x2 / 0xA,
// element 2i in the low nibble of byte i).
template <int FMT>
__global__ void k_expand(const uint64_t *__restrict__ hv, const uint32_t *__restrict__ perm, uint32_t n,
                         uint32_t W, uint8_t *__restrict__ out)
{
    const uint32_t r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const uint32_t lane = threadIdx.x & 31;
    if (r >= n) return;
    const uint64_t *src = hv + (size_t)(perm ? perm[r] : r) * W;
    constexpr uint32_t WB = FMT == FMT_BF16 ? 128 : (FMT == FMT_E4M3 ? 64 : 32);   // bytes per 64 bits
    uint8_t *dst = out + (size_t)r * W * WB;
    for (uint32_t w = lane; w < W; w += 32) {
        const uint64_t x = src[w];
        uint4 *o = reinterpret_cast<uint4 *>(dst + (size_t)w * WB);
#pragma unroll
        for (int q = 0; q < (int)(WB / 16); ++q) {
            uint32_t p[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                uint32_t word = 0;
                if (FMT == FMT_E4M3) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint32_t bit = (uint32_t)(x >> (q * 16 + h * 4 + j)) & 1u;
                        word |= (0x38u | (bit << 7)) << (8 * j);
                    }
                } else if (FMT == FMT_BF16) {
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const uint32_t bit = (uint32_t)(x >> (q * 8 + h * 2 + j)) & 1u;
                        word |= (0x3F80u | (bit << 15)) << (16 * j);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const uint32_t bit = (uint32_t)(x >> (q * 32 + h * 8 + j)) & 1u;
                        word |= (0x2u | (bit << 3)) << (4 * j);
                    }
                }
                p[h] = word;
            }
            o[q] = make_uint4(p[0], p[1], p[2], p[3]);
        }
    }
}

// ------------------------------------------------------------- host side
using encode_fn = PFN_cuTensorMapEncodeTiled_v12000;

encode_fn tensor_map_encoder()
{
    static std::once_flag once;
    static encode_fn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<encode_fn>(p);
    });
    return fn;
}

// Rows of `row_bytes` bytes; boxes of 128 bytes x box_rows rows, 128B swizzle,
// rows past `rows` read as zero.
hd_status make_map(CUtensorMap *m, const void *base, uint64_t rows, uint32_t row_bytes, uint32_t box_rows)
{
    encode_fn enc = tensor_map_encoder();
    if (!enc) return hd_fail(HD_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
    const cuuint64_t dims[2] = {row_bytes, rows};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)KB, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return hd_fail(HD_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return HD_OK;
}

// Rows of `dim` e2m1 values packed two per byte (dim / 2 bytes); boxes of 128
// values x box_rows rows, unpacked into 16-byte containers of 16 values (128
// bytes of shared memory per row), 128B swizzle, rows past `rows` read as 0.
hd_status make_map_e2m1(CUtensorMap *m, const void *base, uint64_t rows, uint32_t dim, uint32_t box_rows)
{
    encode_fn enc = tensor_map_encoder();
    if (!enc) return hd_fail(HD_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
    const cuuint64_t dims[2] = {dim, rows};
    const cuuint64_t strides[1] = {dim / 2};
    const cuuint32_t box[2] = {128u, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_16U4_ALIGN16B, 2, const_cast<void *>(base), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return hd_fail(HD_ERR_CUDA, "cuTensorMapEncodeTiled (e2m1) failed");
    return HD_OK;
}

// Multi-bit search I/O: int8 query components in, scores out.
struct dot_io {
    const int8_t *q_comp;
    int32_t *out_score;
};

template <int FMT>
constexpr uint32_t global_row_bytes(uint32_t dim) { return FMT == FMT_BF16 ? 2 * dim : (FMT == FMT_E4M3 ? dim : dim / 2); }

template <int K, int FMT>
hd_status run_mma(const hd_library *lib, const uint64_t *q_hv, const double *q_mz, const uint8_t *q_z,
                  uint32_t n_q, const hd_qwin &win, uint32_t k, uint32_t *out_idx, uint16_t *out_dist,
                  cudaStream_t s, const hd_mma_tuning &tune, const dot_io *dot = nullptr)
{
    constexpr int XF = FMT == FMT_MXF4 ? FMT_E2M1 : FMT;   // format of the rows in HBM
    const bool pair = FMT == FMT_MXF4 || tune.cta_group == 2;   // SM pairs, M = 256 (cluster of 2)
    const uint32_t cs = pair ? 2u : 1u;      // CTAs per cluster
    const uint32_t n_blocks = (n_q + TM * cs - 1) / (TM * cs);
    // shared-memory bytes of one operand row (the K extent the kernel walks) and HBM bytes
    const uint32_t row_bytes = FMT == FMT_MXF4 ? lib->dim / 2 : lib->dim * (FMT == FMT_BF16 ? 2u : 1u);
    const uint32_t g_row_bytes = global_row_bytes<XF>(lib->dim);
    if (FMT == FMT_MXF4 && lib->dim % 256 != 0)
        return hd_fail(HD_ERR_UNSUPPORTED, "kind::mxf4 form needs D to be a multiple of 256");
    const uint8_t *lib_x = XF == FMT_BF16 ? lib->x_bf16 : (XF == FMT_E4M3 ? lib->x_fp8 : lib->x_fp4);
    if (!lib_x) return hd_fail(HD_ERR_INVALID_ARG, "library not prepared for this tensor-core form");
    // kind::mxf4 on SM pairs may share each query stage between two reference tiles
    const bool ap = FMT == FMT_MXF4 && tune.tiles_per_stage == 2;
    auto kern = [&]() {
        if constexpr (FMT == FMT_MXF4) return ap ? k_search_mma2<K, FMT, true> : k_search_mma2<K, FMT, false>;
        else return pair ? k_search_mma2<K, FMT, false> : k_search_mma<K, FMT>;
    }();
    const uint32_t tn = pair ? pair_tn<FMT>() : (uint32_t)TN;   // reference rows per tile
    const uint32_t smem_bytes = !pair ? SMEM_BYTES : (ap ? pair_smem_bytes<FMT, true>() : pair_smem_bytes<FMT, false>());
    const uint32_t threads = !pair ? (uint32_t)THREADS : (ap ? pair_threads<true>() : pair_threads<false>());
    HD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes));
    if (cs > 1) HD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    uint32_t grid = (uint32_t)lib->num_sms / cs * cs;
    if (cs > 1) {   // only co-resident clusters: a persistent grid must not wait for SMs
        cudaLaunchConfig_t qc = {};
        qc.gridDim = dim3(grid);
        qc.blockDim = dim3(threads);
        qc.dynamicSmemBytes = smem_bytes;
        cudaLaunchAttribute qa[1];
        qa[0].id = cudaLaunchAttributeClusterDimension;
        qa[0].val.clusterDim.x = cs;
        qa[0].val.clusterDim.y = 1;
        qa[0].val.clusterDim.z = 1;
        qc.attrs = qa;
        qc.numAttrs = 1;
        int n_cl = 0;
        HD_CUDA_TRY(cudaOccupancyMaxActiveClusters(&n_cl, kern, &qc));
        if (n_cl < 1) return hd_fail(HD_ERR_UNSUPPORTED, "cluster launch does not fit on this GPU");
        grid = std::min(grid, (uint32_t)n_cl * cs);
    }
    const uint32_t tg = tune.tile_group, sg = tune.super_group;
    const uint32_t n_tiles = (lib->n + tn - 1) / tn;
    const uint32_t n_super = (n_tiles + tg * sg - 1) / (tg * sg);
    const size_t n_pairs = (size_t)n_super * n_blocks;
    if (n_pairs >= 0xFFFFFFFFull) return hd_fail(HD_ERR_UNSUPPORTED, "work list too large");

    auto carve = [&](hd_arena &ar, uint32_t **perm, uint32_t **lo, uint32_t **hi, uint32_t **bt0,
                     uint32_t **bt1, uint32_t **pst, uint64_t **top, uint32_t **locks, uint8_t **qx) {
        *perm = ar.take<uint32_t>(n_q);
        *lo = ar.take<uint32_t>(n_q);
        *hi = ar.take<uint32_t>(n_q);
        *bt0 = ar.take<uint32_t>(n_blocks);
        *bt1 = ar.take<uint32_t>(n_blocks);
        *pst = ar.take<uint32_t>(n_pairs + 1);
        *top = ar.take<uint64_t>((size_t)n_q * K);
        *locks = ar.take<uint32_t>((size_t)n_blocks * cs);
        *qx = ar.take<uint8_t>((size_t)n_q * g_row_bytes);
    };
    uint32_t *perm, *lo, *hi, *bt0, *bt1, *pst, *locks;
    uint64_t *top;
    uint8_t *qx;
    hd_arena plan;
    carve(plan, &perm, &lo, &hi, &bt0, &bt1, &pst, &top, &locks, &qx);
    hd_sort_charge_mz(q_mz, q_z, win.cls, n_q, nullptr, plan, s);
    hd_arena ar;
    if (cudaMallocAsync((void **)&ar.base, plan.used, s) != cudaSuccess) {
        cudaGetLastError();
        return hd_fail(HD_ERR_OOM, "tensor-core search scratch allocation failed");
    }
    carve(ar, &perm, &lo, &hi, &bt0, &bt1, &pst, &top, &locks, &qx);
    CUtensorMap qmap, lmap;
    // e2m1 for kind::f8f6f4 is unpacked by the TMA; every other form copies its bytes as they are
    hd_status st = FMT == FMT_E2M1 ? make_map_e2m1(&qmap, qx, n_q, lib->dim, TM)
                                   : make_map(&qmap, qx, n_q, row_bytes, TM);
    if (st == HD_OK)
        st = FMT == FMT_E2M1 ? make_map_e2m1(&lmap, lib_x, lib->n, lib->dim, tn / cs)
                             : make_map(&lmap, lib_x, lib->n, row_bytes, tn / cs);
    if (st != HD_OK) {
        cudaFreeAsync(ar.base, s);
        return st;
    }
    HD_CUDA_TRY(cudaMemsetAsync(top, 0xFF, (size_t)n_q * K * sizeof(uint64_t), s));
    HD_CUDA_TRY(cudaMemsetAsync(locks, 0, (size_t)n_blocks * cs * sizeof(uint32_t), s));
    hd_sort_charge_mz(q_mz, q_z, win.cls, n_q, perm, ar, s);
    if (dot)
        hd_count_launches(1), k_expand_comp<XF><<<hd_ceil_div(n_q, 8), 256, 0, s>>>(
            dot->q_comp, perm, n_q, lib->dim, (int)hd_comp_max(lib->bits), qx, lib->status.dev);
    else
        hd_count_launches(1), k_expand<XF><<<hd_ceil_div(n_q, 8), 256, 0, s>>>(q_hv, perm, n_q, lib->W, qx);
    const uint32_t mq = hd_comp_max(lib->bits);
    const uint32_t bias = dot ? lib->dim * mq * mq : lib->dim, shift = dot ? 0u : 1u;
    hd_count_launches(1), k_windows<<<hd_ceil_div(n_q, 256), 256, 0, s>>>(lib->mz, lib->charge_start, q_mz, q_z,
                                                                          perm, n_q, win, lo, hi);
    hd_count_launches(1), k_worklist_l2<<<1, 1024, 0, s>>>(lo, hi, n_q, TM * cs, tn, n_blocks, tg, sg, n_super, bt0, bt1, pst);
    mma_args ma{lib->orig, lo, hi, bt0, bt1, pst, top, locks, lib->status.dev, n_q, n_blocks, (uint32_t)n_pairs,
                tg, sg, lib->dim, row_bytes, hd_wait_limit(lib), hd_take_injected_stall(lib) ? 1u : 0u,
                bias, shift};
    {
        hd_prof_scope timed(HD_KERNEL_SEARCH, s);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem_bytes;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        hd_count_launches(1);
        HD_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, qmap, lmap, ma));
    }
    if (dot)
        hd_count_launches(1), k_emit_score<K><<<hd_ceil_div(n_q, 128), 128, 0, s>>>(top, perm, n_q, k, bias, out_idx,
                                                                                 dot->out_score);
    else
        hd_count_launches(1), k_emit<K><<<hd_ceil_div(n_q, 128), 128, 0, s>>>(top, perm, n_q, k, out_idx, out_dist);
    HD_CUDA_TRY(cudaGetLastError());
    HD_CUDA_TRY(cudaFreeAsync(ar.base, s));
    return HD_OK;
}

template <int FMT>
hd_status run_fmt(const hd_library *lib, const uint64_t *q_hv, const double *q_mz, const uint8_t *q_z,
                  uint32_t n_q, const hd_qwin &win, uint32_t k, uint32_t *oi, uint16_t *od, cudaStream_t s,
                  const hd_mma_tuning &tu, const dot_io *dot = nullptr)
{
    if (k <= 1) return run_mma<1, FMT>(lib, q_hv, q_mz, q_z, n_q, win, k, oi, od, s, tu, dot);
    if (k <= 2) return run_mma<2, FMT>(lib, q_hv, q_mz, q_z, n_q, win, k, oi, od, s, tu, dot);
    if (k <= 4) return run_mma<4, FMT>(lib, q_hv, q_mz, q_z, n_q, win, k, oi, od, s, tu, dot);
    if (k <= 8) return run_mma<8, FMT>(lib, q_hv, q_mz, q_z, n_q, win, k, oi, od, s, tu, dot);
    return run_mma<16, FMT>(lib, q_hv, q_mz, q_z, n_q, win, k, oi, od, s, tu, dot);
}

}  // namespace

namespace {
// Operand format of a tensor-core form (kind::mxf4 keeps the e2m1 rows of HD_FORM_TC_FP4).
int form_fmt(hd_search_form form)
{
    return form == HD_FORM_TC_BF16 ? FMT_BF16 : (form == HD_FORM_TC_FP8 ? FMT_E4M3 : FMT_E2M1);
}
}  // namespace

hd_status hd_library_expand(hd_library *lib, hd_search_form form, cudaStream_t s)
{
    const int fmt = form_fmt(form);
    if (fmt == FMT_E2M1 && lib->bits > 3)
        return hd_fail(HD_ERR_UNSUPPORTED, "e2m1 holds components up to 3 only (bits <= 3)");
    uint8_t *&dst = fmt == FMT_BF16 ? lib->x_bf16 : (fmt == FMT_E4M3 ? lib->x_fp8 : lib->x_fp4);
    if (dst || lib->n == 0) return HD_OK;
    const size_t bytes = (size_t)lib->n * (fmt == FMT_BF16 ? global_row_bytes<FMT_BF16>(lib->dim)
                                           : fmt == FMT_E4M3 ? global_row_bytes<FMT_E4M3>(lib->dim)
                                                             : global_row_bytes<FMT_E2M1>(lib->dim));
    if (cudaMalloc(&dst, bytes) != cudaSuccess) {
        cudaGetLastError();
        dst = nullptr;
        return hd_fail(HD_ERR_OOM, "expanded library allocation failed");
    }
    const unsigned g = hd_ceil_div(lib->n, 8);
    if (lib->bits > 1) {   // multi-bit components; range violations flag the library's status
        const int m = (int)hd_comp_max(lib->bits);
        if (fmt == FMT_E4M3)
            hd_count_launches(1), k_expand_comp<FMT_E4M3><<<g, 256, 0, s>>>(lib->comp, nullptr, lib->n, lib->dim, m,
                                                                           dst, lib->status.dev);
        else if (fmt == FMT_BF16)
            hd_count_launches(1), k_expand_comp<FMT_BF16><<<g, 256, 0, s>>>(lib->comp, nullptr, lib->n, lib->dim, m,
                                                                           dst, lib->status.dev);
        else
            hd_count_launches(1), k_expand_comp<FMT_E2M1><<<g, 256, 0, s>>>(lib->comp, nullptr, lib->n, lib->dim, m,
                                                                           dst, lib->status.dev);
    } else if (fmt == FMT_E4M3)
        hd_count_launches(1), k_expand<FMT_E4M3><<<g, 256, 0, s>>>(lib->hv, nullptr, lib->n, lib->W, dst);
    else if (fmt == FMT_BF16)
        hd_count_launches(1), k_expand<FMT_BF16><<<g, 256, 0, s>>>(lib->hv, nullptr, lib->n, lib->W, dst);
    else
        hd_count_launches(1), k_expand<FMT_E2M1><<<g, 256, 0, s>>>(lib->hv, nullptr, lib->n, lib->W, dst);
    HD_CUDA_TRY(cudaGetLastError());
    return HD_OK;
}

hd_status hd_search_mma_run(const hd_library *lib, hd_search_form form, const uint64_t *q_hv, const double *q_mz,
                            const uint8_t *q_charge, uint32_t n_q, const hd_qwin &win, uint32_t k,
                            uint32_t *out_idx, uint16_t *out_dist, cudaStream_t s)
{
    if (lib->n == 0) return hd_search_popc_run(lib, q_hv, q_mz, q_charge, n_q, win, k, out_idx, out_dist, s);
    hd_mma_tuning tu = lib->mma_tuning;
    if (tu.tile_group == 0) tu.tile_group = 16;
    if (tu.super_group == 0) tu.super_group = 16;
    if (tu.cta_group != 1) tu.cta_group = 2;   // default: SM pairs
    tu.cluster = tu.cta_group;
    if (form == HD_FORM_TC_MXF4)
        return run_fmt<FMT_MXF4>(lib, q_hv, q_mz, q_charge, n_q, win, k, out_idx, out_dist, s, tu);
    const int fmt = form_fmt(form);
    if (fmt == FMT_E4M3) return run_fmt<FMT_E4M3>(lib, q_hv, q_mz, q_charge, n_q, win, k, out_idx, out_dist, s, tu);
    if (fmt == FMT_BF16) return run_fmt<FMT_BF16>(lib, q_hv, q_mz, q_charge, n_q, win, k, out_idx, out_dist, s, tu);
    return run_fmt<FMT_E2M1>(lib, q_hv, q_mz, q_charge, n_q, win, k, out_idx, out_dist, s, tu);
}

hd_status hd_search_mma_dot_run(const hd_library *lib, hd_search_form form, const int8_t *q_comp,
                                const double *q_mz, const uint8_t *q_charge, uint32_t n_q, const hd_qwin &win,
                                uint32_t k, uint32_t *out_idx, int32_t *out_score, cudaStream_t s)
{
    if (lib->n == 0) {   // no candidates anywhere
        hd_count_launches(1), k_fill_none<<<hd_ceil_div((size_t)n_q * k, 256), 256, 0, s>>>(out_idx, out_score,
                                                                                          (size_t)n_q * k);
        HD_CUDA_TRY(cudaGetLastError());
        return HD_OK;
    }
    hd_mma_tuning tu = lib->mma_tuning;
    if (tu.tile_group == 0) tu.tile_group = 16;
    if (tu.super_group == 0) tu.super_group = 16;
    if (tu.cta_group != 1) tu.cta_group = 2;   // default: SM pairs
    tu.cluster = tu.cta_group;
    const dot_io io{q_comp, out_score};
    if (form == HD_FORM_TC_MXF4)
        return run_fmt<FMT_MXF4>(lib, nullptr, q_mz, q_charge, n_q, win, k, out_idx, nullptr, s, tu, &io);
    const int fmt = form_fmt(form);
    if (fmt == FMT_E4M3) return run_fmt<FMT_E4M3>(lib, nullptr, q_mz, q_charge, n_q, win, k, out_idx, nullptr, s, tu, &io);
    if (fmt == FMT_BF16) return run_fmt<FMT_BF16>(lib, nullptr, q_mz, q_charge, n_q, win, k, out_idx, nullptr, s, tu, &io);
    return run_fmt<FMT_E2M1>(lib, nullptr, q_mz, q_charge, n_q, win, k, out_idx, nullptr, s, tu, &io);
}

hd_status hd_peak_mma_run(hd_search_form form, uint32_t launches, hd_peak_result *out)
{
    const bool mx = form == HD_FORM_TC_MXF4;
    const int fmt = form_fmt(form);
    using peak_fn = void (*)(uint32_t, uint64_t, uint32_t *);
    const peak_fn kern = fmt == FMT_BF16 ? k_peak_mma2<FMT_BF16>
                       : (fmt == FMT_E4M3 ? k_peak_mma2<FMT_E4M3> : k_peak_mma2<FMT_E2M1>);
    const void *fn = mx ? (const void *)k_peak_mxf4 : (const void *)kern;
    int dev = 0, n_sms = 0;
    HD_CUDA_TRY(cudaGetDevice(&dev));
    HD_CUDA_TRY(cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev));
    HD_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PEAK_SMEM_BYTES));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((uint32_t)n_sms / 2u * 2u);
    cfg.blockDim = dim3(PEAK_THREADS);
    cfg.dynamicSmemBytes = PEAK_SMEM_BYTES;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n_cl = 0;
    HD_CUDA_TRY(cudaOccupancyMaxActiveClusters(&n_cl, fn, &cfg));
    if (n_cl < 1) return hd_fail(HD_ERR_UNSUPPORTED, "peak kernel: SM-pair cluster does not fit on this GPU");
    cfg.gridDim = dim3(std::min((uint32_t)n_sms / 2u, (uint32_t)n_cl) * 2u);
    const uint32_t iters = 16384;   // 65,536 instructions per SM pair
    // components of K per instruction: 32 bytes of bf16, e4m3 / e2m1 containers, or packed e2m1
    const uint32_t k_per_instr = mx ? 64u : (fmt == FMT_BF16 ? 16u : 32u);
    const uint32_t n_per_instr = mx ? (uint32_t)TN_MX : (uint32_t)TN;
    const uint64_t flops =
        (uint64_t)(cfg.gridDim.x / 2) * iters * (KB / 32) * 2ull * (2 * TM) * n_per_instr * k_per_instr;
    uint32_t *status = nullptr;
    HD_CUDA_TRY(cudaMalloc(&status, sizeof(uint32_t)));
    HD_CUDA_TRY(cudaMemset(status, 0, sizeof(uint32_t)));
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cfg.stream = s;
    std::vector<double> ms;
    hd_status st = HD_OK;
    for (uint32_t r = 0; r <= launches && st == HD_OK; ++r) {   // launch 0 warms up (and checks mxf4 sums)
        cudaEventRecord(e0, s);
        hd_count_launches(1);
        cudaError_t e = mx ? cudaLaunchKernelEx(&cfg, k_peak_mxf4, iters, r == 0 ? 1u : 0u, (uint64_t)HD_WAIT_NS, status)
                           : cudaLaunchKernelEx(&cfg, kern, iters, (uint64_t)HD_WAIT_NS, status);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            st = hd_cuda_fail(e, "peak kernel launch");
            break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (r > 0) ms.push_back(t);
    }
    uint32_t flags = 0;
    if (st == HD_OK && cudaMemcpy(&flags, status, sizeof(flags), cudaMemcpyDeviceToHost) != cudaSuccess)
        st = hd_fail(HD_ERR_CUDA, "peak kernel: status read failed");
    if (st == HD_OK && (flags & HD_DEV_BAD_INPUT))
        st = hd_fail(HD_ERR_CUDA, "peak kernel: kind::mxf4 sums differ from the exact value");
    else if (st == HD_OK && flags)
        st = hd_fail(flags & HD_DEV_TIMEOUT ? HD_ERR_TIMEOUT : HD_ERR_CUDA, "peak kernel: device wait failed");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(status);
    if (st != HD_OK) return st;
    std::sort(ms.begin(), ms.end());
    out->ops_per_launch = flops;
    out->ms_best = ms.front();
    out->best_per_s = (double)flops / (ms.front() * 1e-3);
    out->median_per_s = (double)flops / (ms[ms.size() / 2] * 1e-3);
    out->sms = cfg.gridDim.x;
    out->launches = (uint32_t)ms.size();
    return HD_OK;
}
