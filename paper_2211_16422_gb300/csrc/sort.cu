// sort.cu -- device exclusive scan and the stable (charge, m/z) radix sort
// behind the library layout and the query order (Section 3.4 filters
// candidates by charge and precursor m/z, so sorted rows make every window a
// contiguous range).
#include "hd_internal.cuh"

// ---------------------------------------------------------------------------
// Exclusive scan of uint32: out[i] = sum(in[0..i)), out[n] = total.
// Three-phase (per-CTA scan, scan of CTA totals, add), recursive on the totals.
// A call with arena.base == nullptr only sizes the arena.
// ---------------------------------------------------------------------------
namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER_THREAD = 4;
constexpr uint32_t SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;

__global__ void __launch_bounds__(SCAN_THREADS)
k_scan_tiles(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, uint32_t n,
             uint32_t *__restrict__ tile_sums)
{
    __shared__ uint32_t warp_tot[SCAN_THREADS / 32];
    const uint32_t base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER_THREAD;
    uint32_t v[SCAN_PER_THREAD], run = 0;
#pragma unroll
    for (int j = 0; j < SCAN_PER_THREAD; ++j) {
        v[j] = base + j < n ? in[base + j] : 0u;
        const uint32_t t = v[j];
        v[j] = run;
        run += t;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = run;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t x = warp_tot[lane], xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        warp_tot[lane] = xi - x;   // exclusive prefix of warp totals
        if (lane == 31) tile_sums[blockIdx.x] = xi;
    }
    __syncthreads();
    const uint32_t pre = warp_tot[w] + incl - run;
#pragma unroll
    for (int j = 0; j < SCAN_PER_THREAD; ++j)
        if (base + j < n) out[base + j] = pre + v[j];
}

__global__ void k_scan_add(uint32_t *__restrict__ out, uint32_t n, const uint32_t *__restrict__ tile_off)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_off[i / SCAN_TILE];
    if (i == 0) out[n] = tile_off[(n + SCAN_TILE - 1) / SCAN_TILE];
}

}  // namespace

void hd_exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint32_t n, hd_arena &arena,
                           cudaStream_t s)
{
    const uint32_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    uint32_t *sums = arena.take<uint32_t>(tiles + 1);
    uint32_t *offs = arena.take<uint32_t>(tiles + 1);
    if (!arena.base) {
        if (tiles > 1) hd_exclusive_scan_u32(nullptr, nullptr, tiles, arena, s);
        return;
    }
    if (n == 0) {
        cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
        return;
    }
    hd_count_launches(1), k_scan_tiles<<<tiles, SCAN_THREADS, 0, s>>>(in, out, n, sums);
    if (tiles > 1) {
        hd_exclusive_scan_u32(sums, offs, tiles, arena, s);
    } else {
        cudaMemsetAsync(offs, 0, sizeof(uint32_t), s);
        cudaMemcpyAsync(offs + 1, sums, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    }
    hd_count_launches(1), k_scan_add<<<hd_ceil_div(n, 256), 256, 0, s>>>(out, n, offs);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (charge, m/z): eight 8-bit passes over an
// order-preserving image of the IEEE double, then one pass over the charge
// (and one over the group when given).  Stability keeps equal keys in input
// order, so ties fall to the input index.  Small inputs take k_sort_small.
// ---------------------------------------------------------------------------
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr uint32_t RS_TILE = RS_THREADS * RS_ROUNDS;

// Monotone map of a double onto uint64 (-0.0 folded onto +0.0).
__device__ __forceinline__ uint64_t order_key(double x)
{
    if (x == 0.0) x = 0.0;
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_make_keys(const double *__restrict__ mz, uint32_t n, uint64_t *__restrict__ keys,
                            uint32_t *__restrict__ idx)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        keys[i] = order_key(mz[i]);
        idx[i] = i;
    }
}

// BYTE_KEY: the digit is aux[idx[i]] (charge or group); else a byte of keys[i].
template <bool BYTE_KEY>
__device__ __forceinline__ uint32_t digit_of(const uint64_t *keys, const uint32_t *idx,
                                             const uint8_t *aux, uint32_t i, int shift)
{
    if (BYTE_KEY) return aux[idx[i]];
    return (uint32_t)(keys[i] >> shift) & 0xFFu;
}

template <bool BYTE_KEY>
__global__ void __launch_bounds__(RS_THREADS)
k_hist(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ idx,
       const uint8_t *__restrict__ charge, uint32_t n, int shift, uint32_t *__restrict__ hist)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const uint32_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[digit_of<BYTE_KEY>(keys, idx, charge, i, shift)], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

template <bool BYTE_KEY>
__global__ void __launch_bounds__(RS_THREADS)
k_scatter(const uint64_t *__restrict__ keys_in, const uint32_t *__restrict__ idx_in,
          const uint8_t *__restrict__ charge, uint32_t n, int shift,
          const uint32_t *__restrict__ offs, uint64_t *__restrict__ keys_out,
          uint32_t *__restrict__ idx_out)
{
    constexpr int NW = RS_THREADS / 32;
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[NW][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    run[threadIdx.x] = offs[threadIdx.x * gridDim.x + blockIdx.x];
    const uint32_t base = blockIdx.x * RS_TILE;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const uint32_t i = base + r * RS_THREADS + threadIdx.x;
        const bool ok = i < n;
        const uint32_t d = ok ? digit_of<BYTE_KEY>(keys_in, idx_in, charge, i, shift) : 256u + lane;
#pragma unroll
        for (int j = 0; j < NW; ++j) wcnt[j][threadIdx.x] = 0;
        __syncthreads();
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt_mask);
        if (ok && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (ok) {
            uint32_t pos = run[d] + rank;
            for (int j = 0; j < w; ++j) pos += wcnt[j][d];
            if (!BYTE_KEY) keys_out[pos] = keys_in[i];
            idx_out[pos] = idx_in[i];
        }
        __syncthreads();
        uint32_t tot = 0;
#pragma unroll
        for (int j = 0; j < NW; ++j) tot += wcnt[j][threadIdx.x];
        run[threadIdx.x] += tot;
        __syncthreads();
    }
}

// Up to SMALL_SORT_MAX items: one CTA sorts them in shared memory by a
// bitonic network over the composite key (group, charge, m/z image, input
// index) in two 64-bit words -- the same total order the stable radix passes
// give, in one launch instead of about thirty (small query batches, served
// requests).  np is n rounded up to a power of two; the padding keys sort last.
constexpr uint32_t SMALL_SORT_MAX = 4096;
constexpr int SMALL_SORT_THREADS = 1024;

__global__ void __launch_bounds__(SMALL_SORT_THREADS)
k_sort_small(const double *__restrict__ mz, const uint8_t *__restrict__ charge, const uint8_t *__restrict__ group,
             uint32_t n, uint32_t np, uint32_t *__restrict__ perm)
{
    extern __shared__ ulonglong2 sk[];
    for (uint32_t i = threadIdx.x; i < np; i += blockDim.x) {
        ulonglong2 v = make_ulonglong2(~0ull, ~0ull);
        if (i < n) {
            const uint64_t m = order_key(mz[i]);
            v.x = ((uint64_t)(group ? group[i] : 0u) << 56) | ((uint64_t)charge[i] << 48) | (m >> 16);
            v.y = ((m & 0xFFFFull) << 32) | i;
        }
        sk[i] = v;
    }
    __syncthreads();
    for (uint32_t k = 2; k <= np; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < np; i += blockDim.x) {
                const uint32_t l = i ^ j;
                if (l > i) {
                    const ulonglong2 a = sk[i], b = sk[l];
                    const bool a_gt = a.x > b.x || (a.x == b.x && a.y > b.y);
                    if (a_gt == ((i & k) == 0)) {   // ascending runs where bit k of i is 0
                        sk[i] = b;
                        sk[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) perm[i] = (uint32_t)sk[i].y;
}

}  // namespace

void hd_sort_charge_mz(const double *mz, const uint8_t *charge, const uint8_t *group, uint32_t n,
                       uint32_t *perm, hd_arena &arena, cudaStream_t s)
{
    const uint32_t tiles = (n + RS_TILE - 1) / RS_TILE;
    uint64_t *ka = arena.take<uint64_t>(n), *kb = arena.take<uint64_t>(n);
    uint32_t *ia = arena.take<uint32_t>(n), *ib = arena.take<uint32_t>(n);
    uint32_t *hist = arena.take<uint32_t>((size_t)256 * tiles + 1);
    uint32_t *offs = arena.take<uint32_t>((size_t)256 * tiles + 1);
    const size_t mark = arena.used;
    auto scan = [&]() {
        arena.used = mark;
        hd_exclusive_scan_u32(hist, offs, 256 * tiles, arena, s);
    };
    if (!arena.base) {
        scan();
        return;
    }
    if (n == 0) return;
    if (n <= SMALL_SORT_MAX) {
        uint32_t np = 1;
        while (np < n) np <<= 1;
        const size_t smem = (size_t)np * sizeof(ulonglong2);
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_sort_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(SMALL_SORT_MAX * 16));
        hd_count_launches(1), k_sort_small<<<1, SMALL_SORT_THREADS, smem, s>>>(mz, charge, group, n, np, perm);
        return;
    }
    hd_count_launches(1), k_make_keys<<<hd_ceil_div(n, 256), 256, 0, s>>>(mz, n, ka, ia);
    for (int pass = 0; pass < 8; ++pass) {
        hd_count_launches(1), k_hist<false><<<tiles, RS_THREADS, 0, s>>>(ka, ia, charge, n, 8 * pass, hist);
        scan();
        hd_count_launches(1), k_scatter<false><<<tiles, RS_THREADS, 0, s>>>(ka, ia, charge, n, 8 * pass, offs, kb, ib);
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *ti = ia; ia = ib; ib = ti;
    }
    hd_count_launches(1), k_hist<true><<<tiles, RS_THREADS, 0, s>>>(ka, ia, charge, n, 0, hist);
    scan();
    hd_count_launches(1), k_scatter<true><<<tiles, RS_THREADS, 0, s>>>(ka, ia, charge, n, 0, offs, kb,
                                                                        group ? ib : perm);
    if (group) {   // most significant key last
        hd_count_launches(1), k_hist<true><<<tiles, RS_THREADS, 0, s>>>(ka, ib, group, n, 0, hist);
        scan();
        hd_count_launches(1), k_scatter<true><<<tiles, RS_THREADS, 0, s>>>(ka, ib, group, n, 0, offs, kb, perm);
    }
}
