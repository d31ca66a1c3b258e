// item_memory.cu -- position and level hypervectors (Section 3.3.1-3.3.2).
//
// Random bits and permutation keys come from Philox4x32-10 (Salmon et al.,
// SC'11): word i of stream s under key `seed` is component i%4 of the block at
// counter (i/4, s, 0, 0).  Streams: 0 = F_0 bits, 1 = position permutation
// keys, 2 = L_0 bits, 3 = level permutation keys, 4 = flip positions of the
// position walk, 5 = bits of independent random position HVs.
#include "hd_internal.cuh"

namespace {

struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += W0;
        k1 += W1;
    }
    return c;
}

// out[i] = word i of Philox stream `stream`, i < n.
__global__ void k_stream_words(uint64_t seed, uint32_t stream, uint32_t n, uint32_t *out)
{
    const uint32_t blk = blockIdx.x * blockDim.x + threadIdx.x;   // one Philox block
    if (blk * 4u >= n) return;
    const u32x4 r = philox4x32_10(u32x4{blk, stream, 0u, 0u}, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint32_t v[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (blk * 4u + j < n) out[blk * 4u + j] = v[j];
}

// rank[d] = #{e : (key[e], e) < (key[d], d)}: a position's place in the
// ascending order of (key, position).  Keys are staged through shared memory.
__global__ void k_rank(const uint32_t *key, uint32_t D, uint32_t *rank)
{
    __shared__ uint32_t tile[1024];
    const uint32_t d = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t kd = d < D ? key[d] : 0u;
    uint32_t r = 0;
    for (uint32_t base = 0; base < D; base += 1024) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < 1024; i += blockDim.x)
            tile[i] = base + i < D ? key[base + i] : 0xFFFFFFFFu;
        __syncthreads();
        const uint32_t lim = min(1024u, D - base);
        for (uint32_t i = 0; i < lim; ++i) {
            const uint32_t ke = tile[i], e = base + i;
            r += (ke < kd) || (ke == kd && e < d);
        }
    }
    if (d < D) rank[d] = r;
}

// Row i of a nested-flip table: base bits XOR [rank[d] < flips(i)], with
// flips(i) = floor(i * total / (rows - 1)).  One thread per output word.
__global__ void k_flip_table(const uint32_t *base32, const uint32_t *rank, uint32_t D, uint32_t rows,
                             uint64_t total, uint64_t *out)
{
    const uint32_t W = D / 64u;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)rows * W) return;
    const uint32_t row = (uint32_t)(t / W), w = (uint32_t)(t % W);
    const uint64_t flips = rows > 1 ? ((uint64_t)row * total) / (uint64_t)(rows - 1) : 0ull;
    uint64_t word = (uint64_t)base32[2 * w] | ((uint64_t)base32[2 * w + 1] << 32);
    uint64_t mask = 0;
#pragma unroll 8
    for (uint32_t b = 0; b < 64; ++b)
        mask |= (uint64_t)(rank[w * 64u + b] < flips) << b;
    out[t] = word ^ mask;
}

// Position walk, step masks: row i >= 1 has exactly `alpha` distinct bits set,
// drawn by Floyd's algorithm (k = 0..alpha-1: j = D - alpha + k, t = word
// (stream 4, i * 256 + k) mod (j + 1); t unless already drawn, else j); row 0
// is empty.  One thread per row.
__global__ void k_walk_masks(uint64_t seed, uint32_t D, uint32_t rows, uint32_t alpha, uint64_t *masks)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const uint32_t W = D / 64u;
    uint64_t *m = masks + (size_t)i * W;
    for (uint32_t w = 0; w < W; ++w) m[w] = 0ull;
    if (i == 0) return;
    uint32_t chosen[256];
    u32x4 r{};
    for (uint32_t k = 0; k < alpha; ++k) {
        if ((k & 3u) == 0)
            r = philox4x32_10(u32x4{(i * 256u + k) >> 2, 4u, 0u, 0u}, (uint32_t)seed, (uint32_t)(seed >> 32));
        const uint32_t word = (k & 3u) == 0 ? r.x : (k & 3u) == 1 ? r.y : (k & 3u) == 2 ? r.z : r.w;
        const uint32_t j = D - alpha + k;
        uint32_t t = word % (j + 1u);
        for (uint32_t q = 0; q < k; ++q)
            if (chosen[q] == t) {
                t = j;
                break;
            }
        chosen[k] = t;
        m[t >> 6] ^= 1ull << (t & 63u);
    }
}

// F_i = F_0 XOR (XOR of the masks of rows 1..i): one thread per 64-bit column.
__global__ void k_walk_scan(const uint32_t *base32, const uint64_t *masks, uint32_t D, uint32_t rows, uint64_t *out)
{
    const uint32_t W = D / 64u, w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    uint64_t acc = (uint64_t)base32[2 * w] | ((uint64_t)base32[2 * w + 1] << 32);
    for (uint32_t i = 0; i < rows; ++i) {
        acc ^= masks[(size_t)i * W + w];
        out[(size_t)i * W + w] = acc;
    }
}

// Independent random position HVs: bit d of row i is bit d%32 of word
// (stream 5, i * D/32 + d/32).  One thread per 64-bit word.
__global__ void k_random_table(uint64_t seed, uint32_t D, uint32_t rows, uint64_t *out)
{
    const uint32_t W = D / 64u;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (uint64_t)rows * W) return;
    const uint32_t row = (uint32_t)(t / W), w = (uint32_t)(t % W);
    const uint32_t idx = row * (D / 32u) + 2u * w;   // even: both words share one Philox block
    const u32x4 r = philox4x32_10(u32x4{idx >> 2, 5u, 0u, 0u}, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint32_t lo = (idx & 3u) == 0 ? r.x : r.z, hi = (idx & 3u) == 0 ? r.y : r.w;
    out[t] = (uint64_t)lo | ((uint64_t)hi << 32);
}

}  // namespace

void hd_random_words_launch(uint64_t seed, uint32_t stream, uint32_t n, uint32_t *out, cudaStream_t s)
{
    const uint32_t blocks = hd_ceil_div(n, 4);
    hd_count_launches(1), k_stream_words<<<hd_ceil_div(blocks, 256), 256, 0, s>>>(seed, stream, n, out);
}

hd_status hd_item_memory_build(hd_ctx *ctx, cudaStream_t s)
{
    const uint32_t D = ctx->p.dim;
    uint32_t *tmp = nullptr;
    HD_CUDA_TRY(cudaMallocAsync(&tmp, sizeof(uint32_t) * (size_t)(D / 32 + D) * 2, s));
    uint32_t *F0 = tmp, *keyF = F0 + D / 32, *L0 = keyF + D, *keyL = L0 + D / 32;
    const uint64_t seed = ctx->p.seed;
    auto words = [&](uint32_t stream, uint32_t n, uint32_t *out) { hd_random_words_launch(seed, stream, n, out, s); };
    words(0, D / 32, F0);
    words(1, D, keyF);
    words(2, D / 32, L0);
    words(3, D, keyL);
    hd_count_launches(1), k_rank<<<hd_ceil_div(D, 256), 256, 0, s>>>(keyF, D, ctx->rank_F);
    hd_count_launches(1), k_rank<<<hd_ceil_div(D, 256), 256, 0, s>>>(keyL, D, ctx->rank_L);
    const size_t nF = (size_t)ctx->p.n_bins * ctx->W, nL = (size_t)ctx->p.n_levels * ctx->W;
    if (ctx->p.position_mode == HD_POS_WALK) {
        uint64_t *masks = nullptr;
        HD_CUDA_TRY(cudaMallocAsync(&masks, nF * 8, s));
        hd_count_launches(1), k_walk_masks<<<hd_ceil_div(ctx->p.n_bins, 128), 128, 0, s>>>(seed, D, ctx->p.n_bins,
                                                                                         ctx->p.alpha, masks);
        hd_count_launches(1), k_walk_scan<<<hd_ceil_div(ctx->W, 64), 64, 0, s>>>(F0, masks, D, ctx->p.n_bins, ctx->F);
        HD_CUDA_TRY(cudaFreeAsync(masks, s));
    } else if (ctx->p.position_mode == HD_POS_RANDOM) {
        hd_count_launches(1), k_random_table<<<hd_ceil_div(nF, 256), 256, 0, s>>>(seed, D, ctx->p.n_bins, ctx->F);
    } else {
        hd_count_launches(1), k_flip_table<<<hd_ceil_div(nF, 256), 256, 0, s>>>(F0, ctx->rank_F, D, ctx->p.n_bins,
                                                          ctx->p.alpha, ctx->F);
    }
    hd_count_launches(1), k_flip_table<<<hd_ceil_div(nL, 256), 256, 0, s>>>(L0, ctx->rank_L, D, ctx->p.n_levels,
                                                      (uint64_t)(D / 2), ctx->L);
    HD_CUDA_TRY(cudaGetLastError());
    HD_CUDA_TRY(cudaFreeAsync(tmp, s));
    return HD_OK;
}
