// encode.cu -- spectrum vectors -> binary hypervectors (Section 3.3, Eq. 1;
// the random-projection baseline of Section 4.2 as a second encoder), and
// multi-bit components (Section 4.3).
//
// out_d = [2 c_d >= n], with c_d the number of peaks whose bound bit
// F_bin XOR L_level is 1 at d (Eq. 1's bipolar sum is n - 2 c_d and the
// binarisation maps a sum <= 0 to -1, bit 1).
//
// One warp per spectrum; each lane owns WPL 64-bit words of a 32*WPL-word
// slice of the HV and keeps, per word, a bit-sliced counter: plane i holds
// bit i of the 64 per-bit counts.  The warp reads its peaks 32 at a time
// (one per lane), drops the invalid ones and packs the rest into a per-warp
// list in shared memory.  Bound words then enter the counter sixteen at a
// time through a Harley-Seal tree of full adders, which keeps planes 0..3
// exact and emits one carry of weight 16 (rippled from plane 4); the rest of
// a chunk goes four at a time (full adders into planes 0 and 1) and then one
// at a time.  The majority test compares the planes with ceil(n/2) from the
// top bit down.
#include "hd_internal.cuh"

namespace {

constexpr int ENC_PLANES = 10;          // counts up to 1023 peaks
constexpr uint32_t ENC_MAX_PEAKS = (1u << ENC_PLANES) - 1u;
constexpr int ENC_WARPS = 8;
// Widest per-lane word slice of the binary encoder.  Timed at D = 8192 for
// 200,000 spectra of 50 peaks: 2 words per lane with two CTAs per SM
// (128 registers) 1.13 ms; 200 registers and one CTA per SM 1.58 ms; 80
// registers (three CTAs, spills) 1.17 ms; 1 word per lane 1.33 ms; 4 words
// 1.35 ms; the four-at-a-time adder without the tree 2.03 ms.
#ifndef HD_ENC_WPL_MAX
#define HD_ENC_WPL_MAX 2
#endif

__device__ __forceinline__ uint64_t maj3(uint64_t a, uint64_t b, uint64_t c) { return (a & b) | (a & c) | (b & c); }

// Transpose of an 8 x 8 bit matrix held as 8 bytes (row r = byte r, column
// c = bit c): three rounds of masked exchanges of the off-diagonal 1 x 1,
// 2 x 2 and 4 x 4 blocks (H. S. Warren, Hacker's Delight, section 7-3).
__device__ __forceinline__ uint64_t transpose8x8(uint64_t x)
{
    uint64_t t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
    x ^= t ^ (t << 7);
    t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
    x ^= t ^ (t << 14);
    t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
    x ^= t ^ (t << 28);
    return x;
}

// Bound words F_bin XOR L_level of one peak (pk = (bin, level)) for the
// lane's WPL words wl, wl + 32, ...; 0 beyond the row unless FULL (W a
// multiple of 32 * WPL, every word in range).
template <int WPL, bool FULL>
__device__ __forceinline__ void bound_words(const uint64_t *__restrict__ F, const uint64_t *__restrict__ L,
                                            uint32_t W, uint2 pk, uint32_t wl, uint64_t (&x)[WPL])
{
    const uint64_t *fr = F + (size_t)pk.x * W + wl, *lr = L + (size_t)pk.y * W + wl;
#pragma unroll
    for (int j = 0; j < WPL; ++j)
        x[j] = (FULL || wl + 32u * j < W) ? (__ldg(fr + 32 * j) ^ __ldg(lr + 32 * j)) : 0ull;
}

// Full adder of plane `plane` with inputs a, b: the plane takes the sum bit,
// `carry` the carry bit (weight of the next plane).
template <int WPL>
__device__ __forceinline__ void full_add(uint64_t (&c)[WPL][ENC_PLANES], int plane, const uint64_t (&a)[WPL],
                                         const uint64_t (&b)[WPL], uint64_t (&carry)[WPL])
{
#pragma unroll
    for (int j = 0; j < WPL; ++j) {
        const uint64_t u = c[j][plane];
        carry[j] = maj3(u, a[j], b[j]);
        c[j][plane] = u ^ a[j] ^ b[j];
    }
}

// Adds carry words of weight 2^P into planes P..Q-1.
template <int P, int Q, int WPL>
__device__ __forceinline__ void ripple(uint64_t (&c)[WPL][ENC_PLANES], const uint64_t (&k)[WPL])
{
#pragma unroll
    for (int j = 0; j < WPL; ++j) {
        uint64_t carry = k[j];
#pragma unroll
        for (int i = P; i < Q; ++i) {
            const uint64_t t = c[j][i] & carry;
            c[j][i] ^= carry;
            carry = t;
        }
    }
}

// The same, over the planes that can be non-zero once the count reaches
// `added` (a warp-uniform branch: planes up to 6 hold counts below 128).
template <int P, int WPL>
__device__ __forceinline__ void ripple_to(uint64_t (&c)[WPL][ENC_PLANES], const uint64_t (&k)[WPL], uint32_t added)
{
    if (added < 128u) ripple<P, 7, WPL>(c, k);
    else ripple<P, ENC_PLANES, WPL>(c, k);
}

// Bit-sliced counts of the bound words of the valid peaks of [beg, end):
// c[j][i] holds bit i of the 64 per-bit counts of the lane's word j (words
// w0 + lane + 32 j).  A peak with bin >= n_bins or level >= n_levels is
// skipped and sets `bad` in every lane.  Called by all 32 lanes of a warp with the same
// row; `pk` is the warp's 32-entry list in shared memory.  Returns the
// number of peaks counted.
template <int WPL, bool FULL>
__device__ __forceinline__ uint32_t sliced_count(const uint64_t *__restrict__ F, uint32_t n_bins,
                                                 const uint64_t *__restrict__ L, uint32_t n_levels, uint32_t W,
                                                 const uint32_t *__restrict__ bins,
                                                 const uint8_t *__restrict__ levels, uint32_t beg, uint32_t end,
                                                 uint32_t w0, uint32_t lane, uint64_t (&c)[WPL][ENC_PLANES],
                                                 bool &bad, uint2 *pk)
{
#pragma unroll
    for (int j = 0; j < WPL; ++j)
#pragma unroll
        for (int i = 0; i < ENC_PLANES; ++i) c[j][i] = 0;
    const uint32_t wl = w0 + lane;
    uint32_t added = 0;
    for (uint32_t p0 = beg; p0 < end; p0 += 32) {
        const uint32_t p = p0 + lane;
        bool ok = false;
        uint32_t b = 0, l = 0;
        if (p < end) {
            b = __ldg(bins + p);
            l = __ldg(levels + p);
            ok = b < n_bins && l < n_levels;
        }
        if (__ballot_sync(0xFFFFFFFFu, p < end && !ok)) bad = true;   // every lane learns of a bad peak
        const uint32_t valid = __ballot_sync(0xFFFFFFFFu, ok);
        const uint32_t nv = __popc(valid);
        __syncwarp();   // the previous chunk's reads of pk are done
        if (ok) pk[__popc(valid & ((1u << lane) - 1u))] = make_uint2(b, l);
        __syncwarp();
        uint32_t t = 0;
        for (; t + 16 <= nv; t += 16) {
            // Harley-Seal: pairs into plane 0 give weight-2 carries, pairs of
            // those into plane 1 weight 4, then plane 2 weight 8, plane 3 weight 16.
            uint64_t xa[WPL], xb[WPL], k2a[WPL], k2b[WPL], k4a[WPL], k4b[WPL], k8a[WPL], k8b[WPL], k16[WPL];
            auto pair = [&](uint32_t i, uint64_t(&k2)[WPL]) {
                bound_words<WPL, FULL>(F, L, W, pk[t + i], wl, xa);
                bound_words<WPL, FULL>(F, L, W, pk[t + i + 1], wl, xb);
                full_add<WPL>(c, 0, xa, xb, k2);
            };
            pair(0, k2a);
            pair(2, k2b);
            full_add<WPL>(c, 1, k2a, k2b, k4a);
            pair(4, k2a);
            pair(6, k2b);
            full_add<WPL>(c, 1, k2a, k2b, k4b);
            full_add<WPL>(c, 2, k4a, k4b, k8a);
            pair(8, k2a);
            pair(10, k2b);
            full_add<WPL>(c, 1, k2a, k2b, k4a);
            pair(12, k2a);
            pair(14, k2b);
            full_add<WPL>(c, 1, k2a, k2b, k4b);
            full_add<WPL>(c, 2, k4a, k4b, k8b);
            full_add<WPL>(c, 3, k8a, k8b, k16);
            added += 16;
            ripple_to<4, WPL>(c, k16, added);
        }
        for (; t + 4 <= nv; t += 4) {
            uint64_t xa[WPL], xb[WPL], k2a[WPL], k2b[WPL], k4[WPL];
            bound_words<WPL, FULL>(F, L, W, pk[t], wl, xa);
            bound_words<WPL, FULL>(F, L, W, pk[t + 1], wl, xb);
            full_add<WPL>(c, 0, xa, xb, k2a);
            bound_words<WPL, FULL>(F, L, W, pk[t + 2], wl, xa);
            bound_words<WPL, FULL>(F, L, W, pk[t + 3], wl, xb);
            full_add<WPL>(c, 0, xa, xb, k2b);
            full_add<WPL>(c, 1, k2a, k2b, k4);
            added += 4;
            ripple_to<2, WPL>(c, k4, added);
        }
        for (; t < nv; ++t) {
            uint64_t x[WPL];
            bound_words<WPL, FULL>(F, L, W, pk[t], wl, x);
            ++added;
            ripple_to<0, WPL>(c, x, added);
        }
    }
    return added;
}

template <int WPL, bool FULL>
__global__ void __launch_bounds__(ENC_WARPS * 32, WPL == 2 ? 2 : 1)
k_encode(const uint64_t *__restrict__ F, uint32_t n_bins, const uint64_t *__restrict__ L,
         uint32_t n_levels, uint32_t W, const uint32_t *__restrict__ off,
         const uint32_t *__restrict__ bins, const uint8_t *__restrict__ levels, uint32_t n_spec,
         uint64_t *__restrict__ out, uint32_t *status)
{
    __shared__ uint2 s_pk[ENC_WARPS][32];
    const uint32_t wi = threadIdx.x >> 5;
    const uint32_t sp = blockIdx.x * ENC_WARPS + wi;
    const uint32_t lane = threadIdx.x & 31;
    if (sp >= n_spec) return;
    uint32_t beg = off[sp], end = off[sp + 1];
    if (end < beg || end - beg > ENC_MAX_PEAKS) {
        if (lane == 0) hd_flag(status, HD_DEV_BAD_INPUT);
        end = beg;   // encode as an empty row
    }
    bool any_bad = false;
    for (uint32_t w0 = 0; w0 < W; w0 += 32u * WPL) {
        uint64_t c[WPL][ENC_PLANES];
        const uint32_t added = sliced_count<WPL, FULL>(F, n_bins, L, n_levels, W, bins, levels, beg, end, w0, lane,
                                                       c, any_bad, s_pk[wi]);
        const uint32_t thresh = (added + 1) >> 1;   // c >= ceil(n/2)  <=>  2c >= n
#pragma unroll
        for (int j = 0; j < WPL; ++j) {
            const uint32_t w = w0 + lane + 32u * j;
            uint64_t gt = 0, eq = ~0ull;
#pragma unroll
            for (int i = ENC_PLANES - 1; i >= 0; --i) {
                if ((thresh >> i) & 1u) eq &= c[j][i];
                else gt |= eq & c[j][i];
            }
            if (FULL || w < W) out[(size_t)sp * W + w] = gt | eq;
        }
    }
    if (any_bad && lane == 0) hd_flag(status, HD_DEV_BAD_INPUT);
}

// Random-projection encoder (the LSH baseline of Section 4.2): out_d = [I_d <= 0]
// with I_d = sum over peaks of (level + 1) * (1 - 2 F_bin[d]).  One warp per
// spectrum; each lane owns one 64-bit word at a time and keeps its 64 sums in
// registers.
__global__ void __launch_bounds__(ENC_WARPS * 32)
k_encode_projection(const uint64_t *__restrict__ F, uint32_t n_bins, uint32_t n_levels, uint32_t W,
                    const uint32_t *__restrict__ off, const uint32_t *__restrict__ bins,
                    const uint8_t *__restrict__ levels, uint32_t n_spec, uint64_t *__restrict__ out,
                    uint32_t *status)
{
    const uint32_t sp = blockIdx.x * ENC_WARPS + (threadIdx.x >> 5);
    const uint32_t lane = threadIdx.x & 31;
    if (sp >= n_spec) return;
    uint32_t beg = off[sp], end = off[sp + 1];
    if (end < beg || end - beg > ENC_MAX_PEAKS) {
        if (lane == 0) hd_flag(status, HD_DEV_BAD_INPUT);
        end = beg;   // encode as an empty row
    }
    bool any_bad = false;
    for (uint32_t w = lane; w < W; w += 32) {
        int32_t acc[64];
#pragma unroll
        for (int b = 0; b < 64; ++b) acc[b] = 0;
        for (uint32_t p = beg; p < end; ++p) {
            const uint32_t bn = __ldg(bins + p), l = __ldg(levels + p);
            if (bn >= n_bins || l >= n_levels) {
                any_bad = true;
                continue;
            }
            const uint64_t x = __ldg(F + (size_t)bn * W + w);
            const int32_t wt = (int32_t)l + 1;
#pragma unroll
            for (int b = 0; b < 64; ++b) acc[b] += ((x >> b) & 1ull) ? -wt : wt;
        }
        uint64_t o = 0;
#pragma unroll
        for (int b = 0; b < 64; ++b) o |= (uint64_t)(acc[b] <= 0) << b;
        out[(size_t)sp * W + w] = o;
    }
    if (any_bad) hd_flag(status, HD_DEV_BAD_INPUT);
}

// Multi-bit components (Section 4.3 reading): h_d = sign(I_d) *
// floor((2 m |I_d| + M) / (2 M)), M = max_d |I_d|, h = 0 when M = 0, with
// I_d = sum over peaks of w (1 - 2 x_d): x = F_bin XOR L_level and w = 1
// (Eq. 1), or x = F_bin and w = level + 1 (projection).  One warp per
// spectrum and two passes over its peaks: the first finds M, the second
// recomputes each 64-bit word's sums and writes them quantised, component d
// at byte d of the row.
template <bool PROJ>
__device__ __forceinline__ bool word_sums(const uint64_t *__restrict__ F, uint32_t n_bins,
                                          const uint64_t *__restrict__ L, uint32_t n_levels, uint32_t W,
                                          const uint32_t *__restrict__ bins, const uint8_t *__restrict__ levels,
                                          uint32_t beg, uint32_t end, uint32_t w, int32_t (&acc)[64])
{
    bool bad = false;
#pragma unroll
    for (int b = 0; b < 64; ++b) acc[b] = 0;
    for (uint32_t p = beg; p < end; ++p) {
        const uint32_t bn = __ldg(bins + p), l = __ldg(levels + p);
        if (bn >= n_bins || l >= n_levels) {
            bad = true;
            continue;
        }
        const uint64_t x = PROJ ? __ldg(F + (size_t)bn * W + w) : (__ldg(F + (size_t)bn * W + w) ^ __ldg(L + (size_t)l * W + w));
        const int32_t wt = PROJ ? (int32_t)l + 1 : 1;
#pragma unroll
        for (int b = 0; b < 64; ++b) acc[b] += ((x >> b) & 1ull) ? -wt : wt;
    }
    return bad;
}

template <bool PROJ>
__global__ void __launch_bounds__(ENC_WARPS * 32)
k_encode_mb(const uint64_t *__restrict__ F, uint32_t n_bins, const uint64_t *__restrict__ L, uint32_t n_levels,
            uint32_t W, const uint32_t *__restrict__ off, const uint32_t *__restrict__ bins,
            const uint8_t *__restrict__ levels, uint32_t n_spec, uint32_t m, int8_t *__restrict__ out,
            uint32_t *status)
{
    const uint32_t sp = blockIdx.x * ENC_WARPS + (threadIdx.x >> 5);
    const uint32_t lane = threadIdx.x & 31;
    if (sp >= n_spec) return;
    uint32_t beg = off[sp], end = off[sp + 1];
    if (end < beg || end - beg > ENC_MAX_PEAKS) {
        if (lane == 0) hd_flag(status, HD_DEV_BAD_INPUT);
        end = beg;   // encode as an empty row
    }
    bool bad = false;
    int32_t acc[64];
    uint32_t M = 0;
    for (uint32_t w = lane; w < W; w += 32) {
        bad |= word_sums<PROJ>(F, n_bins, L, n_levels, W, bins, levels, beg, end, w, acc);
#pragma unroll
        for (int b = 0; b < 64; ++b) M = max(M, (uint32_t)abs(acc[b]));
    }
    M = __reduce_max_sync(0xFFFFFFFFu, M);
    for (uint32_t w = lane; w < W; w += 32) {
        word_sums<PROJ>(F, n_bins, L, n_levels, W, bins, levels, beg, end, w, acc);
        uint32_t p[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) p[i] = 0;
#pragma unroll
        for (int b = 0; b < 64; ++b) {
            const uint32_t a = (uint32_t)abs(acc[b]);
            const int32_t h = M ? (int32_t)((2u * m * a + M) / (2u * M)) : 0;
            p[b >> 2] |= (uint32_t)(uint8_t)(int8_t)(acc[b] < 0 ? -h : h) << (8 * (b & 3));
        }
        uint4 *o = reinterpret_cast<uint4 *>(out + (size_t)sp * W * 64 + (size_t)w * 64);
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = make_uint4(p[4 * i], p[4 * i + 1], p[4 * i + 2], p[4 * i + 3]);
    }
    if (bad) hd_flag(status, HD_DEV_BAD_INPUT);
}

// Multi-bit components of Eq. 1 from the bit-sliced counters of k_encode.
// With c_d the count of 1-bits among the n bound bits, I_d = n - 2 c_d, so
// |I| is largest at the smallest or the largest count: pass 1 finds both from
// the planes (a descent over the planes, no per-bit count), pass 2 recounts
// and maps each component's count through a per-spectrum table h(c), c = 0..n,
// in shared memory.  Same result as k_encode_mb<false>.
template <int WPL, bool FULL>
__global__ void __launch_bounds__(ENC_WARPS * 32)
k_encode_mb_sliced(const uint64_t *__restrict__ F, uint32_t n_bins, const uint64_t *__restrict__ L,
                   uint32_t n_levels, uint32_t W, const uint32_t *__restrict__ off,
                   const uint32_t *__restrict__ bins, const uint8_t *__restrict__ levels, uint32_t n_spec,
                   uint32_t m, int8_t *__restrict__ out, uint32_t *status)
{
    __shared__ int8_t s_tab[ENC_WARPS][ENC_MAX_PEAKS + 1];   // component as a function of the count
    __shared__ uint2 s_pk[ENC_WARPS][32];
    const uint32_t wi = threadIdx.x >> 5;
    const uint32_t sp = blockIdx.x * ENC_WARPS + wi;
    const uint32_t lane = threadIdx.x & 31;
    if (sp >= n_spec) return;
    uint32_t beg = off[sp], end = off[sp + 1];
    if (end < beg || end - beg > ENC_MAX_PEAKS) {
        if (lane == 0) hd_flag(status, HD_DEV_BAD_INPUT);
        end = beg;   // encode as an empty row
    }
    bool bad = false;
    uint64_t c[WPL][ENC_PLANES];
    uint32_t n = 0, cmin = 0xFFFFFFFFu, cmax = 0;
    for (uint32_t w0 = 0; w0 < W; w0 += 32u * WPL) {
        n = sliced_count<WPL, FULL>(F, n_bins, L, n_levels, W, bins, levels, beg, end, w0, lane, c, bad,
                                    s_pk[wi]);
#pragma unroll
        for (int j = 0; j < WPL; ++j) {
            if (w0 + lane + 32u * j >= W) continue;
            // largest count among the 64 bits: keep the bits that are 1 in the highest plane possible
            uint64_t hi_c = ~0ull, lo_c = ~0ull;
            uint32_t mx = 0, mn = 0;
#pragma unroll
            for (int i = ENC_PLANES - 1; i >= 0; --i) {
                const uint64_t t = hi_c & c[j][i];
                if (t) { hi_c = t; mx |= 1u << i; }
                const uint64_t u = lo_c & ~c[j][i];
                if (u) lo_c = u; else mn |= 1u << i;
            }
            cmin = min(cmin, mn);
            cmax = max(cmax, mx);
        }
    }
    cmin = __reduce_min_sync(0xFFFFFFFFu, cmin);
    cmax = __reduce_max_sync(0xFFFFFFFFu, cmax);
    const int32_t a_lo = abs((int32_t)n - 2 * (int32_t)cmin), a_hi = abs(2 * (int32_t)cmax - (int32_t)n);
    const uint32_t M = (uint32_t)max(a_lo, a_hi);
    for (uint32_t cc = lane; cc <= n; cc += 32) {
        const int32_t I = (int32_t)n - 2 * (int32_t)cc;
        const uint32_t a = (uint32_t)abs(I);
        const int32_t h = M ? (int32_t)((2u * m * a + M) / (2u * M)) : 0;
        s_tab[wi][cc] = (int8_t)(I < 0 ? -h : h);
    }
    __syncwarp();
    const int lim = 32 - __clz(n);   // planes that can be non-zero
    for (uint32_t w0 = 0; w0 < W; w0 += 32u * WPL) {
        if (W > 32u * WPL)
            sliced_count<WPL, FULL>(F, n_bins, L, n_levels, W, bins, levels, beg, end, w0, lane, c, bad, s_pk[wi]);
#pragma unroll
        for (int j = 0; j < WPL; ++j) {
            const uint32_t w = w0 + lane + 32u * j;
            if (w >= W) continue;
            uint32_t p[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) p[q] = 0;
            if (lim <= 8) {
                // counts below 256: the eight planes' byte g, transposed as an 8 x 8
                // bit matrix, give the counts of components 8g..8g+7 as bytes
#pragma unroll
                for (int g = 0; g < 8; ++g) {
                    uint64_t x = 0;
#pragma unroll
                    for (int i = 0; i < 8; ++i) x |= ((c[j][i] >> (8 * g)) & 0xFFull) << (8 * i);
                    x = transpose8x8(x);
#pragma unroll
                    for (int b = 0; b < 8; ++b)
                        p[2 * g + (b >> 2)] |= (uint32_t)(uint8_t)s_tab[wi][(x >> (8 * b)) & 0xFF] << (8 * (b & 3));
                }
            } else {
#pragma unroll
                for (int b = 0; b < 64; ++b) {
                    uint32_t cnt = 0;
#pragma unroll
                    for (int i = 0; i < ENC_PLANES; ++i)
                        if (i < lim) cnt |= (uint32_t)((c[j][i] >> b) & 1ull) << i;
                    p[b >> 2] |= (uint32_t)(uint8_t)s_tab[wi][cnt] << (8 * (b & 3));
                }
            }
            uint4 *o = reinterpret_cast<uint4 *>(out + (size_t)sp * W * 64 + (size_t)w * 64);
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = make_uint4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
        }
    }
    if (bad && lane == 0) hd_flag(status, HD_DEV_BAD_INPUT);
}

// Launchers choosing the form without per-word range checks when every
// slice of 32 * WPL words lies inside the row.
template <int WPL>
void mb_sliced(const hd_ctx *ctx, const uint32_t *off, const uint32_t *bins, const uint8_t *levels, uint32_t n,
               uint32_t m, int8_t *out, uint32_t *st, unsigned grid, cudaStream_t s)
{
    hd_count_launches(1);
    if (ctx->W % (32u * WPL) == 0)
        k_encode_mb_sliced<WPL, true><<<grid, ENC_WARPS * 32, 0, s>>>(ctx->F, ctx->p.n_bins, ctx->L, ctx->p.n_levels,
                                                                     ctx->W, off, bins, levels, n, m, out, st);
    else
        k_encode_mb_sliced<WPL, false><<<grid, ENC_WARPS * 32, 0, s>>>(ctx->F, ctx->p.n_bins, ctx->L, ctx->p.n_levels,
                                                                      ctx->W, off, bins, levels, n, m, out, st);
}

template <int WPL>
void binary(const hd_ctx *ctx, const uint32_t *off, const uint32_t *bins, const uint8_t *levels, uint32_t n,
            uint64_t *out, uint32_t *st, unsigned grid, cudaStream_t s)
{
    hd_count_launches(1);
    if (ctx->W % (32u * WPL) == 0)
        k_encode<WPL, true><<<grid, ENC_WARPS * 32, 0, s>>>(ctx->F, ctx->p.n_bins, ctx->L, ctx->p.n_levels, ctx->W,
                                                           off, bins, levels, n, out, st);
    else
        k_encode<WPL, false><<<grid, ENC_WARPS * 32, 0, s>>>(ctx->F, ctx->p.n_bins, ctx->L, ctx->p.n_levels, ctx->W,
                                                            off, bins, levels, n, out, st);
}

}  // namespace

void hd_encode_mb_launch(const hd_ctx *ctx, const uint32_t *off, const uint32_t *bins, const uint8_t *levels,
                         uint32_t n, uint32_t bits, int8_t *out, cudaStream_t s)
{
    const unsigned grid = hd_ceil_div(n, ENC_WARPS);
    uint32_t *st = ctx->status.dev;
    const uint32_t m = hd_comp_max(bits);
    hd_prof_scope timed(HD_KERNEL_ENCODE, s);
    if (ctx->p.encoder == HD_ENC_PROJECTION)
        hd_count_launches(1), k_encode_mb<true><<<grid, ENC_WARPS * 32, 0, s>>>(
            ctx->F, ctx->p.n_bins, ctx->L, ctx->p.n_levels, ctx->W, off, bins, levels, n, m, out, st);
    else if (ctx->W >= 128)
        mb_sliced<4>(ctx, off, bins, levels, n, m, out, st, grid, s);
    else if (ctx->W >= 64)
        mb_sliced<2>(ctx, off, bins, levels, n, m, out, st, grid, s);
    else
        mb_sliced<1>(ctx, off, bins, levels, n, m, out, st, grid, s);
}

void hd_encode_launch(const hd_ctx *ctx, const uint32_t *off, const uint32_t *bins,
                      const uint8_t *levels, uint32_t n, uint64_t *out, cudaStream_t s)
{
    const uint32_t W = ctx->W;
    const unsigned grid = hd_ceil_div(n, ENC_WARPS);
    uint32_t *st = ctx->status.dev;
    hd_prof_scope timed(HD_KERNEL_ENCODE, s);
    if (ctx->p.encoder == HD_ENC_PROJECTION)
        hd_count_launches(1), k_encode_projection<<<grid, ENC_WARPS * 32, 0, s>>>(ctx->F, ctx->p.n_bins,
                                                                              ctx->p.n_levels, W, off, bins,
                                                                              levels, n, out, st);
#if HD_ENC_WPL_MAX >= 4
    else if (W >= 128)
        binary<4>(ctx, off, bins, levels, n, out, st, grid, s);
#endif
    else if (W >= 64)
        binary<2>(ctx, off, bins, levels, n, out, st, grid, s);
    else
        binary<1>(ctx, off, bins, levels, n, out, st, grid, s);
}
