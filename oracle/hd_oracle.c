/*
 * hd_oracle.c -- CPU oracle of the HyperOMS hot path.  TEST INFRASTRUCTURE.
 *
 * A plain, slow restatement of what the method computes, written from
 * "Massively Parallel Open Modification Spectral Library Searching with
 * Hyperdimensional Computing" (Kang, Xu, Bittremieux, Rosing).  Only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg load this
 * file.  It shares no source, header, table or helper with the GPU library,
 * and the GPU library never links it.
 *
 * Conventions (readings of the paper where it is silent):
 *  - A hypervector (HV) of D components is stored as D/64 little-endian
 *    uint64 words; bit d lives in word d/64 at position d%64.  Bit value b
 *    stands for the bipolar component 1-2b (0 -> +1, 1 -> -1), so the
 *    element-wise product of two bipolar vectors is the XOR of their bits.
 *  - Floating point is IEEE double, compiled with -ffp-contract=off.
 *
 * Every function returns 0 on success and a negative value on bad input.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  The paper draws its position and level HVs "at
 * random" without naming a generator (Section 3.3.1-3.3.2); this counter-based
 * generator is the reading used on both sides.
 * ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 32-bit word number `i` of Philox word stream `stream` under `seed`:
 * component i%4 of the block at counter (i/4, stream, 0, 0). */
static uint32_t stream_word(uint64_t seed, uint32_t stream, uint32_t i)
{
    uint32_t ctr[4] = { i >> 2, stream, 0u, 0u };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[i & 3u];
}

/* Words 0..n-1 of one stream, word by word from the definition above. */
void orc_random_words(uint64_t seed, uint32_t stream, uint32_t n, uint32_t *out)
{
    for (uint32_t i = 0; i < n; ++i) out[i] = stream_word(seed, stream, i);
}

static int get_bit(const uint64_t *hv, uint32_t d) { return (int)((hv[d >> 6] >> (d & 63u)) & 1u); }
static void set_bit(uint64_t *hv, uint32_t d, int b)
{
    uint64_t m = (uint64_t)1 << (d & 63u);
    if (b) hv[d >> 6] |= m; else hv[d >> 6] &= ~m;
}

/* ---------------------------------------------------------------------------
 * Item memory: position HVs F_0..F_{f-1} (Section 3.3.1) and level HVs
 * L_0..L_{Q-1} (Section 3.3.2).
 *
 * Section 3.3.1: a random base HV, then alpha components flipped at random
 * positions so that similarity falls with the distance between bins while far
 * bins end up near-orthogonal.  Reading: the flips are nested -- F_i differs
 * from F_0 in the m_i = floor(i*alpha/(f-1)) positions of lowest rank under
 * one random permutation of [0, D) -- so the total number of flips from the
 * first to the last bin is alpha.
 * Section 3.3.2: L_p flips (D/2)*(p/100) components of L_0 for level p in
 * percent.  Reading: Q levels 0..Q-1, level j at p = 100*j/(Q-1), nested
 * flips n_j = floor(j*(D/2)/(Q-1)).
 * The random bits come from Philox word streams of `seed`: stream 0 = bits of
 * F_0, 1 = permutation keys for F, 2 = bits of L_0, 3 = permutation keys for
 * L.  The permutation rank of position d is its place in the ascending order
 * of (key_d, d).
 * ------------------------------------------------------------------------- */
typedef struct { uint32_t key; uint32_t pos; } keypos;

static int cmp_keypos(const void *a, const void *b)
{
    const keypos *x = (const keypos *)a, *y = (const keypos *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->pos < y->pos ? -1 : (x->pos > y->pos);
}

static int make_rank(uint32_t D, uint64_t seed, uint32_t stream, uint32_t *rank)
{
    keypos *kp = (keypos *)malloc(sizeof(keypos) * D);
    if (!kp) return -2;
    for (uint32_t d = 0; d < D; ++d) { kp[d].key = stream_word(seed, stream, d); kp[d].pos = d; }
    qsort(kp, D, sizeof(keypos), cmp_keypos);
    for (uint32_t r = 0; r < D; ++r) rank[kp[r].pos] = r;
    free(kp);
    return 0;
}

static void make_base(uint32_t D, uint64_t seed, uint32_t stream, uint64_t *hv)
{
    for (uint32_t d = 0; d < D; ++d)
        set_bit(hv, d, (int)((stream_word(seed, stream, d >> 5) >> (d & 31u)) & 1u));
}

/* Encoder variants compared in Section 4.2 ("Encoding strategy"):
 *  mode 0 -- the nested flips above;
 *  mode 1 -- reading B of Section 3.3.1, a random walk: F_i is F_{i-1} with
 *           exactly `alpha` components flipped (alpha <= 256) at distinct
 *           positions drawn by Floyd's sampling algorithm: for k = 0..alpha-1,
 *           j = D - alpha + k, t = word(stream 4, i * 256 + k) mod (j + 1);
 *           take t unless already taken, else take j;
 *  mode 2 -- ID-Level HDC: independent random F_i, bit d of F_i = bit d%32 of
 *           word(stream 5, i * D/32 + d/32).
 * The level HVs are the same in every mode. */
static int in_set(const uint32_t *s, uint32_t n, uint32_t v)
{
    for (uint32_t i = 0; i < n; ++i) if (s[i] == v) return 1;
    return 0;
}

int orc_item_memory(uint32_t D, uint32_t Q, uint32_t f, uint32_t alpha, uint64_t seed, uint32_t mode,
                    uint64_t *F, uint64_t *L, uint32_t *rank_F, uint32_t *rank_L)
{
    if (D == 0 || D % 64u || Q < 2 || f == 0 || alpha > D || mode > 2) return -1;
    if (mode == 1 && (alpha > 256u || f > (1u << 24))) return -1;           /* counters i * 256 + k */
    if (mode == 2 && (uint64_t)f * (D / 32u) > 0xFFFFFFFFull) return -1;  /* counters i * D/32 + w */
    const uint32_t W = D / 64u;
    uint64_t *F0 = (uint64_t *)calloc(W, 8), *L0 = (uint64_t *)calloc(W, 8);
    if (!F0 || !L0) { free(F0); free(L0); return -2; }
    make_base(D, seed, 0, F0);
    make_base(D, seed, 2, L0);
    if (make_rank(D, seed, 1, rank_F) || make_rank(D, seed, 3, rank_L)) { free(F0); free(L0); return -2; }
    if (mode == 0) {
        for (uint32_t i = 0; i < f; ++i) {
            uint64_t m = (f > 1) ? ((uint64_t)i * alpha) / (uint64_t)(f - 1) : 0;
            uint64_t *Fi = F + (size_t)i * W;
            for (uint32_t d = 0; d < D; ++d)
                set_bit(Fi, d, get_bit(F0, d) ^ (rank_F[d] < m));
        }
    } else if (mode == 1) {
        uint32_t chosen[256];
        memcpy(F, F0, (size_t)W * 8);
        for (uint32_t i = 1; i < f; ++i) {
            uint64_t *Fi = F + (size_t)i * W;
            memcpy(Fi, Fi - W, (size_t)W * 8);
            for (uint32_t k = 0; k < alpha; ++k) {
                uint32_t j = D - alpha + k;
                uint32_t t = stream_word(seed, 4, i * 256u + k) % (j + 1u);
                chosen[k] = in_set(chosen, k, t) ? j : t;
                set_bit(Fi, chosen[k], !get_bit(Fi, chosen[k]));
            }
        }
    } else {
        for (uint32_t i = 0; i < f; ++i) {
            uint64_t *Fi = F + (size_t)i * W;
            for (uint32_t d = 0; d < D; ++d)
                set_bit(Fi, d, (int)((stream_word(seed, 5, i * (D / 32u) + d / 32u) >> (d & 31u)) & 1u));
        }
    }
    for (uint32_t j = 0; j < Q; ++j) {
        uint64_t n = ((uint64_t)j * (D / 2u)) / (uint64_t)(Q - 1);
        uint64_t *Lj = L + (size_t)j * W;
        for (uint32_t d = 0; d < D; ++d)
            set_bit(Lj, d, get_bit(L0, d) ^ (rank_L[d] < n));
    }
    free(F0); free(L0);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Preprocessing (Section 3.2, Table 1): raw peaks -> CSR spectrum vector of
 * (bin, quantised level).  Steps, in order:
 *   0. drop peaks whose m/z or intensity is not finite, or whose intensity
 *      is <= 0 (reading: such peaks carry no signal);
 *   1. drop peaks with m/z outside [mz_min, mz_max];
 *   2. drop peaks whose intensity is below min_rel * (most intense peak);
 *   3. keep the max_peaks most intense (ties: lower m/z, then lower input
 *      position);
 *   4. bin = floor((mz - mz_min) / bin_width), clamped to [0, n_bins-1];
 *   5. peaks that share a bin have their intensities summed, in ascending
 *      m/z order (ties: input position);
 *   6. level = min(Q-1, floor(Q * v / v_max)) with v_max the largest bin
 *      sum (reading of the garbled "i in [0, Q]": Q levels 0..Q-1).
 * Output rows are in ascending bin order.  out_bin / out_level need room for
 * n_spec * max_peaks entries.  Returns the number of entries written, < 0 on
 * error.
 * ------------------------------------------------------------------------- */
typedef struct { double mz, it; uint32_t pos; } peak;

static int cmp_intensity_desc(const void *a, const void *b)
{
    const peak *x = (const peak *)a, *y = (const peak *)b;
    if (x->it != y->it) return x->it > y->it ? -1 : 1;
    if (x->mz != y->mz) return x->mz < y->mz ? -1 : 1;
    return x->pos < y->pos ? -1 : (x->pos > y->pos);
}

static int cmp_mz_asc(const void *a, const void *b)
{
    const peak *x = (const peak *)a, *y = (const peak *)b;
    if (x->mz != y->mz) return x->mz < y->mz ? -1 : 1;
    return x->pos < y->pos ? -1 : (x->pos > y->pos);
}

long long orc_preprocess(uint32_t n_spec, const uint32_t *raw_off, const double *raw_mz,
                         const double *raw_int, double mz_min, double mz_max, double bin_width,
                         uint32_t n_bins, uint32_t max_peaks, double min_rel, uint32_t n_levels,
                         uint32_t *out_off, uint32_t *out_bin, uint8_t *out_level)
{
    if (n_bins == 0 || max_peaks == 0 || n_levels < 2 || n_levels > 256 || !(bin_width > 0.0))
        return -1;
    uint32_t longest = 0;
    for (uint32_t s = 0; s < n_spec; ++s) {
        if (raw_off[s + 1] < raw_off[s]) return -1;
        if (raw_off[s + 1] - raw_off[s] > longest) longest = raw_off[s + 1] - raw_off[s];
    }
    peak *pk = (peak *)malloc(sizeof(peak) * (longest ? longest : 1));
    double *sums = (double *)malloc(sizeof(double) * max_peaks);
    uint32_t *bins = (uint32_t *)malloc(sizeof(uint32_t) * max_peaks);
    if (!pk || !sums || !bins) { free(pk); free(sums); free(bins); return -2; }
    uint64_t nnz = 0;
    out_off[0] = 0;
    for (uint32_t s = 0; s < n_spec; ++s) {
        uint32_t n = 0;
        for (uint32_t i = raw_off[s]; i < raw_off[s + 1]; ++i) {
            double mz = raw_mz[i], it = raw_int[i];
            if (!isfinite(mz) || !isfinite(it) || !(it > 0.0)) continue;          /* step 0 */
            if (mz < mz_min || mz > mz_max) continue;                              /* step 1 */
            pk[n].mz = mz; pk[n].it = it; pk[n].pos = i - raw_off[s]; ++n;
        }
        double top = 0.0;
        for (uint32_t i = 0; i < n; ++i) if (pk[i].it > top) top = pk[i].it;
        double floor_it = min_rel * top;
        uint32_t m = 0;
        for (uint32_t i = 0; i < n; ++i) if (!(pk[i].it < floor_it)) pk[m++] = pk[i];  /* step 2 */
        qsort(pk, m, sizeof(peak), cmp_intensity_desc);                            /* step 3 */
        if (m > max_peaks) m = max_peaks;
        qsort(pk, m, sizeof(peak), cmp_mz_asc);
        uint32_t nb = 0;
        for (uint32_t i = 0; i < m; ++i) {                                         /* step 4-5 */
            double x = floor((pk[i].mz - mz_min) / bin_width);
            uint32_t b = (x < 0.0) ? 0u : (x > (double)(n_bins - 1) ? n_bins - 1 : (uint32_t)x);
            if (nb > 0 && bins[nb - 1] == b) sums[nb - 1] += pk[i].it;
            else { bins[nb] = b; sums[nb] = pk[i].it; ++nb; }
        }
        double vmax = 0.0;
        for (uint32_t i = 0; i < nb; ++i) if (sums[i] > vmax) vmax = sums[i];
        for (uint32_t i = 0; i < nb; ++i) {                                        /* step 6 */
            double q = floor((double)n_levels * sums[i] / vmax);
            uint32_t lv = (q >= (double)(n_levels - 1)) ? n_levels - 1 : (uint32_t)q;
            out_bin[nnz] = bins[i];
            out_level[nnz] = (uint8_t)lv;
            ++nnz;
        }
        out_off[s + 1] = (uint32_t)nnz;
    }
    free(pk); free(sums); free(bins);
    return (long long)nnz;
}

/* ---------------------------------------------------------------------------
 * Encoding, Eq. 1 and the binarisation after it (Section 3.3): in bipolar
 * arithmetic I = sum over peaks (i, j) of F_i (.) L_j, then component d of
 * the output is +1 when I_d > 0 and -1 otherwise.
 * encoder 1 -- the random-projection LSH baseline of Section 4.2: the
 * spectrum vector (value level + 1 at each peak's bin) projected on D random
 * +-1 directions, direction d taking component d of F_bin for each bin:
 * I_d = sum over peaks of (level + 1) * F_bin[d], then the same sign rule.
 *
 * Multi-bit components (bits > 1; Section 4.3 names a higher precision per
 * HV component as a way to raise the identification rate, without a
 * quantiser).  Reading: the same sum I is quantised symmetrically to
 * m = 2^(bits-1) - 1 magnitude levels with the spectrum's own step M / m,
 * M = max_d |I_d|:
 *     h_d = sign(I_d) * round(m * |I_d| / M), halves rounded up in magnitude,
 * computed in integers as floor((2 m |I_d| + M) / (2 M)); h = 0 when M = 0.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t D, n_bins, n_levels, s0, s1, encoder, bits;
    const uint64_t *F, *L;
    const uint32_t *off, *bin;
    const uint8_t *level;
    uint64_t *out;      /* bits == 1: [n][D/64] */
    int8_t *out_mb;     /* bits > 1: [n][D] */
    int rc;
} encode_job;

static void *encode_worker(void *arg)
{
    encode_job *j = (encode_job *)arg;
    const uint32_t D = j->D, W = D / 64u;
    int32_t *I = (int32_t *)malloc(sizeof(int32_t) * D);
    if (!I) { j->rc = -2; return NULL; }
    for (uint32_t s = j->s0; s < j->s1; ++s) {
        memset(I, 0, sizeof(int32_t) * D);
        for (uint32_t p = j->off[s]; p < j->off[s + 1]; ++p) {
            if (j->bin[p] >= j->n_bins || j->level[p] >= j->n_levels) { j->rc = -1; free(I); return NULL; }
            const uint64_t *Fi = j->F + (size_t)j->bin[p] * W, *Lj = j->L + (size_t)j->level[p] * W;
            for (uint32_t d = 0; d < D; ++d) {
                int f = 1 - 2 * get_bit(Fi, d), l = 1 - 2 * get_bit(Lj, d);
                I[d] += j->encoder == 1 ? f * ((int)j->level[p] + 1) : f * l;
            }
        }
        if (j->bits == 1) {
            uint64_t *o = j->out + (size_t)s * W;
            for (uint32_t d = 0; d < D; ++d) set_bit(o, d, I[d] > 0 ? 0 : 1);
        } else {
            const int64_t m = ((int64_t)1 << (j->bits - 1)) - 1;
            int64_t M = 0;
            for (uint32_t d = 0; d < D; ++d) {
                int64_t a = I[d] < 0 ? -(int64_t)I[d] : (int64_t)I[d];
                if (a > M) M = a;
            }
            int8_t *o = j->out_mb + (size_t)s * D;
            for (uint32_t d = 0; d < D; ++d) {
                if (M == 0) { o[d] = 0; continue; }
                int64_t a = I[d] < 0 ? -(int64_t)I[d] : (int64_t)I[d];
                int64_t h = (2 * m * a + M) / (2 * M);
                o[d] = (int8_t)(I[d] < 0 ? -h : h);
            }
        }
    }
    free(I);
    return NULL;
}

/* Spectra are split into `n_threads` contiguous ranges, one per thread.
 * bits == 1 writes binary HVs to `out`, bits in 2..8 multi-bit components to
 * `out_mb`. */
static int encode_any(uint32_t D, const uint64_t *F, uint32_t n_bins, const uint64_t *L, uint32_t n_levels,
                      uint32_t n_spec, const uint32_t *off, const uint32_t *bin, const uint8_t *level,
                      uint64_t *out, int8_t *out_mb, uint32_t bits, uint32_t n_threads, uint32_t encoder)
{
    if (D == 0 || D % 64u || encoder > 1 || bits == 0 || bits > 8) return -1;
    for (uint32_t s = 0; s < n_spec; ++s) if (off[s + 1] < off[s]) return -1;
    if (n_threads == 0) n_threads = 1;
    if (n_threads > n_spec) n_threads = n_spec ? n_spec : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
    encode_job *jobs = (encode_job *)malloc(sizeof(encode_job) * n_threads);
    char *started = (char *)calloc(n_threads, 1);
    if (!th || !jobs || !started) { free(th); free(jobs); free(started); return -2; }
    for (uint32_t t = 0; t < n_threads; ++t) {
        encode_job j = { D, n_bins, n_levels, (uint32_t)((uint64_t)n_spec * t / n_threads),
                         (uint32_t)((uint64_t)n_spec * (t + 1) / n_threads), encoder, bits, F, L, off, bin, level,
                         out, out_mb, 0 };
        jobs[t] = j;
    }
    for (uint32_t t = 1; t < n_threads; ++t) started[t] = pthread_create(&th[t], NULL, encode_worker, &jobs[t]) == 0;
    for (uint32_t t = 1; t < n_threads; ++t) if (!started[t]) encode_worker(&jobs[t]);
    encode_worker(&jobs[0]);
    int rc = 0;
    for (uint32_t t = 0; t < n_threads; ++t) {
        if (t > 0 && started[t]) pthread_join(th[t], NULL);
        if (jobs[t].rc) rc = jobs[t].rc;
    }
    free(th); free(jobs); free(started);
    return rc;
}

int orc_encode(uint32_t D, const uint64_t *F, uint32_t n_bins, const uint64_t *L, uint32_t n_levels,
               uint32_t n_spec, const uint32_t *off, const uint32_t *bin, const uint8_t *level,
               uint64_t *out, uint32_t n_threads, uint32_t encoder)
{
    return encode_any(D, F, n_bins, L, n_levels, n_spec, off, bin, level, out, NULL, 1, n_threads, encoder);
}

int orc_encode_multibit(uint32_t D, const uint64_t *F, uint32_t n_bins, const uint64_t *L, uint32_t n_levels,
                        uint32_t n_spec, const uint32_t *off, const uint32_t *bin, const uint8_t *level,
                        uint32_t bits, int8_t *out, uint32_t n_threads, uint32_t encoder)
{
    if (bits < 2) return -1;
    return encode_any(D, F, n_bins, L, n_levels, n_spec, off, bin, level, NULL, out, bits, n_threads, encoder);
}

/* ---------------------------------------------------------------------------
 * Candidate predicate (Section 3.4, Table 1): same charge, and the precursor
 * difference within the tolerance, bound inclusive.  unit 0 ("Da") and 1
 * (ppm) compare precursor m/z:
 *     fabs(mz_r - mz_q) <= tol_q,
 * tol_q = tol for a tolerance in m/z units, mz_q * (tol * 1e-6) for ppm
 * (reading: "500 Da" is a literal precursor m/z difference).  unit 2 compares
 * neutral precursor masses M = (mz - 1.007276) * z, the m/z less one proton
 * mass per charge:
 *     fabs(M_r - M_q) <= tol.
 * ------------------------------------------------------------------------- */
#define ORC_PROTON_MASS 1.007276

static double neutral_mass(double mz, uint8_t z) { return (mz - ORC_PROTON_MASS) * (double)z; }

static int is_candidate(double mz_r, uint8_t z_r, double mz_q, uint8_t z_q, double tol, int unit)
{
    if (z_r != z_q) return 0;
    if (unit == 2) return fabs(neutral_mass(mz_r, z_r) - neutral_mass(mz_q, z_q)) <= tol;
    double tol_q = unit == 1 ? mz_q * (tol * 1e-6) : tol;
    return fabs(mz_r - mz_q) <= tol_q;
}

int orc_window_count(uint32_t n_ref, const double *ref_mz, const uint8_t *ref_z, uint32_t n_q,
                     const double *q_mz, const uint8_t *q_z, double tol, int unit, uint32_t *count)
{
    for (uint32_t q = 0; q < n_q; ++q) {
        uint32_t c = 0;
        for (uint32_t r = 0; r < n_ref; ++r) c += (uint32_t)is_candidate(ref_mz[r], ref_z[r], q_mz[q], q_z[q], tol, unit);
        count[q] = c;
    }
    return 0;
}

/* Library order (Section 3.4 filters by charge and precursor m/z): the row
 * order of references sorted by (charge, precursor m/z, input index). */
static const double *g_sort_mz;
static const uint8_t *g_sort_z;
static int cmp_lib(const void *a, const void *b)
{
    uint32_t i = *(const uint32_t *)a, j = *(const uint32_t *)b;
    if (g_sort_z[i] != g_sort_z[j]) return g_sort_z[i] < g_sort_z[j] ? -1 : 1;
    if (g_sort_mz[i] < g_sort_mz[j]) return -1;
    if (g_sort_mz[i] > g_sort_mz[j]) return 1;
    return i < j ? -1 : (i > j);
}

int orc_library_order(uint32_t n, const double *mz, const uint8_t *z, uint32_t *order)
{
    for (uint32_t i = 0; i < n; ++i) order[i] = i;
    g_sort_mz = mz; g_sort_z = z;
    qsort(order, n, sizeof(uint32_t), cmp_lib);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Hamming search (Section 3.4).  Hamming similarity counts equal components;
 * the best match has the fewest differing components,
 *     dist(x, y) = popcount(x XOR y) over the D bits.
 * For each query, every reference is tested with the candidate predicate and
 * the k smallest keys (dist, reference index) are kept, ascending; the lowest
 * reference index wins a tie.  With fewer than k candidates the remaining
 * slots hold idx 0xFFFFFFFF and dist 0xFFFF.
 * `which` lists the query indices to answer (NULL = all); results go to row
 * t of out_* for which[t].  Queries are spread over `n_threads` threads.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t D, n_ref, n_q, k, n_which, tid, n_threads;
    const uint64_t *ref_hv, *q_hv;
    const double *ref_mz, *q_mz;
    const uint8_t *ref_z, *q_z;
    const uint32_t *which;
    double tol; int unit;
    uint32_t *out_idx; uint16_t *out_dist;
} search_job;

static void *search_worker(void *arg)
{
    search_job *j = (search_job *)arg;
    const uint32_t W = j->D / 64u;
    uint64_t *best = (uint64_t *)malloc(sizeof(uint64_t) * j->k);
    for (uint32_t t = j->tid; t < j->n_which; t += j->n_threads) {
        uint32_t q = j->which ? j->which[t] : t;
        for (uint32_t s = 0; s < j->k; ++s) best[s] = UINT64_MAX;
        const uint64_t *qh = j->q_hv + (size_t)q * W;
        for (uint32_t r = 0; r < j->n_ref; ++r) {
            if (!is_candidate(j->ref_mz[r], j->ref_z[r], j->q_mz[q], j->q_z[q], j->tol, j->unit)) continue;
            const uint64_t *rh = j->ref_hv + (size_t)r * W;
            uint64_t dist = 0;
            for (uint32_t w = 0; w < W; ++w) dist += (uint64_t)__builtin_popcountll(qh[w] ^ rh[w]);
            uint64_t key = (dist << 32) | r;
            if (key >= best[j->k - 1]) continue;
            uint32_t s = j->k - 1;
            while (s > 0 && best[s - 1] > key) { best[s] = best[s - 1]; --s; }
            best[s] = key;
        }
        for (uint32_t s = 0; s < j->k; ++s) {
            if (best[s] == UINT64_MAX) { j->out_idx[(size_t)t * j->k + s] = 0xFFFFFFFFu; j->out_dist[(size_t)t * j->k + s] = 0xFFFFu; }
            else { j->out_idx[(size_t)t * j->k + s] = (uint32_t)best[s]; j->out_dist[(size_t)t * j->k + s] = (uint16_t)(best[s] >> 32); }
        }
    }
    free(best);
    return NULL;
}

int orc_search(uint32_t D, uint32_t n_ref, const uint64_t *ref_hv, const double *ref_mz, const uint8_t *ref_z,
               uint32_t n_q, const uint64_t *q_hv, const double *q_mz, const uint8_t *q_z,
               double tol, int unit, uint32_t k, const uint32_t *which, uint32_t n_which,
               uint32_t *out_idx, uint16_t *out_dist, uint32_t n_threads)
{
    if (D == 0 || D % 64u || D > 65534u || k == 0 || !(tol >= 0.0)) return -1;
    if (!which) n_which = n_q;
    if (n_threads == 0) n_threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
    search_job *jobs = (search_job *)malloc(sizeof(search_job) * n_threads);
    if (!th || !jobs) { free(th); free(jobs); return -2; }
    for (uint32_t t = 0; t < n_threads; ++t) {
        search_job j = { D, n_ref, n_q, k, n_which, t, n_threads, ref_hv, q_hv, ref_mz, q_mz, ref_z, q_z,
                         which, tol, unit, out_idx, out_dist };
        jobs[t] = j;
    }
    uint32_t started = 0;
    for (uint32_t t = 1; t < n_threads; ++t)
        if (pthread_create(&th[t], NULL, search_worker, &jobs[t]) == 0) ++started; else break;
    /* threads that failed to start leave their queries to this thread */
    if (started + 1 < n_threads)
        for (uint32_t t = started + 1; t < n_threads; ++t) search_worker(&jobs[t]);
    search_worker(&jobs[0]);
    for (uint32_t t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    free(th); free(jobs);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Search over multi-bit components (the Section 4.3 variant above).  With
 * integer components the Hamming similarity generalises to the dot product
 *     S(x, y) = sum_d x_d * y_d,
 * which for +-1 components equals D - 2 * dist.  For each query every
 * candidate (the same predicate as orc_search) is scored and the k best are
 * kept: higher S first, the lower reference index on a tie.  With fewer than
 * k candidates the remaining slots hold idx 0xFFFFFFFF and score INT32_MIN.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t D, n_ref, k, n_which, tid, n_threads;
    const int8_t *ref, *qv;
    const double *ref_mz, *q_mz;
    const uint8_t *ref_z, *q_z;
    const uint32_t *which;
    double tol; int unit;
    uint32_t *out_idx; int32_t *out_score;
} dot_job;

static void *dot_worker(void *arg)
{
    dot_job *j = (dot_job *)arg;
    int64_t *bs = (int64_t *)malloc(sizeof(int64_t) * j->k);
    uint32_t *bi = (uint32_t *)malloc(sizeof(uint32_t) * j->k);
    for (uint32_t t = j->tid; t < j->n_which; t += j->n_threads) {
        uint32_t q = j->which ? j->which[t] : t, filled = 0;
        const int8_t *qh = j->qv + (size_t)q * j->D;
        for (uint32_t r = 0; r < j->n_ref; ++r) {
            if (!is_candidate(j->ref_mz[r], j->ref_z[r], j->q_mz[q], j->q_z[q], j->tol, j->unit)) continue;
            const int8_t *rh = j->ref + (size_t)r * j->D;
            int64_t S = 0;
            for (uint32_t d = 0; d < j->D; ++d) S += (int64_t)qh[d] * (int64_t)rh[d];
            /* position of (S, r) among the kept entries, best first */
            uint32_t pos = filled;
            while (pos > 0 && (bs[pos - 1] < S || (bs[pos - 1] == S && bi[pos - 1] > r))) --pos;
            if (pos >= j->k) continue;
            uint32_t last = filled < j->k ? filled : j->k - 1;
            for (uint32_t u = last; u > pos; --u) { bs[u] = bs[u - 1]; bi[u] = bi[u - 1]; }
            bs[pos] = S; bi[pos] = r;
            if (filled < j->k) ++filled;
        }
        for (uint32_t s = 0; s < j->k; ++s) {
            j->out_idx[(size_t)t * j->k + s] = s < filled ? bi[s] : 0xFFFFFFFFu;
            j->out_score[(size_t)t * j->k + s] = s < filled ? (int32_t)bs[s] : INT32_MIN;
        }
    }
    free(bs); free(bi);
    return NULL;
}

int orc_search_dot(uint32_t D, uint32_t n_ref, const int8_t *ref, const double *ref_mz, const uint8_t *ref_z,
                   uint32_t n_q, const int8_t *qv, const double *q_mz, const uint8_t *q_z,
                   double tol, int unit, uint32_t k, const uint32_t *which, uint32_t n_which,
                   uint32_t *out_idx, int32_t *out_score, uint32_t n_threads)
{
    if (D == 0 || k == 0 || !(tol >= 0.0)) return -1;
    if (!which) n_which = n_q;
    if (n_threads == 0) n_threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
    dot_job *jobs = (dot_job *)malloc(sizeof(dot_job) * n_threads);
    if (!th || !jobs) { free(th); free(jobs); return -2; }
    for (uint32_t t = 0; t < n_threads; ++t) {
        dot_job j = { D, n_ref, k, n_which, t, n_threads, ref, qv, ref_mz, q_mz, ref_z, q_z, which, tol, unit,
                      out_idx, out_score };
        jobs[t] = j;
    }
    uint32_t started = 0;
    for (uint32_t t = 1; t < n_threads; ++t)
        if (pthread_create(&th[t], NULL, dot_worker, &jobs[t]) == 0) ++started; else break;
    if (started + 1 < n_threads)
        for (uint32_t t = started + 1; t < n_threads; ++t) dot_worker(&jobs[t]);
    dot_worker(&jobs[0]);
    for (uint32_t t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    free(th); free(jobs);
    return 0;
}
