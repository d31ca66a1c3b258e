/*
 * hd.h -- C ABI of the GB300 HyperOMS hot path: hyperdimensional encoding of
 * preprocessed MS/MS spectra and the open-modification Hamming search.
 *
 * Method: Kang, Xu, Bittremieux, Rosing, "Massively Parallel Open
 * Modification Spectral Library Searching with Hyperdimensional Computing".
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Hypervector (HV): D bits stored as D/64 little-endian uint64 words, bit d
 *    in word d/64 at position d%64.  Bit b is the bipolar component 1-2b
 *    (0 -> +1, 1 -> -1); the element-wise product of bipolar HVs is the XOR
 *    of their bits.  Rows of an HV array are contiguous (stride D/8 bytes);
 *    D is a multiple of 128, so every row starts on a 16-byte boundary when
 *    the array does.
 *  - Pointers named d_* are DEVICE pointers on the current CUDA device; h_*
 *    are host pointers (page-locked memory gives asynchronous copies).  The
 *    caller owns every buffer it passes; the library owns hd_ctx and
 *    hd_library objects and the scratch it allocates (stream-ordered, freed
 *    on the same stream).
 *  - Scratch is allocated stream-ordered (cudaMallocAsync) from the device's
 *    default memory pool; hd_ctx_create raises that pool's release threshold
 *    to 4 GiB (never lowers it) so scratch stays mapped across the calls
 *    that synchronise.
 *  - Calls taking a stream are asynchronous on it unless stated otherwise;
 *    results are valid once the stream has been synchronised.  A NULL stream
 *    is the legacy default stream.
 *  - Argument errors are detected on the host before anything is launched
 *    and return HD_ERR_INVALID_ARG.  Errors found by a kernel (a malformed
 *    CSR row, a bounded device wait that expired) are recorded in the
 *    status word of the hd_ctx or hd_library used; hd_ctx_status() /
 *    hd_library_status() return and clear it after the caller synchronised.
 *  - hd_last_error_message() gives a text for the last failure on the
 *    calling thread.
 *  - Thread safety: distinct objects are independent.  One hd_ctx or
 *    hd_library may serve concurrent read-only calls (hd_encode,
 *    hd_search_open, hd_search_open_ex, hd_search_open_multi, hd_search_dot,
 *    hd_search_dot_multi)
 *    from several host threads and streams.  hd_search_open_noalloc is the
 *    exception: all its calls share one scratch buffer, so its calls that
 *    overlap on the GPU race and must be serialised by the caller.
 */
#ifndef HD_H
#define HD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define HD_API __attribute__((visibility("default")))
#else
#define HD_API
#endif

struct CUstream_st;                       /* == cudaStream_t */
typedef struct CUstream_st *hd_stream;

typedef enum {
    HD_OK = 0,
    HD_ERR_INVALID_ARG = 1,   /* bad argument, or malformed input found on the device */
    HD_ERR_OOM = 2,           /* device allocation failed; nothing launched */
    HD_ERR_CUDA = 3,          /* a CUDA runtime call failed (message has details) */
    HD_ERR_TIMEOUT = 4,       /* a bounded device wait expired; results are invalid */
    HD_ERR_UNSUPPORTED = 5    /* valid request that this library or GPU does not serve */
} hd_status;

/* Precursor tolerance units.  HD_TOL_DA and HD_TOL_PPM bound the precursor
 * m/z difference (Section 3.4, Table 1); HD_TOL_MASS bounds the neutral
 * precursor mass difference, mass = (mz - 1.007276) * charge, in Da. */
typedef enum { HD_TOL_DA = 0, HD_TOL_PPM = 1, HD_TOL_MASS = 2 } hd_tol_unit;

/* Position-HV generation (Section 3.3.1; variants compared in Section 4.2).
 *  HD_POS_NESTED  F_i = F_0 with the floor(i * alpha / (f - 1)) lowest-ranked
 *                 components of one random permutation flipped (alpha in
 *                 total from the first to the last bin) -- the default
 *  HD_POS_WALK    F_i = F_{i-1} with exactly alpha (<= 256) components flipped
 *                 at distinct random positions (Floyd's sampling on Philox
 *                 stream 4, counter i * 256 + k)
 *  HD_POS_RANDOM  independent random F_i (ID-Level HDC; Philox stream 5) */
typedef enum { HD_POS_NESTED = 0, HD_POS_WALK = 1, HD_POS_RANDOM = 2 } hd_position_mode;
/* Spectrum encoder (Section 3.3, Eq. 1; baseline of Section 4.2).
 *  HD_ENC_ID_LEVEL    sign of sum over peaks of F_bin (.) L_level (Eq. 1)
 *  HD_ENC_PROJECTION  random-projection LSH: sign of sum over peaks of
 *                     (level + 1) * F_bin, F_bin as +-1 directions
 * Both map a sum <= 0 to -1 (bit 1). */
typedef enum { HD_ENC_ID_LEVEL = 0, HD_ENC_PROJECTION = 1 } hd_encoder_kind;

/* Item-memory parameters (Section 3.3).
 *  dim      D, multiple of 128, 128..32768 (paper: 8192, Section 4.2)
 *  n_levels Q intensity levels 0..Q-1, 2..256 (paper: 16)
 *  n_bins   f spectrum-vector dimensionality (m/z bins), >= 1
 *  alpha    HD_POS_NESTED: total position flips from the first to the last
 *           bin, <= D (paper: D/2, Section 4.2); HD_POS_WALK: flips per
 *           step, <= 256; HD_POS_RANDOM: unused
 *  seed     Philox4x32-10 key of the random base vectors and permutations
 *  position_mode  an hd_position_mode (0: the paper's, as read here)
 *  encoder        an hd_encoder_kind (0: Eq. 1) */
typedef struct {
    uint32_t dim;
    uint32_t n_levels;
    uint32_t n_bins;
    uint32_t alpha;
    uint64_t seed;
    uint32_t position_mode;
    uint32_t encoder;
} hd_params;

/* Preprocessing parameters (Section 3.2, Table 1). */
typedef struct {
    double mz_min, mz_max;     /* fragment m/z range kept, inclusive (Table 1: 101 / 1500) */
    double bin_width;          /* > 0 (Table 1: 0.05 or 0.04) */
    double min_rel_intensity;  /* peaks below this fraction of the top peak are dropped (0.01) */
    uint32_t n_bins;           /* bins 0..n_bins-1; m/z beyond are clamped */
    uint32_t max_peaks;        /* most intense peaks kept, 1..1023 (Table 1: 50) */
    uint32_t n_levels;         /* Q, 2..256 */
} hd_preprocess_params;

typedef struct hd_ctx hd_ctx;
typedef struct hd_library hd_library;

/* Scoring forms; all give identical results.  The tensor-core forms score
 * bipolar copies (bit 0 -> +1, bit 1 -> -1) of the HVs by matrix multiply,
 * S = sum_d x_d y_d = D - 2*dist, accumulated exactly in fp32.  HD_FORM_AUTO
 * takes the autotuner's choice, else the fastest prepared tensor-core form
 * (kind::mxf4 when the e2m1 copy exists and D is a multiple of 256), else
 * popc. */
typedef enum {
    HD_FORM_AUTO = 0,     /* fastest form the library was prepared for */
    HD_FORM_POPC = 1,     /* XOR + population count on the integer pipes */
    HD_FORM_TC_FP8 = 2,   /* tcgen05 kind::f8f6f4, +-1 as e4m3 (library: D bytes/row) */
    HD_FORM_TC_BF16 = 3,  /* tcgen05 kind::f16, +-1 as bf16 (library: 2D bytes/row) */
    HD_FORM_TC_FP4 = 4,   /* tcgen05 kind::f8f6f4, +-1 as e2m1 packed two per byte
                             (library: D/2 bytes/row; the TMA unpacks into shared memory) */
    HD_FORM_TC_MXF4 = 5   /* tcgen05 kind::mxf4 (block-scaled, unit ue8m0 scales) on the same
                             packed e2m1 rows, kept packed in shared memory; SM pairs, N = 240
                             per MMA; D a multiple of 256 (else HD_ERR_UNSUPPORTED) */
} hd_search_form;

/* Name of a status code ("HD_OK", ...); a static string, never NULL. */
HD_API const char *hd_status_string(hd_status s);
/* Message of the last failing call on the calling host thread (thread-local,
 * valid until that thread's next failing call). */
HD_API const char *hd_last_error_message(void);
/* Library version as major*10000 + minor*100 + patch. */
HD_API uint32_t hd_version(void);

/* Item memory (Section 3.3.1 position HVs, Section 3.3.2 level HVs).
 * Builds F_0..F_{f-1} and L_0..L_{Q-1} on the current device.  Position HVs
 * share one random base F_0; F_i differs from it in the m_i lowest-ranked
 * positions of one random permutation, m_i = floor(i*alpha/(f-1)), so the
 * distance between bins grows linearly and the last bin is alpha flips away.
 * Level HVs do the same from L_0 with n_j = floor(j*(D/2)/(Q-1)) (level j is
 * j/(Q-1) of the way, Section 3.3.2), so L_{Q-1} is orthogonal to L_0.
 * Random words: Philox4x32-10 of `seed`, counter (i/4, stream, 0, 0), word
 * i%4; stream 0 = F_0 bits, 1 = F permutation keys, 2 = L_0 bits, 3 = L
 * permutation keys; a position's rank is its place in ascending (key, pos).
 * Synchronous.  Allocates f*D/8 + Q*D/8 bytes of device memory. */
HD_API hd_status hd_ctx_create(const hd_params *params, hd_ctx **out);
HD_API void hd_ctx_destroy(hd_ctx *ctx);
/* Copies the item memory out: d_F [n_bins][D/64], d_L [n_levels][D/64],
 * d_rank_F / d_rank_L [D] (each may be NULL).  Asynchronous on `stream`. */
HD_API hd_status hd_ctx_item_memory(const hd_ctx *ctx, uint64_t *d_F, uint64_t *d_L,
                             uint32_t *d_rank_F, uint32_t *d_rank_L, hd_stream stream);
/* Returns and clears the device status recorded by kernels of this ctx. */
HD_API hd_status hd_ctx_status(hd_ctx *ctx);
/* The random words behind the item memory (Section 3.3.1-3.3.2 draw the base
 * HVs and flip positions at random; the generator is Philox4x32-10, Salmon et
 * al., SC'11): d_out[i] = component i%4 of Philox4x32-10 applied to the
 * counter (i/4, stream_id, 0, 0) under the key (seed low 32 bits, seed high
 * 32 bits), for i < n.  Stream 0 holds the F_0 bits, 1 the position-
 * permutation keys, 2 the L_0 bits, 3 the level-permutation keys, 4 the
 * walk's flip draws, 5 the independent position HVs.  d_out [n] uint32
 * device buffer owned by the caller; n <= 2^32 - 4.  Asynchronous. */
HD_API hd_status hd_random_words(uint64_t seed, uint32_t stream_id, uint32_t n, uint32_t *d_out,
                                 hd_stream stream);

/* Preprocessing (Section 3.2, Table 1): raw peaks -> CSR spectrum vectors.
 * Per spectrum: drop peaks with non-finite values or intensity <= 0; drop
 * m/z outside [mz_min, mz_max]; drop intensity < min_rel * top intensity;
 * keep the max_peaks most intense (ties: lower m/z, then input position);
 * bin = clamp(floor((mz - mz_min)/bin_width), 0, n_bins-1); sum intensities
 * sharing a bin in ascending m/z order; level = min(Q-1, floor(Q*v/v_max)).
 * All arithmetic in IEEE double.  Rows come out in ascending bin order.
 *  d_raw_off  [n+1] uint32 offsets into d_raw_mz / d_raw_int (non-decreasing)
 *  d_out_off  [n+1]; d_out_bins / d_out_levels need n*max_peaks entries.
 * A spectrum with more than 8192 raw peaks is emptied and flagged
 * (HD_ERR_INVALID_ARG from hd_ctx_status).  Asynchronous. */
HD_API hd_status hd_preprocess(hd_ctx *ctx, const hd_preprocess_params *pp, const uint32_t *d_raw_off,
                        const double *d_raw_mz, const double *d_raw_int, uint32_t n_spectra,
                        uint32_t *d_out_off, uint32_t *d_out_bins, uint8_t *d_out_levels,
                        hd_stream stream);

/* Encoding (Section 3.3, Eq. 1): for each CSR row with n peaks (bin i,
 * level j), out = sign(sum F_i (.) L_j), positive -> +1 (bit 0), zero or
 * negative -> -1 (bit 1).  Equivalently with c_d the number of bound bits
 * equal to 1 at d: out_d = [2*c_d >= n]; an empty row gives all ones.
 *  d_offsets [n+1] non-decreasing; rows hold <= 1023 peaks; d_bins < n_bins,
 *  d_levels < n_levels (violations flag HD_ERR_INVALID_ARG and the bad peak
 *  or row is skipped).  d_out_hv [n][D/64], 16-byte aligned.  Asynchronous. */
HD_API hd_status hd_encode(hd_ctx *ctx, const uint32_t *d_offsets, const uint32_t *d_bins,
                    const uint8_t *d_levels, uint32_t n_spectra, uint64_t *d_out_hv,
                    hd_stream stream);

/* Reference library (Section 3.3 reuse of reference HVs; Section 3.4
 * candidate filter by charge and precursor m/z).  Copies the n_refs HVs,
 * precursor m/z and charges into library-owned memory sorted by (charge,
 * m/z, input index), so every query window is one contiguous row range.
 * m/z must be finite (else HD_ERR_INVALID_ARG).  Synchronous; the caller
 * may free its buffers afterwards. */
HD_API hd_status hd_build_library(hd_ctx *ctx, const uint64_t *d_hv, const double *d_prec_mz,
                           const uint8_t *d_charge, uint32_t n_refs, hd_library **out);
HD_API void hd_library_free(hd_library *lib);
HD_API hd_status hd_library_info(const hd_library *lib, uint32_t *n_refs, uint32_t *dim);
/* Saves the library to `path` and loads it back (reference HVs are encoded
 * once and reused by later runs, Section 3.3).  File, little-endian: the
 * 8-byte magic "HDLIB001"; u32 dim, n_levels, n_bins, alpha, u64 seed and u32
 * position_mode, encoder of the context that encoded the rows; u32 n, u32
 * flags (bit 0: decoy flags
 * follow; bits 8..15: component bits of a multi-bit library, 0 for binary
 * HVs); then the rows in sorted order, hv [n][D/64] u64 (binary) or
 * components [n][D] int8 (multi-bit), mz [n] f64, charge [n] u8, orig [n]
 * u32, decoy [n] u8 (input order, if flagged); then a u64 FNV-1a hash of
 * every preceding byte.  Tensor-core copies are not stored (load rebuilds a
 * multi-bit library's default copy, as hd_build_library_multibit does;
 * hd_library_prepare adds others).  Load requires a context with the same
 * parameters, checks the hash and the row order (charge, then m/z,
 * ascending, m/z finite), and fails with HD_ERR_INVALID_ARG otherwise.  Both
 * calls are synchronous. */
HD_API hd_status hd_library_save(const hd_library *lib, const hd_ctx *ctx, const char *path);
HD_API hd_status hd_library_load(hd_ctx *ctx, const char *path, hd_library **out);
/* Copies the sorted rows out (any pointer may be NULL): d_hv [n][D/64],
 * d_mz [n], d_charge [n], d_orig [n] (input index of each row). */
HD_API hd_status hd_library_export(const hd_library *lib, uint64_t *d_hv, double *d_mz,
                            uint8_t *d_charge, uint32_t *d_orig, hd_stream stream);
HD_API hd_status hd_library_status(hd_library *lib);
/* Builds the bipolar copy of the library a tensor-core form scores
 * (HD_FORM_TC_FP8: n*D bytes; HD_FORM_TC_BF16: n*2D bytes; HD_FORM_TC_FP4:
 * n*D/2 bytes of device memory, owned by the library).  HD_FORM_POPC needs
 * nothing on binary HVs; on a multi-bit library it builds the bit planes of
 * the popcount dot product (n*bits*D/8 + 4n bytes).  Synchronous;
 * idempotent. */
HD_API hd_status hd_library_prepare(hd_library *lib, hd_search_form form);
/* Schedule of the tensor-core forms (no counterpart in the paper).  Reference
 * rows form tiles of 256 (240 for HD_FORM_TC_MXF4) on a grid fixed to row 0;
 * one work item scores one block of 128 sorted queries (256 on SM pairs)
 * against `tile_group` consecutive tiles, and items are ordered so that the
 * CTAs running at once share `super_group` consecutive groups of tiles
 * through L2.  (cluster, cta_group) = (2, 2)
 * pairs two CTAs on neighbouring SMs into one M = 256 tensor-core operation
 * (each SM stages its own query block and half of every reference tile);
 * (1, 1) runs one CTA per SM at M = 128.  A 0 in either place takes the
 * other's value; 0 everywhere keeps the default (16, 16, 2, 2).  Other
 * combinations fail with HD_ERR_INVALID_ARG.  Every tensor load goes to the
 * issuing CTA's own shared memory (no multicast).  Results do not depend on
 * the schedule.  Not to be changed while a search on this library is in
 * flight. */
HD_API hd_status hd_library_set_schedule(hd_library *lib, uint32_t tile_group, uint32_t super_group,
                                         uint32_t cluster, uint32_t cta_group);
/* Schedule of the kind::mxf4 form (no counterpart in the paper): reference
 * tiles per query stage.  2: each query chunk staged in shared memory is
 * scored against two consecutive reference tiles at once, into both
 * tensor-memory accumulators, so a quarter fewer operand bytes leave L2 per
 * product, but the accumulators drain together and the reference tiles'
 * L2 hit rate falls (faster for large query sets, slower for small ones);
 * 0 or 1: one tile per stage with double-buffered accumulators (the
 * default).  The other forms always stage one tile.  hd_library_autotune
 * tries both.  HD_ERR_INVALID_ARG above 2.  Results do not depend on it.
 * Not to be changed while a search on this library is in flight. */
HD_API hd_status hd_library_set_stage_tiles(hd_library *lib, uint32_t tiles_per_stage);

/* Candidate windows (Section 3.4, Table 1): for each query, rows [lo, hi) of
 * the sorted library whose charge equals the query's and whose precursor
 * m/z satisfies fabs(mz_r - mz_q) <= tol_q in IEEE double, tol_q = tol
 * (HD_TOL_DA, an m/z difference) or mz_q * (tol * 1e-6) (HD_TOL_PPM); with
 * HD_TOL_MASS, fabs(M_r - M_q) <= tol for M = (mz - 1.007276) * charge in
 * IEEE double.  A query with no candidate gets lo == hi.  tol >= 0 and
 * finite. */
HD_API hd_status hd_query_windows(const hd_library *lib, const double *d_q_mz, const uint8_t *d_q_charge,
                           uint32_t n_q, double tol, hd_tol_unit unit, uint32_t *d_lo,
                           uint32_t *d_hi, hd_stream stream);

/* Open-modification search (Section 3.4): for each query, the k candidates
 * with the smallest Hamming distance popcount(q XOR r), ascending, ties to
 * the lowest input reference index.  d_out_idx [n_q][k] input indices of
 * the references, d_out_dist [n_q][k]; fewer than k candidates leave
 * idx 0xFFFFFFFF, dist 0xFFFF in the remaining slots.  1 <= k <= 16.
 * Query rows d_q_hv [n_q][D/64], 16-byte aligned.  Scratch is allocated and
 * freed stream-ordered on `stream`.  Asynchronous. */
HD_API hd_status hd_search_open(const hd_library *lib, const uint64_t *d_q_hv, const double *d_q_mz,
                         const uint8_t *d_q_charge, uint32_t n_q, double tol, hd_tol_unit unit,
                         uint32_t k, uint32_t *d_out_idx, uint16_t *d_out_dist, hd_stream stream);
/* Same, with the scoring form chosen by the caller. */
HD_API hd_status hd_search_open_ex(const hd_library *lib, const uint64_t *d_q_hv, const double *d_q_mz,
                            const uint8_t *d_q_charge, uint32_t n_q, double tol, hd_tol_unit unit,
                            uint32_t k, hd_search_form form, uint32_t *d_out_idx,
                            uint16_t *d_out_dist, hd_stream stream);

/* Candidate window of a class of queries (Section 3.4, Table 1): half-width
 * `tol` in m/z units (HD_TOL_DA) or ppm of the query's precursor m/z. */
typedef struct {
    double tol;
    hd_tol_unit unit;
} hd_window;
#define HD_MAX_WINDOWS 16

/* Open search where each query carries its own window: query q uses
 * windows[d_q_class[q]] (d_q_class NULL: every query uses windows[0]),
 * 1 <= n_windows <= HD_MAX_WINDOWS; classes beyond n_windows-1 use the last.
 * Queries are ordered by (class, charge, m/z) so that a block of queries
 * shares one window width (Table 1's narrow 20 ppm and wide 500 Da searches
 * can run in one call).  Results and padding as hd_search_open.  Async. */
HD_API hd_status hd_search_open_multi(const hd_library *lib, const uint64_t *d_q_hv, const double *d_q_mz,
                                      const uint8_t *d_q_charge, const uint8_t *d_q_class, uint32_t n_q,
                                      const hd_window *windows, uint32_t n_windows, uint32_t k,
                                      hd_search_form form, uint32_t *d_out_idx, uint16_t *d_out_dist,
                                      hd_stream stream);

/* Decoy flags of the library's references (target-decoy strategy, Section
 * 2.1): d_is_decoy [n_refs] in input order, nonzero = decoy.  Copied (the
 * caller keeps its buffer); replaces earlier flags.  Synchronous. */
HD_API hd_status hd_library_set_decoys(hd_library *lib, const uint8_t *d_is_decoy);

/* Cascade search (Section 3.4: a narrow precursor window first, FDR
 * filtering, then a wider window for the spectra still unidentified; FDR by
 * the target-decoy strategy of Section 2.1).  Levels run in order, each with
 * its window levels[l] (1 <= n_levels <= 16).  At a level, the queries not yet
 * identified are searched with k = 1 (as hd_search_open_ex with `form`); the
 * level's spectrum-spectrum matches (SSMs: queries with a candidate) are
 * ranked by score D - dist; the FDR of the threshold at score s is (decoy
 * SSMs with score >= s) / max(1, target SSMs with score >= s), and the
 * q-value of an SSM with score s is the smallest FDR over thresholds <= s,
 * in IEEE double.  An SSM whose reference is a target and whose q-value is
 * <= fdr identifies its query at that level.
 *   d_out_idx [n_q], d_out_dist [n_q]: the SSM of the last level the query
 *     was searched at (the identifying level, else the last level);
 *     idx 0xFFFFFFFF and dist 0xFFFF when that level had no candidate.
 *   d_out_q [n_q]: that SSM's q-value (NaN without a candidate).
 *   d_out_level [n_q]: the identifying level, 0xFF if none.
 * Requires decoy flags (hd_library_set_decoys).  Query rows d_q_hv 16-byte
 * aligned.  Scratch is allocated stream-ordered; the call synchronizes
 * `stream` once per level (the next level's query count is read back). */
HD_API hd_status hd_cascade_search(const hd_library *lib, const uint64_t *d_q_hv, const double *d_q_mz,
                                   const uint8_t *d_q_charge, uint32_t n_q, const hd_window *levels,
                                   uint32_t n_levels, double fdr, hd_search_form form, uint32_t *d_out_idx,
                                   uint16_t *d_out_dist, double *d_out_q, uint8_t *d_out_level,
                                   hd_stream stream);
/* hd_cascade_search for a multi-bit library (Section 4.3 components scored
 * by the dot product): each level searches the unidentified queries' rows
 * d_q_comp [n_q][D] int8 (16-byte aligned) with k = 1 as hd_search_dot with
 * `form` (AUTO, HD_FORM_POPC or a tensor-core form the library holds), and the SSMs are
 * ranked by their score S.  Thresholds, q-values and identification as
 * hd_cascade_search.  d_out_score [n_q] receives S (INT32_MIN without a
 * candidate).  HD_ERR_INVALID_ARG on a binary library (and
 * hd_cascade_search refuses a multi-bit one). */
HD_API hd_status hd_cascade_search_dot(const hd_library *lib, const int8_t *d_q_comp, const double *d_q_mz,
                                       const uint8_t *d_q_charge, uint32_t n_q, const hd_window *levels,
                                       uint32_t n_levels, double fdr, hd_search_form form, uint32_t *d_out_idx,
                                       int32_t *d_out_score, double *d_out_q, uint8_t *d_out_level,
                                       hd_stream stream);

/* Batched plan (no counterpart in the paper, which batches to fill memory,
 * Section 4.1): encoding (Eq. 1) of a fixed set of query batches plus the
 * multi-window search of all of them, captured once into a CUDA graph whose
 * search is a single persistent launch over every batch.  The plan binds the
 * given device buffers: refill their contents and call hd_plan_launch to run
 * again.  d_q_hv_work [n_q][D/64] receives the query HVs.  The library's
 * current form and schedule are frozen into the plan. */
typedef struct hd_plan hd_plan;
HD_API hd_status hd_plan_create(hd_ctx *ctx, const hd_library *lib, const uint32_t *d_offsets,
                                const uint32_t *d_bins, const uint8_t *d_levels, const double *d_q_mz,
                                const uint8_t *d_q_charge, const uint8_t *d_q_class, uint32_t n_q,
                                const hd_window *windows, uint32_t n_windows, uint32_t k, hd_search_form form,
                                uint64_t *d_q_hv_work, uint32_t *d_out_idx, uint16_t *d_out_dist,
                                hd_plan **out);
/* The plan for a multi-bit library (Section 4.3): multi-bit encoding
 * (hd_encode_multibit with the library's bits) into d_q_comp_work [n_q][D]
 * int8 (16-byte aligned) plus hd_search_dot_multi with `form` (AUTO,
 * HD_FORM_POPC or a tensor-core form the library holds); d_out_score [n_q][k] receives the
 * scores.  hd_plan_create refuses a multi-bit library and this call a
 * binary one (HD_ERR_INVALID_ARG). */
HD_API hd_status hd_plan_create_dot(hd_ctx *ctx, const hd_library *lib, const uint32_t *d_offsets,
                                    const uint32_t *d_bins, const uint8_t *d_levels, const double *d_q_mz,
                                    const uint8_t *d_q_charge, const uint8_t *d_q_class, uint32_t n_q,
                                    const hd_window *windows, uint32_t n_windows, uint32_t k, hd_search_form form,
                                    int8_t *d_q_comp_work, uint32_t *d_out_idx, int32_t *d_out_score,
                                    hd_plan **out);
HD_API hd_status hd_plan_launch(hd_plan *plan, hd_stream stream);
/* Kernel nodes in the plan's graph (the launches one hd_plan_launch makes). */
HD_API hd_status hd_plan_info(const hd_plan *plan, uint32_t *kernel_nodes);
HD_API void hd_plan_destroy(hd_plan *plan);

/* Autotuner (no counterpart in the paper): times each search form the library
 * is prepared for (HD_FORM_TC_MXF4 too when the e2m1 copy exists and D is a
 * multiple of 256) and, for the tensor-core forms, work-item shapes
 * tile_group x super_group x (cluster, cta_group) in {4, 8, 16, 32} x {2, 4, 16} x
 * {(1, 1), (2, 2)} ((2, 2) only for kind::mxf4, with one and with two
 * reference tiles per query stage, hd_library_set_stage_tiles), on the
 * given queries (the real query set, or one of the same density per window:
 * a subset's sorted blocks span wider m/z ranges and can favour another
 * schedule), and keeps the fastest as the library's
 * HD_FORM_AUTO form and schedule.  `all` (capacity `cap`) receives every
 * timing.  Synchronous; results never depend on the choice. */
typedef struct {
    hd_search_form form;
    uint32_t tile_group, super_group, cluster, cta_group;
    uint32_t tiles_per_stage;   /* see hd_library_set_stage_tiles; 1 for the other forms, 0 for popc */
    double ms;
} hd_tune_result;
HD_API hd_status hd_library_autotune(hd_library *lib, const uint64_t *d_q_hv, const double *d_q_mz,
                                     const uint8_t *d_q_charge, const uint8_t *d_q_class, uint32_t n_q,
                                     const hd_window *windows, uint32_t n_windows, uint32_t k,
                                     hd_tune_result *best, hd_tune_result *all, uint32_t cap,
                                     uint32_t *n_all);
/* The autotuner for a multi-bit library (Section 4.3): times the
 * dot-product search (hd_search_dot_multi) over the same tensor-core forms
 * and schedules, and the popcount form when hd_library_prepare built the bit
 * planes, on the queries' components d_q_comp [n_q][D] int8 (16-byte
 * aligned) and keeps the fastest as the library's HD_FORM_AUTO, which every
 * dot-product call then takes.  HD_ERR_INVALID_ARG on a binary library or
 * one with neither a tensor-core copy nor bit planes (and
 * hd_library_autotune refuses a multi-bit library). */
HD_API hd_status hd_library_autotune_dot(hd_library *lib, const int8_t *d_q_comp, const double *d_q_mz,
                                         const uint8_t *d_q_charge, const uint8_t *d_q_class, uint32_t n_q,
                                         const hd_window *windows, uint32_t n_windows, uint32_t k,
                                         hd_tune_result *best, hd_tune_result *all, uint32_t cap,
                                         uint32_t *n_all);

/* Continuous-batching server (no counterpart in the paper, which batches to
 * fill memory, Section 4.1).  A scheduler thread keeps the library resident
 * and coalesces the pending requests into batches whenever one of `slots`
 * execution slots (each its own stream) is free and the device-memory budget
 * allows; batches in different slots overlap on the device.  Each request's
 * results equal those of searching it alone.  A multi-bit library (Section
 * 4.3) is served too: its requests are encoded into components
 * (hd_encode_multibit with the library's bits), scored by the dot-product
 * search (hd_search_dot; `form` AUTO or a tensor-core form the library holds)
 * and submitted with hd_server_submit_dot. */
typedef struct hd_server hd_server;
typedef struct {
    uint32_t slots;               /* batches in flight at once, 1..64 */
    uint32_t max_batch_queries;   /* most queries coalesced into one batch (a larger request runs alone) */
    uint64_t mem_budget_bytes;    /* device bytes in-flight batches may hold; 0 = half the free memory */
    uint32_t k;                   /* top-k of every request, 1..16 */
    hd_search_form form;          /* scoring form of every batch */
} hd_server_params;
typedef struct {
    double latency_s;             /* submit -> results in the caller's buffers */
    double queue_s;               /* submit -> its batch started */
    uint32_t n_queries, batch_queries;
} hd_request_info;
typedef struct {
    uint64_t submitted, completed, queries, batches;
    uint32_t max_inflight;        /* most batches seen in flight at once */
} hd_server_stats;
HD_API hd_status hd_server_create(hd_ctx *ctx, const hd_library *lib, const hd_server_params *params,
                                  hd_server **out);
/* Queues one request: a CSR batch of n_q spectra (h_offsets [n_q+1] into
 * h_bins / h_levels), precursor m/z and charges, and its window.  Inputs are
 * copied before returning; h_out_idx / h_out_dist [n_q][k] must stay valid
 * until hd_server_wait returns for this request. */
HD_API hd_status hd_server_submit(hd_server *srv, const uint32_t *h_offsets, const uint32_t *h_bins,
                                  const uint8_t *h_levels, const double *h_q_mz, const uint8_t *h_q_charge,
                                  uint32_t n_q, double tol, hd_tol_unit unit, uint32_t *h_out_idx,
                                  uint16_t *h_out_dist, uint64_t *request_id);
/* hd_server_submit for a server on a multi-bit library: h_out_score
 * [n_q][k] receives the dot-product scores (padding INT32_MIN, as
 * hd_search_dot).  Each submit call fails with HD_ERR_INVALID_ARG on the
 * other kind of library. */
HD_API hd_status hd_server_submit_dot(hd_server *srv, const uint32_t *h_offsets, const uint32_t *h_bins,
                                      const uint8_t *h_levels, const double *h_q_mz, const uint8_t *h_q_charge,
                                      uint32_t n_q, double tol, hd_tol_unit unit, uint32_t *h_out_idx,
                                      int32_t *h_out_score, uint64_t *request_id);
/* Blocks until the request is done (HD_ERR_TIMEOUT after timeout_s > 0). */
HD_API hd_status hd_server_wait(hd_server *srv, uint64_t request_id, double timeout_s, hd_request_info *info);
HD_API hd_status hd_server_stats_get(hd_server *srv, hd_server_stats *out);
/* Device-time record of finished batches (the last 4096), oldest first: two
 * batches ran on the device at the same time when their [start, end)
 * intervals intersect.  start: the batch's first host-to-device copy began;
 * end: its last device-to-host copy finished; both in ms of device time
 * since the server was created (CUDA events on the slot's stream). */
typedef struct {
    uint64_t batch;               /* launch order, from 0 */
    uint32_t slot;                /* execution slot (stream) it ran on */
    uint32_t n_queries, n_requests;
    double device_start_ms, device_end_ms;
} hd_batch_record;
HD_API hd_status hd_server_batch_log(hd_server *srv, hd_batch_record *out, uint32_t cap, uint32_t *n);
/* Drains every queued request, then stops the scheduler. */
HD_API void hd_server_destroy(hd_server *srv);

/* End to end from host memory: copies a CSR query batch (h_offsets [n_q+1],
 * h_bins / h_levels [h_offsets[n_q]]), its precursor m/z and charges to the
 * device, encodes it with `ctx`, searches `lib`, copies the results to
 * h_out_idx / h_out_dist [n_q][k] and synchronises `stream`.  Synchronous. */
HD_API hd_status hd_search_host(hd_ctx *ctx, const hd_library *lib, const uint32_t *h_offsets,
                         const uint32_t *h_bins, const uint8_t *h_levels, const double *h_q_mz,
                         const uint8_t *h_q_charge, uint32_t n_q, double tol, hd_tol_unit unit,
                         uint32_t k, uint32_t *h_out_idx, uint16_t *h_out_dist, hd_stream stream);

/* hd_search_open with no device allocation (the paper has no counterpart:
 * this serves callers that cannot allocate device memory while running, e.g.
 * a server that reserved its memory up front or a host thread that must not
 * block in the allocator).  Same arguments, results and padding as
 * hd_search_open; the scratch comes from one fixed device buffer of 32 MiB
 * held by every GPU that loads libhd until the process exits.  A request
 * that needs more scratch than that (on a 152-SM GPU: above about 140,000
 * queries at 9 <= k <= 16, more at smaller k) is rejected with
 * HD_ERR_INVALID_ARG before any launch.
 * Set-up: the first call on a device (n_q = 0 is enough; it launches
 * nothing) looks up the buffer's device address, and with lazy module
 * loading (the CUDA default) that lookup is what loads the buffer, so its
 * 32 MiB are reserved then.  Make that call once per device at start-up,
 * before reserving the rest of the device memory and before any stream
 * capture.  The address is kept for the life of the process: do not use this
 * entry point on a device after cudaDeviceReset.  All calls share the
 * buffer: calls whose kernels overlap on the GPU (other streams, other host
 * threads) race and corrupt each other -- serialise them.  Asynchronous. */
HD_API hd_status hd_search_open_noalloc(const hd_library *lib, const uint64_t *d_q_hv,
                                        const double *d_q_mz, const uint8_t *d_q_charge, uint32_t n_q,
                                        double tol, hd_tol_unit unit, uint32_t k, uint32_t *d_out_idx,
                                        uint16_t *d_out_dist, hd_stream stream);

/* Multi-bit HV components (Section 4.3: a higher precision per component
 * is the paper's second way to raise the identification rate; it names no
 * quantiser).  Reading: the encoder's integer bundle I (Eq. 1, or the
 * projection sum when the context's encoder is HD_ENC_PROJECTION) is
 * quantised with the spectrum's own step, M = max_d |I_d|,
 * m = 2^(bits-1) - 1:
 *     h_d = sign(I_d) * floor((2 m |I_d| + M) / (2 M))    (h = 0 if M = 0),
 * i.e. m |I_d| / M rounded half up in magnitude; h_d in [-m, m].  Two
 * spectra score by the dot product S = sum_d h_q,d h_r,d, which for +-1
 * components is D - 2 dist; higher is better.
 *
 * hd_encode_multibit writes d_out [n_spectra][D] int8 (16-byte aligned),
 * bits in 2..5; same CSR input and errors as hd_encode.
 * hd_build_library_multibit sorts and copies such rows like hd_build_library
 * (d_comp [n_refs][D] int8, 16-byte aligned, components in [-m, m]; rows out
 * of range fail with HD_ERR_INVALID_ARG) and prepares the tensor-core copy
 * HD_FORM_TC_FP4 (bits <= 3: every |h| <= 3 is exact in e2m1) or
 * HD_FORM_TC_FP8 (e4m3 holds the integers up to 16 exactly);
 * hd_library_prepare adds HD_FORM_TC_FP8 or HD_FORM_TC_BF16 (and
 * HD_FORM_TC_FP4 for bits <= 3).  Every partial sum is an integer of size at
 * most D m^2 < 2^24, so the fp32 accumulation is exact.  HD_FORM_POPC
 * scores the same S on the integer pipes once hd_library_prepare built the
 * bit planes: with u = h + m in `bits` planes Q_i, R_i and U the row sums of
 * u, S = sum over plane pairs of 2^(i+j) popc(Q_i & R_j) - m (U_q + U_r) +
 * D m^2 (exact integer arithmetic).  Such a library is searched only with
 * the dot-product calls (hd_search_dot, hd_search_dot_multi,
 * hd_cascade_search_dot, hd_plan_create_dot, hd_library_autotune_dot); the
 * binary entry points (hd_search_*, cascade, plan, autotune, export) reject
 * it with HD_ERR_INVALID_ARG; hd_library_save / hd_library_load keep it and
 * the server serves it (hd_server_submit_dot).  `form` of the dot-product
 * calls: AUTO, HD_FORM_POPC or a tensor-core form the library holds.
 * hd_search_dot: windows as hd_search_open (Section 3.4); per query the k
 * best candidates by S, higher first, the lower input index on a tie; d_q_comp
 * [n_q][D] int8 (16-byte aligned, components in [-m, m]; others flag
 * HD_ERR_INVALID_ARG on the library's status), d_out_idx / d_out_score
 * [n_q][k]; missing slots hold 0xFFFFFFFF / INT32_MIN.  Asynchronous. */
HD_API hd_status hd_encode_multibit(hd_ctx *ctx, const uint32_t *d_offsets, const uint32_t *d_bins,
                                    const uint8_t *d_levels, uint32_t n_spectra, uint32_t bits, int8_t *d_out,
                                    hd_stream stream);
HD_API hd_status hd_build_library_multibit(hd_ctx *ctx, const int8_t *d_comp, const double *d_prec_mz,
                                           const uint8_t *d_charge, uint32_t n_refs, uint32_t bits,
                                           hd_library **out);
/* Component bits of a library: 1 for binary HVs. */
HD_API hd_status hd_library_component_bits(const hd_library *lib, uint32_t *bits);
HD_API hd_status hd_search_dot(const hd_library *lib, const int8_t *d_q_comp, const double *d_q_mz,
                               const uint8_t *d_q_charge, uint32_t n_q, double tol, hd_tol_unit unit, uint32_t k,
                               hd_search_form form, uint32_t *d_out_idx, int32_t *d_out_score, hd_stream stream);
/* hd_search_dot with a window per query, as hd_search_open_multi: query q
 * uses windows[d_q_class[q]] (windows[0] for every query when d_q_class is
 * NULL), in one persistent search launch. */
HD_API hd_status hd_search_dot_multi(const hd_library *lib, const int8_t *d_q_comp, const double *d_q_mz,
                                     const uint8_t *d_q_charge, const uint8_t *d_q_class, uint32_t n_q,
                                     const hd_window *windows, uint32_t n_windows, uint32_t k, hd_search_form form,
                                     uint32_t *d_out_idx, int32_t *d_out_score, hd_stream stream);

/* Failure-detection hooks (no counterpart in the paper).  Every device wait
 * of a search (stage loads, tensor-core commits, merge locks) gives up after
 * a bounded time, records HD_ERR_TIMEOUT in the library's status word and
 * lets its kernel return, leaving the CUDA context usable.
 * hd_library_set_wait_limit sets that bound (0: 2 s; otherwise >= 1 ms).
 * hd_library_inject_stall makes the next n searches on this library arm one
 * stage barrier and never issue its load, so that a wait does run out: the
 * test hook for that path.  No trap, fault or endless loop is involved. */
HD_API hd_status hd_library_set_wait_limit(hd_library *lib, uint64_t ns);
HD_API hd_status hd_library_inject_stall(hd_library *lib, uint32_t n_searches);

/* Measurement hooks (no counterpart in the paper).  While enabled, libhd
 * records a CUDA event pair around every launch of the given kernel kind, on
 * the stream the kernel runs on.  hd_profile_collect() waits for the
 * recorded events, returns their summed milliseconds and the launch count,
 * and forgets them.  hd_launch_count() is the number of kernels libhd has
 * launched in this process. */
typedef enum { HD_KERNEL_ENCODE = 0, HD_KERNEL_SEARCH = 1, HD_KERNEL_KINDS = 2 } hd_kernel_kind;

/* Instruction-rate microbenchmarks (no counterpart in the paper; the rates
 * the search kernels are held to).  Synchronous; each kind runs one warm-up
 * launch and `launches` (1..1000) timed launches on a stream of its own, on
 * the current device, and reports operations per second.
 *  HD_PEAK_TC_FP4 / _FP8 / _BF16  tcgen05.mma.cta_group::2 with M = 256,
 *      N = 256 and 32 bytes of K per instruction (kind::f8f6f4 with e2m1 or
 *      e4m3 operands, kind::f16 with bf16), the pair search's instruction
 *      and shape, on operands resident in shared memory, one CTA per SM, all
 *      SM pairs; an operation is a flop (2 per multiply-add).
 *  HD_PEAK_TC_MXF4  tcgen05.mma.cta_group::2.kind::mxf4.block_scale with
 *      M = 256, N = 240, K = 64 packed e2m1 components and unit ue8m0 scale
 *      factors; its warm-up launch runs on all-(+1) operands and checks that
 *      every accumulator holds the exact sum (HD_ERR_CUDA otherwise).
 *  HD_PEAK_POPC  32-bit population counts (the popcount form's counting
 *      instruction, Section 4.1); an operation is one popcount.
 *  HD_PEAK_LOP3  three-input logic operations on 32-bit words (the carry-save
 *      popcount form's adder); an operation is one LOP3. */
typedef enum { HD_PEAK_TC_FP4 = 0, HD_PEAK_TC_FP8 = 1, HD_PEAK_TC_BF16 = 2, HD_PEAK_POPC = 3,
               HD_PEAK_LOP3 = 4, HD_PEAK_TC_MXF4 = 5 } hd_peak_kind;
typedef struct {
    double best_per_s;        /* operations per second of the fastest timed launch */
    double median_per_s;      /* ... of the median timed launch */
    double ms_best;           /* duration of the fastest timed launch */
    uint64_t ops_per_launch;
    uint32_t sms;             /* SMs the launch covered */
    uint32_t launches;        /* timed launches */
} hd_peak_result;
HD_API hd_status hd_measure_peak(hd_peak_kind kind, uint32_t launches, hd_peak_result *out);
HD_API hd_status hd_profile_enable(int on);
HD_API hd_status hd_profile_collect(hd_kernel_kind kind, double *total_ms, uint32_t *launches);
HD_API uint64_t hd_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* HD_H */
