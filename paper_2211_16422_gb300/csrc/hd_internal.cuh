// hd_internal.cuh -- definitions shared by the CUDA translation units of
// libhd: object layouts, device status flags, launch helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "hd.h"

// ---------------------------------------------------------------------------
// Device status word.  Kernels OR these bits into a word in mapped page-locked
// host memory; the host reads it without a device synchronisation.
// ---------------------------------------------------------------------------
enum : uint32_t {
    HD_DEV_BAD_INPUT = 1u,   // malformed CSR row, bin or level out of range, ...
    HD_DEV_TIMEOUT = 2u,     // a bounded wait (mbarrier, work queue) expired
    HD_DEV_TMEM = 4u         // the two CTAs of a pair were given different tensor-memory columns
};

__device__ __forceinline__ void hd_flag(uint32_t *status, uint32_t bits)
{
    if (status) atomicOr_system(status, bits);
}

// Every device-side wait gives up after this much wall time, flags
// HD_DEV_TIMEOUT and lets its kernel return.
constexpr uint64_t HD_WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint64_t hd_globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct hd_status_word {
    uint32_t *host = nullptr;   // mapped, page-locked
    uint32_t *dev = nullptr;    // device alias of `host`
};

struct hd_ctx {
    hd_params p{};
    int device = 0;
    int num_sms = 0;
    uint32_t W = 0;               // D / 64
    uint64_t *F = nullptr;        // [n_bins][W]
    uint64_t *L = nullptr;        // [n_levels][W]
    uint32_t *rank_F = nullptr;   // [D]
    uint32_t *rank_L = nullptr;   // [D]
    hd_status_word status;
};

// Schedule of the tensor-core search: tiles of 256 reference rows are grouped
// in runs of `tile_group` (one work item per query block and group), and
// `super_group` groups form the slice of the library the running CTAs share
// through L2.  0 = default.
struct hd_mma_tuning {
    uint32_t tile_group = 0;
    uint32_t super_group = 0;
    uint32_t cluster = 0;    // CTAs per cluster: 2 for the SM pair, 1 for one SM
    uint32_t cta_group = 0;  // 2: SM pairs issue M = 256 MMAs (cluster of 2); 0/1: one SM per MMA
    uint32_t tiles_per_stage = 0;   // kind::mxf4 on SM pairs: reference tiles per query stage (0/1 or 2)
};

struct hd_library {
    uint32_t n = 0, dim = 0, W = 0;
    int device = 0;
    int num_sms = 0;
    uint64_t *hv = nullptr;        // [n][W] sorted rows
    double *mz = nullptr;          // [n]
    uint8_t *charge = nullptr;     // [n]
    uint32_t *orig = nullptr;      // [n] input index of each row
    uint32_t *charge_start = nullptr;   // [257] first row with charge >= c (device)
    uint8_t *x_fp8 = nullptr;      // [n][D] bipolar e4m3 rows (tensor-core form), optional
    uint8_t *x_bf16 = nullptr;     // [n][2D] bipolar bf16 rows (tensor-core form), optional
    uint8_t *x_fp4 = nullptr;      // [n][D/2] bipolar e2m1 rows, two per byte (tensor-core form), optional
    uint8_t *decoy = nullptr;      // [n] decoy flags, input order, optional
    uint32_t bits = 1;             // component bits: 1 = binary rows in hv; 2..5 = int8 rows in comp
    int8_t *comp = nullptr;        // [n][D] multi-bit components, sorted rows (bits > 1)
    uint32_t *x_planes = nullptr;  // popc form of a multi-bit library: bit planes of h + m, [n][bits * D/32]
    uint32_t *usum = nullptr;      // [n] sum over d of (h_d + m) of each sorted row
    hd_mma_tuning mma_tuning;
    hd_search_form auto_form = HD_FORM_AUTO;   // set by the autotuner
    uint64_t wait_ns = 0;                      // device wait limit (0: HD_WAIT_NS)
    mutable uint32_t inject_stalls = 0;        // test hook: searches that drop their first load
    uint32_t charge_start_h[257] = {};
    hd_status_word status;
};

// ---------------------------------------------------------------------------
// Host-side error reporting.
// ---------------------------------------------------------------------------
hd_status hd_fail(hd_status s, const std::string &msg);
hd_status hd_cuda_fail(cudaError_t e, const char *what);

#define HD_CUDA_TRY(call)                                                   \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return hd_cuda_fail(e_, #call);              \
    } while (0)

// Launch accounting and the optional event timing of the hot kernels.
void hd_count_launches(uint32_t n);
struct hd_prof_scope {
    hd_prof_scope(hd_kernel_kind kind, cudaStream_t s);
    ~hd_prof_scope();
    hd_kernel_kind kind;
    cudaStream_t s;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
};

static inline unsigned hd_ceil_div(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// Stream-ordered scratch arena: one cudaMallocAsync, carved in 256-byte
// aligned pieces, released with cudaFreeAsync on the same stream.
// ---------------------------------------------------------------------------
struct hd_arena {
    size_t used = 0;
    char *base = nullptr;
    template <class T> T *take(size_t count)
    {
        size_t off = (used + 255) & ~size_t(255);
        used = off + count * sizeof(T);
        return base ? reinterpret_cast<T *>(base + off) : nullptr;
    }
};

// ---------------------------------------------------------------------------
// Launchers implemented in the other translation units.
// ---------------------------------------------------------------------------
hd_status hd_item_memory_build(hd_ctx *ctx, cudaStream_t s);
void hd_random_words_launch(uint64_t seed, uint32_t stream, uint32_t n, uint32_t *out, cudaStream_t s);

hd_status hd_preprocess_launch(const hd_preprocess_params &pp, const uint32_t *raw_off,
                               const double *raw_mz, const double *raw_int, uint32_t n,
                               uint32_t *out_off, uint32_t *out_bins, uint8_t *out_levels,
                               uint32_t *status, cudaStream_t s);

void hd_encode_launch(const hd_ctx *ctx, const uint32_t *off, const uint32_t *bins,
                      const uint8_t *levels, uint32_t n, uint64_t *out, cudaStream_t s);

// Candidate windows of a query set (Section 3.4): query q uses window
// w[cls[q]] (w[0] when cls is null).  `unit` is an hd_tol_unit.  For ppm,
// `tol` holds tol * 1e-6 and the window half-width is mz_q * tol; for
// neutral masses the half-width applies to (mz - 1.007276) * charge.  Passed
// to kernels by value.
struct hd_win {
    double tol;
    int unit;
};
struct hd_qwin {
    const uint8_t *cls = nullptr;
    uint32_t n = 1;
    hd_win w[HD_MAX_WINDOWS] = {};
};
hd_qwin hd_single_window(double tol, hd_tol_unit unit);

// Test hook: true (and one fewer pending) when this search must drop its
// first stage load so that a bounded device wait runs out.
bool hd_take_injected_stall(const hd_library *lib);
inline uint64_t hd_wait_limit(const hd_library *lib) { return lib->wait_ns ? lib->wait_ns : HD_WAIT_NS; }

// Stable sort of n items by (group, charge, m/z), group optional: writes the
// permutation `perm` (perm[rank] = input index).  Scratch from `arena`
// (sized by a first call with arena.base == nullptr).
void hd_sort_charge_mz(const double *mz, const uint8_t *charge, const uint8_t *group, uint32_t n,
                       uint32_t *perm, hd_arena &arena, cudaStream_t s);

void hd_windows_launch(const hd_library *lib, const double *q_mz, const uint8_t *q_charge,
                       const uint32_t *perm, uint32_t n_q, const hd_qwin &win, uint32_t *lo,
                       uint32_t *hi, cudaStream_t s);

hd_status hd_search_popc_run(const hd_library *lib, const uint64_t *q_hv, const double *q_mz,
                             const uint8_t *q_charge, uint32_t n_q, const hd_qwin &win,
                             uint32_t k, uint32_t *out_idx, uint16_t *out_dist, cudaStream_t s);

// hd_search_popc_run on caller-provided device scratch (nothing allocated);
// fails with HD_ERR_INVALID_ARG when the request needs more than
// `scratch_bytes`.
hd_status hd_search_popc_run_scratch(const hd_library *lib, const uint64_t *q_hv, const double *q_mz,
                                     const uint8_t *q_charge, uint32_t n_q, const hd_qwin &win,
                                     uint32_t k, uint32_t *out_idx, uint16_t *out_dist, cudaStream_t s,
                                     void *scratch, size_t scratch_bytes);

// Tensor-core form: the bipolar copy of the library rows, and the search.
hd_status hd_library_expand(hd_library *lib, hd_search_form form, cudaStream_t s);
hd_status hd_peak_mma_run(hd_search_form form, uint32_t launches, hd_peak_result *out);
hd_status hd_peak_alu_run(bool popc, uint32_t launches, hd_peak_result *out);
hd_status hd_search_mma_run(const hd_library *lib, hd_search_form form, const uint64_t *q_hv, const double *q_mz,
                            const uint8_t *q_charge, uint32_t n_q, const hd_qwin &win, uint32_t k,
                            uint32_t *out_idx, uint16_t *out_dist, cudaStream_t s);

// Multi-bit components: encode, and the dot-product search on the tensor-core
// forms (scores S = sum_d h_q,d h_r,d; keys (D m^2 - S, orig)).
void hd_encode_mb_launch(const hd_ctx *ctx, const uint32_t *off, const uint32_t *bins, const uint8_t *levels,
                         uint32_t n, uint32_t bits, int8_t *out, cudaStream_t s);
hd_status hd_search_mma_dot_run(const hd_library *lib, hd_search_form form, const int8_t *q_comp,
                                const double *q_mz, const uint8_t *q_charge, uint32_t n_q, const hd_qwin &win,
                                uint32_t k, uint32_t *out_idx, int32_t *out_score, cudaStream_t s);
// The popcount form of the dot product (bit planes of the offset components
// h + m, S = sum over plane pairs of 2^(i+j) popc(Q_i & R_j) - m (U_q + U_r)
// + D m^2), and the library's planes it reads (hd_library_prepare).
hd_status hd_library_planes(hd_library *lib, cudaStream_t s);
hd_status hd_search_popc_dot_run(const hd_library *lib, const int8_t *q_comp, const double *q_mz,
                                 const uint8_t *q_charge, uint32_t n_q, const hd_qwin &win, uint32_t k,
                                 uint32_t *out_idx, int32_t *out_score, cudaStream_t s);
inline hd_status hd_search_dot_dispatch(const hd_library *lib, hd_search_form form, const int8_t *q_comp,
                                        const double *q_mz, const uint8_t *q_charge, uint32_t n_q,
                                        const hd_qwin &win, uint32_t k, uint32_t *out_idx, int32_t *out_score,
                                        cudaStream_t s)
{
    return form == HD_FORM_POPC
               ? hd_search_popc_dot_run(lib, q_comp, q_mz, q_charge, n_q, win, k, out_idx, out_score, s)
               : hd_search_mma_dot_run(lib, form, q_comp, q_mz, q_charge, n_q, win, k, out_idx, out_score, s);
}
inline uint32_t hd_comp_max(uint32_t bits) { return (1u << (bits - 1)) - 1u; }
// The tensor-core copy a form scores (kind::mxf4 shares the e2m1 rows), and
// the fastest tensor-core form the library is prepared for (HD_FORM_AUTO when
// none): kind::mxf4 needs D to be a multiple of 256.
inline const uint8_t *hd_tc_copy(const hd_library *lib, hd_search_form f)
{
    return f == HD_FORM_TC_FP8 ? lib->x_fp8
         : f == HD_FORM_TC_BF16 ? lib->x_bf16
         : (f == HD_FORM_TC_FP4 || f == HD_FORM_TC_MXF4) ? lib->x_fp4 : nullptr;
}
inline bool hd_is_tc_form(hd_search_form f)
{
    return f == HD_FORM_TC_FP8 || f == HD_FORM_TC_BF16 || f == HD_FORM_TC_FP4 || f == HD_FORM_TC_MXF4;
}
inline hd_search_form hd_fastest_tc_form(const hd_library *lib)
{
    if (lib->x_fp4) return lib->dim % 256 == 0 ? HD_FORM_TC_MXF4 : HD_FORM_TC_FP4;
    if (lib->x_fp8) return HD_FORM_TC_FP8;
    if (lib->x_bf16) return HD_FORM_TC_BF16;
    return HD_FORM_AUTO;
}
// The copy a dot-product form reads: the bit planes for popc, else the
// tensor-core copy.
inline const void *hd_dot_copy(const hd_library *lib, hd_search_form f)
{
    return f == HD_FORM_POPC ? static_cast<const void *>(lib->x_planes) : static_cast<const void *>(hd_tc_copy(lib, f));
}
// Form of a dot-product search (multi-bit library): AUTO takes the
// autotuner's choice when the library holds its copy, else the fastest
// prepared tensor-core form, else popc on prepared bit planes, else bf16
// (which the caller then finds unprepared).
inline hd_search_form hd_dot_form(const hd_library *lib, hd_search_form f)
{
    if (f != HD_FORM_AUTO) return f;
    if (lib->auto_form != HD_FORM_AUTO && hd_dot_copy(lib, lib->auto_form)) return lib->auto_form;
    const hd_search_form g = hd_fastest_tc_form(lib);
    if (g != HD_FORM_AUTO) return g;
    return lib->x_planes ? HD_FORM_POPC : HD_FORM_TC_BF16;
}
// Checks of a dot-product form (resolving AUTO): a known form the library
// holds the copy of (an empty library needs none); kind::mxf4 needs D % 256.
hd_status hd_dot_check(const hd_library *lib, hd_search_form *form, const std::string &name);
// Entry points that score binary HVs refuse a multi-bit library.
inline bool hd_lib_binary(const hd_library *lib) { return lib->bits == 1; }

// Search dispatch shared by the entry points: resolves HD_FORM_AUTO and runs
// the chosen form.
hd_status hd_search_dispatch(const hd_library *lib, const uint64_t *q_hv, const double *q_mz,
                             const uint8_t *q_charge, uint32_t n_q, const hd_qwin &win, uint32_t k,
                             hd_search_form form, uint32_t *out_idx, uint16_t *out_dist, cudaStream_t s);
// Host-side validation of a window table into an hd_qwin.
hd_status hd_make_qwin(const uint8_t *cls, const hd_window *windows, uint32_t n_windows, hd_qwin *out);
