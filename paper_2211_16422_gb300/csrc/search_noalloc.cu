// search_noalloc.cu -- hd_search_open_noalloc: the open search with no device
// allocation at all.
//
// Who needs it: callers that cannot call cudaMalloc (or the stream-ordered
// allocator) while they run -- a serving process that reserved all of its
// device memory up front and must not grow, a real-time host thread that may
// not block in the allocator, a host program whose memory budget forbids new
// allocations after start-up.  hd_search_open allocates its scratch (query
// order, windows, work list, partial top-k lists) on every call; this entry
// point takes it from one fixed buffer instead.
//
// The scratch is a file-scope device array of HD_NOALLOC_SCRATCH_BYTES.  It
// exists once per GPU that loads this library and stays reserved until the
// process exits.  In host code the array's name is only a host-side stand-in,
// not a device address, so its device address is looked up with
// cudaGetSymbolAddress -- once per device, with that device current, on the
// first call made on that device, even one with no queries -- and that
// address is what the kernels get.  With lazy module loading that lookup is
// what loads this file's module and reserves the 32 MiB, so callers make a
// first call at start-up, before the rest of their memory is reserved and
// before any stream capture.  The cached address would be stale after
// cudaDeviceReset, which callers of this entry point must not do.
//
// All calls share the one array and it keeps whatever the last call left in
// it.  Every piece of it is written before it is read within a call (the work
// counter, the one value that must start at zero, is cleared by the work-list
// kernel of each call), so leftovers do no harm.  Two calls whose kernels
// overlap on the GPU -- different streams, or different host threads -- race
// on the array and corrupt each other's results: serialise them.
#include <mutex>

#include "hd_internal.cuh"

namespace {

constexpr size_t HD_NOALLOC_SCRATCH_BYTES = size_t(32) << 20;   // 32 MiB
constexpr int HD_NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[HD_NOALLOC_SCRATCH_BYTES];

std::mutex g_addr_mu;
void *g_addr[HD_NOALLOC_MAX_DEVICES] = {};

// Device address of g_noalloc_scratch on the current device (looked up once).
hd_status scratch_address(int device, void **out)
{
    if (device < 0 || device >= HD_NOALLOC_MAX_DEVICES)
        return hd_fail(HD_ERR_UNSUPPORTED, "hd_search_open_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> g(g_addr_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return hd_cuda_fail(e, "hd_search_open_noalloc: cudaGetSymbolAddress");
        g_addr[device] = p;
    }
    *out = g_addr[device];
    return HD_OK;
}

}  // namespace

extern "C" hd_status hd_search_open_noalloc(const hd_library *lib, const uint64_t *d_q_hv,
                                            const double *d_q_mz, const uint8_t *d_q_charge,
                                            uint32_t n_q, double tol, hd_tol_unit unit, uint32_t k,
                                            uint32_t *d_out_idx, uint16_t *d_out_dist,
                                            hd_stream stream)
{
    if (!lib) return hd_fail(HD_ERR_INVALID_ARG, "hd_search_open_noalloc: null library");
    if (!hd_lib_binary(lib)) return hd_fail(HD_ERR_INVALID_ARG, "hd_search_open_noalloc: multi-bit library (binary HVs only)");
    if (k < 1 || k > 16) return hd_fail(HD_ERR_INVALID_ARG, "hd_search_open_noalloc: k must be in [1, 16]");
    if (!(tol >= 0.0) || tol > 1.7976931348623157e308)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_search_open_noalloc: tol must be finite and >= 0");
    if (unit != HD_TOL_DA && unit != HD_TOL_PPM && unit != HD_TOL_MASS)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_search_open_noalloc: bad unit");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != lib->device)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_search_open_noalloc: library belongs to another device");
    // set-up first, so that a call with no queries prepares the device
    void *scratch = nullptr;
    const hd_status st = scratch_address(dev, &scratch);
    if (st != HD_OK) return st;
    if (n_q == 0) return HD_OK;
    if (!d_q_hv || !d_q_mz || !d_q_charge || !d_out_idx || !d_out_dist)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_search_open_noalloc: null buffer");
    if (reinterpret_cast<uintptr_t>(d_q_hv) & 15u)
        return hd_fail(HD_ERR_INVALID_ARG, "hd_search_open_noalloc: d_q_hv must be 16-byte aligned");
    return hd_search_popc_run_scratch(lib, d_q_hv, d_q_mz, d_q_charge, n_q,
                                      hd_single_window(tol, unit), k,
                                      d_out_idx, d_out_dist, (cudaStream_t)stream, scratch,
                                      HD_NOALLOC_SCRATCH_BYTES);
}
