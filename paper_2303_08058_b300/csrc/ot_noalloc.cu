// Allocation-free variant of the multipole pass.
//
// Some callers cannot allocate device memory at the point where they call the
// interaction kernels: code running while a stream is being captured into a
// CUDA graph (cudaMalloc is not a stream operation and breaks the capture),
// real-time loops that forbid allocator calls after set-up, and hosts whose
// device memory is fully reserved by another allocator.  The regular
// ot_multipole_interactions keeps its per-cell scratch (pre-scaled, reduced
// source moments) in the grid's arena, which ot_grid_create obtains with
// cudaMalloc.  The entry point below instead keeps that scratch in one
// file-scope device array of fixed size, so the call itself allocates
// nothing.
#include <cuda.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

#include "ot.h"
#include "ot_internal.h"

// defined in ot_lib.cu: the multipole pass with caller-supplied scratch, the
// setter of the calling thread's error message, and the live-handle check
ot_status otk_multipole_with_scratch(ot_grid* g, const double* M, double* L, double* Lc, double* scratch,
                                     size_t scratch_doubles, cudaStream_t s);
ot_status otk_set_error(ot_status code, const char* msg);
bool otk_grid_live(const ot_grid* g);

namespace {

// 16 MiB: reduced moments of 256 consecutive sub-grid indices (64 KiB each).
// Every device that loads the library holds this array until the process exits.
constexpr size_t kNoAllocScratchDoubles = static_cast<size_t>(OT_NOALLOC_SCRATCH_BYTES) / sizeof(double);
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;

// The array's device address, found once per device and context: a context
// destroyed and created again (cudaDeviceReset, a torn-down primary context)
// gets a new id, and the address is looked up again for it.
struct ScratchAddr {
    unsigned long long ctx_id;
    double* ptr;
};
ScratchAddr g_scratch_addr[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult(CUDAAPI*)(CUcontext*);
using CtxGetIdFn = CUresult(CUDAAPI*)(CUcontext, unsigned long long*);

// id of the calling thread's current context (unique over the process's
// lifetime), through the driver entry points the runtime resolves
bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            cudaGetLastError();
            return false;
        }
        get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the array on the current device.  In host code the name
// g_noalloc_scratch is only a host-side stand-in, not a device address, so
// it is looked up with the device current: on the first call on a device
// (and again only if that device's context was replaced).
ot_status scratch_address(int dev, double** out, const char** why) {
    if (dev < 0 || dev >= kMaxDevices) {
        *why = "device index beyond the supported 64";
        return OT_EINVAL;
    }
    unsigned long long ctx = 0;
    if (!current_context_id(&ctx)) {
        *why = "no current CUDA context on this thread";
        return OT_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    ScratchAddr& a = g_scratch_addr[dev];
    if (!a.ptr || a.ctx_id != ctx) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            *why = "cudaGetSymbolAddress of the static scratch array failed";
            return OT_ECUDA;
        }
        a.ptr = static_cast<double*>(p);
        a.ctx_id = ctx;
    }
    *out = a.ptr;
    return OT_OK;
}

}  // namespace

extern "C" ot_status ot_multipole_interactions_noalloc(ot_grid* grid, const double* M, double* L, double* Lc,
                                                       void* stream) {
    try {
        if (!grid) return otk_set_error(OT_EINVAL, "grid is NULL");
        if (!otk_grid_live(grid))
            return otk_set_error(OT_EINVAL, "grid handle is not live (destroyed or never created)");
        int dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            return otk_set_error(OT_ECUDA, "cudaGetDevice failed");
        }
        double* scratch = nullptr;
        const char* why = "";
        const ot_status st = scratch_address(dev, &scratch, &why);
        if (st != OT_OK) return otk_set_error(st, why);
        return otk_multipole_with_scratch(grid, M, L, Lc, scratch, kNoAllocScratchDoubles,
                                          static_cast<cudaStream_t>(stream));
    } catch (...) {
        // std::mutex can throw std::system_error; nothing crosses the C ABI
        return otk_set_error(OT_EINVAL, "unexpected host exception");
    }
}
