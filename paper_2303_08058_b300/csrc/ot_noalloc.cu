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
#include <cstddef>
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
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device.  In host code the name
// g_noalloc_scratch is only a host-side stand-in, not a device address, so
// it is looked up once per device with that device current.
ot_status scratch_address(int dev, double** out) {
    if (dev < 0 || dev >= kMaxDevices) return OT_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return OT_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return OT_OK;
}

}  // namespace

extern "C" ot_status ot_multipole_interactions_noalloc(ot_grid* grid, const double* M, double* L, double* Lc,
                                                       void* stream) {
    if (!grid) return otk_set_error(OT_EINVAL, "grid is NULL");
    if (!otk_grid_live(grid)) return otk_set_error(OT_EINVAL, "grid handle is not live (destroyed or never created)");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return otk_set_error(OT_ECUDA, "cudaGetDevice failed");
    }
    double* scratch = nullptr;
    if (scratch_address(dev, &scratch) != OT_OK)
        return otk_set_error(OT_ECUDA, "cudaGetSymbolAddress of the static scratch array failed");
    return otk_multipole_with_scratch(grid, M, L, Lc, scratch, kNoAllocScratchDoubles,
                                      static_cast<cudaStream_t>(stream));
}
