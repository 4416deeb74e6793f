// grid_static.cu -- hash-grid build that allocates no device memory.
//
// Some callers cannot allocate device memory: a host whose device memory is owned by another
// allocator or memory pool (which forbids side allocations), a plugin that is handed fixed
// buffers, a real-time loop that must not block on cudaMalloc's implicit synchronisation.
// gsp_hash_grid_build_static serves them: the caller passes the input and output buffers, and
// the scratch the build needs comes from a fixed array in this library's device image instead of
// cudaMalloc.
#include <cuda.h>  // CUcontext / CUresult types only: the driver call is reached through the runtime

#include <cmath>
#include <mutex>
#include <string>

#include "gsp_internal.h"
#include "scan_sort.h"

// Shared with gsp_hash_grid_build (sppm.cu).
int64_t gsp_grid_scratch_words(int64_t n, int64_t T);
gsp_status gsp_grid_build_with(const float4* pos, int64_t n, float cell_h, int64_t T, uint32_t* order,
                               uint32_t* bstart, uint32_t* scratch, cudaStream_t st, bool skip_invalid);

namespace {

constexpr int64_t kMaxPoints = GSP_GRID_STATIC_MAX_POINTS;
constexpr int64_t kMaxTable = GSP_GRID_STATIC_MAX_TABLE;
// The scratch of the largest allowed build, from the same formula the allocating entry point
// sizes its scratch with: 2,236,481 words (8.53 MiB).
constexpr int64_t kWords = gsp_grid_scratch_words_c(kMaxPoints, kMaxTable);
static_assert(kWords == 2236481, "the documented size of the static scratch");

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) uint32_t g_grid_scratch[kWords];

// Device address of g_grid_scratch per device, with the context it was looked up in. A device
// reset or another context made current (driver-API hosts) loads the module again, possibly at
// another address, so the address is looked up again whenever the current context is another one.
// Contexts are told apart by their driver ID, unique for each context the process creates (a
// handle value can come back after a reset; an ID does not).
struct Slot {
    unsigned long long ctx_id = 0;  // 0: unknown
    uint32_t* ptr = nullptr;
};
constexpr int kMaxDevices = 64;
std::mutex g_mu;
Slot g_slot[kMaxDevices];

using CtxGetCurrent = CUresult (*)(CUcontext*);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// A driver entry point through the runtime's query (no link against libcuda); null if the
// driver does not offer it.
void* driver_fn(const char* name) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
        (void)cudaGetLastError();  // the query's own failure: not left for the next call to report
        return nullptr;
    }
    return p;
}

// ID of the calling thread's current context; 0 when there is none or the driver cannot say.
unsigned long long current_context_id() {
    static const CtxGetCurrent get = (CtxGetCurrent)driver_fn("cuCtxGetCurrent");
    static const CtxGetId get_id = (CtxGetId)driver_fn("cuCtxGetId");
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get || !get_id || get(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

}  // namespace

extern "C" gsp_status gsp_hash_grid_build_static(const float* d_pos, int64_t n, float cell_h, int64_t table_size,
                                                 uint32_t* d_order, uint32_t* d_bstart, void* stream) {
    if (n < 0 || !(cell_h > 0.0f) || !std::isfinite(cell_h) || table_size < 1 || (table_size & (table_size - 1)) ||
        !d_bstart || (n > 0 && (!d_pos || !d_order)) || ((uintptr_t)d_pos & 15))
        return GSP_ERR_INVALID_ARG;
    if (n > kMaxPoints || table_size > kMaxTable || gsp_grid_scratch_words(n, table_size) > kWords) {
        gsp_set_last_error("gsp_hash_grid_build_static: at most " + std::to_string(kMaxPoints) + " points and " +
                           std::to_string(kMaxTable) + " buckets fit its static scratch of " +
                           std::to_string(kWords) + " words (got n = " + std::to_string(n) +
                           ", table_size = " + std::to_string(table_size) + ")");
        return GSP_ERR_INVALID_ARG;
    }
    GSP_NO_PENDING_ERROR("gsp_hash_grid_build_static");
    const cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    GSP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return GSP_ERR_INVALID_ARG;
    cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
    GSP_CUDA_TRY(cudaStreamIsCapturing(st, &capture));
    uint32_t* scratch = nullptr;
    {
        // Host code cannot use g_grid_scratch directly (its host-side name is only a stand-in):
        // look up its device address with the device current, once per device and context.
        std::lock_guard<std::mutex> lock(g_mu);
        Slot& s = g_slot[dev];
        const unsigned long long cur = current_context_id();
        // Without a context ID the address is looked up on every call outside capture, and the
        // last one found is used during a capture.
        const bool valid = s.ptr && (cur ? s.ctx_id == cur : capture != cudaStreamCaptureStatusNone);
        if (!valid) {
            if (capture != cudaStreamCaptureStatusNone) {
                gsp_set_last_error("gsp_hash_grid_build_static: the first call on a device or context must come "
                                   "before any stream capture (it looks up the static scratch's address)");
                return GSP_ERR_BAD_STATE;
            }
            void* p = nullptr;
            GSP_CUDA_TRY(cudaGetSymbolAddress(&p, g_grid_scratch));
            s.ptr = (uint32_t*)p;
            s.ctx_id = current_context_id();  // the lookup made the primary context current if none was
        }
        scratch = s.ptr;
    }
    return gsp_grid_build_with((const float4*)d_pos, n, cell_h, table_size, d_order, d_bstart, scratch, st, false);
}
