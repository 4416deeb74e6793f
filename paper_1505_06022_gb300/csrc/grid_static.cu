// grid_static.cu -- hash-grid build that allocates no device memory.
//
// Some callers cannot allocate device memory: a host whose device memory is owned by another
// allocator or memory pool (which forbids side allocations), a plugin that is handed fixed
// buffers, a real-time loop that must not block on cudaMalloc's implicit synchronisation.
// gsp_hash_grid_build_static serves them: the caller passes the input and output buffers, and
// the scratch the build needs comes from a fixed array in this library's device image instead of
// cudaMalloc.
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
// 4 key/value words per point + radix histogram (256 x 512) + scan partials of the largest
// table (2^24 / 2048 + 1) + 64 words for the device-side count: 2,236,481 words (8.53 MiB).
constexpr int64_t kWords = 4 * kMaxPoints + 256 * 512 + (kMaxTable / 2048 + 1) + 64;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) uint32_t g_grid_scratch[kWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_ptr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" gsp_status gsp_hash_grid_build_static(const float* d_pos, int64_t n, float cell_h, int64_t table_size,
                                                 uint32_t* d_order, uint32_t* d_bstart, void* stream) {
    if (n < 0 || !(cell_h > 0.0f) || !std::isfinite(cell_h) || table_size < 1 || (table_size & (table_size - 1)) ||
        !d_bstart || (n > 0 && (!d_pos || !d_order)) || ((uintptr_t)d_pos & 15))
        return GSP_ERR_INVALID_ARG;
    if (n > kMaxPoints || table_size > kMaxTable) {
        gsp_set_last_error("gsp_hash_grid_build_static: at most " + std::to_string(kMaxPoints) + " points and " +
                           std::to_string(kMaxTable) + " buckets fit its static scratch (got n = " +
                           std::to_string(n) + ", table_size = " + std::to_string(table_size) + ")");
        return GSP_ERR_INVALID_ARG;
    }
    if (gsp_grid_scratch_words(n, table_size) > kWords) return GSP_ERR_INVALID_ARG;
    int dev = 0;
    GSP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return GSP_ERR_INVALID_ARG;
    uint32_t* scratch = nullptr;
    {
        // Host code cannot use g_grid_scratch directly (its host-side name is only a stand-in):
        // look up its device address once per device, with that device current.
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_ptr[dev]) {
            void* p = nullptr;
            GSP_CUDA_TRY(cudaGetSymbolAddress(&p, g_grid_scratch));
            g_ptr[dev] = (uint32_t*)p;
        }
        scratch = g_ptr[dev];
    }
    (void)cudaGetLastError();
    return gsp_grid_build_with((const float4*)d_pos, n, cell_h, table_size, d_order, d_bstart, scratch,
                               (cudaStream_t)stream, false);
}
