// launch.h -- launch configuration and cross-file helpers of the library.
#pragma once

#include "devcommon.cuh"
#include "gsp_internal.h"

constexpr int kTraceThreads = 128;
#ifndef GSP_TRACE_CHUNK
#define GSP_TRACE_CHUNK 64
#endif
#ifndef GSP_TRACE_INNER
#define GSP_TRACE_INNER 8
#endif
#ifndef GSP_TRACE_LEAF_BATCH
#define GSP_TRACE_LEAF_BATCH 12
#endif
#ifndef GSP_TRACE_MIN_BLOCKS
#define GSP_TRACE_MIN_BLOCKS 9
#endif
#ifndef GSP_PATH_CHUNK
#define GSP_PATH_CHUNK 32
#endif
#ifndef GSP_PATH_MIN_BLOCKS
#define GSP_PATH_MIN_BLOCKS 8
#endif
constexpr int kTraceChunk = GSP_TRACE_CHUNK;           // rays a warp takes from the global counter at once
constexpr int kTraceInner = GSP_TRACE_INNER;           // traversal steps between refills
constexpr int kTraceLeafBatch = GSP_TRACE_LEAF_BATCH;  // pending leaves that trigger a warp-wide leaf test
constexpr int kPathChunk = GSP_PATH_CHUNK;  // paths a warp of the path kernels takes at once (a block's
                                            // grid share is 128 paths: every warp of a short launch gets some)

// Persistent grid size of the closest-hit kernel: SMs x resident blocks per SM.
int gsp_trace_grid(int device);
gspd::DevScene gsp_dev_scene(const gsp_scene* s);

// Closest hit of rays already on the device (a wavefront queue) whose count is read from d_n.
// With a finite refine_factor, hits whose error factor exceeds it get the FP64 distance (and the
// scene's trace counters are reset first); with refine_factor = INFINITY nothing is re-evaluated
// and the counters are reset only if zero_counters is set (else the caller has reset them).
// out_slot: tri receives the hit's leaf-ordered triangle slot instead of its upload-order index.
// ctr (2 u64: next ray, list length) and rlist (max_n entries) belong to the caller.
cudaError_t gsp_trace_queue(const gsp_scene* s, const float4* rays, int64_t max_n, const uint32_t* d_n, int32_t* tri,
                            float* t, float refine_factor, bool zero_counters, bool out_slot, unsigned long long* ctr,
                            int2* rlist, cudaStream_t st);
