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
#define GSP_TRACE_MIN_BLOCKS 10
#endif
constexpr int kTraceChunk = GSP_TRACE_CHUNK;           // rays a warp takes from the global counter at once
constexpr int kTraceInner = GSP_TRACE_INNER;           // traversal steps between refills
constexpr int kTraceLeafBatch = GSP_TRACE_LEAF_BATCH;  // pending leaves that trigger a warp-wide leaf test

// Persistent grid size of the closest-hit kernel: SMs x resident blocks per SM.
int gsp_trace_grid(int device);
gspd::DevScene gsp_dev_scene(const gsp_scene* s);
