// launch.h -- launch configuration and cross-file helpers of the library.
#pragma once

#include "devcommon.cuh"
#include "gsp_internal.h"

constexpr int kTraceThreads = 128;

// Persistent grid size of the closest-hit kernel: SMs x resident blocks per SM.
int gsp_trace_grid(int device);
gspd::DevScene gsp_dev_scene(const gsp_scene* s);
