// gsp_internal.h -- host-side structures shared by the library's translation units.
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "gsp.h"

// Host copy of the packed BVH (Sec. 3.1): per link set, nodes in that set's preorder.
// Node = 2 float4: {min.xyz, miss link}, {max.xyz, leaf word}; triangle = 3 float4:
// {v0.xyz, triangle index}, {v1.xyz, 0}, {v2.xyz, 0}.
struct HostBVH {
    int64_t nnodes = 0;
    int64_t stride = 0;  // nodes per link set in memory: nnodes + 1 (one padding node)
    int64_t nleaves = 0;
    int32_t depth = 0;
    int32_t link_sets = 0;
    std::vector<float4> nodes;  // link_sets * stride * 2
    std::vector<float4> tris;   // nt * 3, leaf order
    // The same tree as child pairs, for stack-based traversal: per internal node (preorder) four
    // float4 {left.min, left ref}, {left.max, right ref}, {right.min, 0}, {right.max, 0}; a ref
    // >= 0 is an internal node, < 0 is ~(leaf word). bin_root: ref of the root.
    std::vector<float4> bin;
    int32_t bin_root = 0;
    double build_ms = 0, thread_ms = 0;
};

// Builds the binned-SAH tree and writes its hit/miss links (one set per ray direction
// class when link_sets == 6). Returns an empty string on success, else an error message.
std::string bvh_build_host(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                           const gsp_bvh_params& p, HostBVH& out);

// Instrumented host walk of a packed BVH (same control flow as the device traversal).
void bvh_host_walk(const HostBVH& bvh, const float* rays, int64_t n, int32_t* tri, float* t,
                   int32_t* visits, int32_t* tests);

struct gsp_context {
    int32_t device = 0;
    int32_t* d_status = nullptr;  // first device-side error (0 = none)
    uint32_t* grid_scratch = nullptr;  // scratch of gsp_hash_grid_build, grown on demand
    int64_t grid_words = 0;
};

struct gsp_scene {
    gsp_context* ctx = nullptr;
    int64_t nv = 0, nt = 0;
    int32_t nmat = 0;
    std::vector<float> verts;
    std::vector<int32_t> tris, tri_mat;
    std::vector<gsp_material> mats;
    bool has_cam = false;
    gsp_camera cam{};
    double extent = 0;  // diagonal of the vertex bounding box
    // device copies
    float4* d_shade = nullptr;  // per triangle (upload order): unit normal xyz, material (int bits)
    float4* d_nlo = nullptr;    // per triangle (upload order): unit normal - its FP32 rounding (xyz)
    float4* d_mats = nullptr;   // per material: {albedo.rgb, type bits}, {emission.rgb, ior}
    float4* d_nodes = nullptr;
    float4* d_tris = nullptr;
    float4* d_bin = nullptr;  // child-pair layout (HostBVH::bin)
    unsigned long long* d_counter = nullptr;  // trace kernel: next ray, refine-list length
    int2* d_rlist = nullptr;                  // trace kernel: hits re-evaluated in FP64
    int64_t rlist_cap = 0;
    bool built = false;
    int32_t step_limit = 0;  // gsp_scene_set_step_limit (0 = the default cap)
    // per-vertex shading data (gsp_scene_set_attributes, gsp_scene_set_texture)
    float4* d_attr = nullptr;  // per triangle (upload order): {n0, s0}, {n1, s1}, {n2, s2}, {t0, t1, t2, flags}
    bool has_texcoords = false;
    std::vector<std::vector<float4>> tex;  // per material: texels {r, g, b, 0}, row-major (empty = none)
    std::vector<int2> tex_size;            // per material: width, height
    float4* d_texels = nullptr;            // every texture, one after the other
    int4* d_mtex = nullptr;                // per material: {first texel, width, height, 0}; null if none
    HostBVH bvh;
    int64_t device_bytes = 0;
    // host-buffer tracing (gsp_trace_closest_hit_host): a pipeline of chunks over kHostLanes
    // streams, each with its own device buffers, trace counters, refine list and pinned staging
    static constexpr int kHostLanes = 3;
    struct HostLane {
        cudaStream_t st = nullptr;
        cudaEvent_t done = nullptr;
        float4* d_rays = nullptr;
        int32_t* d_tri = nullptr;
        float* d_t = nullptr;
        float2* d_uv = nullptr;
        unsigned long long* d_ctr = nullptr;
        int2* d_rlist = nullptr;
        void* h_in = nullptr;   // pinned staging for pageable caller buffers
        void* h_out = nullptr;
    } lanes[kHostLanes];
    int64_t lane_cap = 0;  // rays per chunk the lanes were allocated for
    // per-launch timing of k_trace in gsp_trace_closest_hit (gsp_trace_time_launches): event
    // pairs made up front, the first `tev_used` of them recorded
    std::vector<cudaEvent_t> tev;
    int64_t tev_used = 0;
};

// Installs a BVH built elsewhere (host copies + device arrays the scene takes ownership of),
// replacing the scene's current one.
void gsp_scene_adopt_bvh(gsp_scene* s, HostBVH&& bvh, float4* d_nodes, float4* d_tris, float4* d_bin);

// NVTX range around a host-side stage (header-only NVTX3: a no-op unless a profiler attaches).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

void gsp_set_last_error(const std::string& msg);

// Reports a CUDA failure of the library's own work: sets the message, consumes the runtime's
// last error (so that the next call does not see it as left over by the caller) and maps it to
// GSP_ERR_OOM or GSP_ERR_CUDA.
gsp_status gsp_cuda_fail(cudaError_t e);

// An error that the caller's earlier CUDA work left pending on this thread (the runtime's last
// error, shared with every user of the same CUDA runtime): reported as GSP_ERR_CUDA before the call
// touches anything, rather than discarded or returned later as a failure of the call's own launches.
// The library's failure paths consume the errors they report, so a pending error is never its own.
gsp_status gsp_pending_error(const char* who, cudaError_t e);

#define GSP_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return gsp_cuda_fail(e_);     \
    } while (0)

#define GSP_NO_PENDING_ERROR(who)                                        \
    do {                                                                 \
        const cudaError_t p_ = cudaGetLastError();                       \
        if (p_ != cudaSuccess) return gsp_pending_error((who), p_);      \
    } while (0)
