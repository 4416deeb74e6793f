// capi.cu -- context, scene, BVH and closest-hit entry points of the C ABI (include/gsp.h).
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "devcommon.cuh"
#include "gsp_internal.h"
#include "launch.h"
#include "persist.cuh"

namespace {
thread_local std::string g_last_error;
}

void gsp_set_last_error(const std::string& msg) { g_last_error = msg; }

gsp_status gsp_cuda_fail(cudaError_t e) {
    gsp_set_last_error(cudaGetErrorString(e));
    (void)cudaGetLastError();  // reported here; a sticky error stays and fails every later call
    return e == cudaErrorMemoryAllocation ? GSP_ERR_OOM : GSP_ERR_CUDA;
}

gsp_status gsp_pending_error(const char* who, cudaError_t e) {
    gsp_set_last_error(std::string(who) + ": a CUDA error was pending before the call (left by earlier CUDA work "
                       "on this thread): " + cudaGetErrorString(e));
    return GSP_ERR_CUDA;
}

namespace gspd {

// Closest-hit kernel (Fig. 3), persistent. A warp takes chunks of kTraceChunk consecutive rays
// and hands them to its lanes (WarpQueue); a lane whose ray has finished takes the next ray of
// the chunk right away, so lanes do not idle until the slowest ray of a batch ends. Lanes run up
// to kTraceInner traversal steps between refills. Rays and results are streamed with evict-first
// hints so that the BVH stays resident in L2. Hits whose FP32 t may be inaccurate are appended
// to a list that k_refine re-evaluates in FP64 with full warps.
// ctr[0] = next ray, ctr[1] = refine-list length.
__global__ void __launch_bounds__(kTraceThreads, GSP_TRACE_MIN_BLOCKS)
k_trace(DevScene S, const float4* __restrict__ rays, int64_t n, const uint32_t* __restrict__ d_n,
        int32_t* __restrict__ tri, float* __restrict__ tout, float2* __restrict__ uv,
        unsigned long long* __restrict__ ctr, int2* __restrict__ rlist, float refine_factor, int32_t out_slot) {
    if (d_n) n = min(n, (int64_t)*d_n);  // wavefront queues: the length lives on the device
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    const int32_t cap = trav_cap(S);
    Trav st;
    st.node = -1;
    st.slot = -1;
    WarpQueue<> wq;
    wq.init((int32_t)n);  // ray indices fit in 31 bits (the entry point rejects larger batches)
    int32_t ray = -1;
    int32_t pend = -1;  // leaf word of a postponed leaf, -1 = none
    uint32_t ntri = 0;  // not reported by this kernel
    while (true) {
        const int32_t got = wq.take(ray < 0, ctr);
        if (got >= 0) {
            ray = got;
            const float4 a = __ldcs(rays + 2 * (int64_t)ray), b = __ldcs(rays + 2 * (int64_t)ray + 1);
            trav_init(S, f3(a), f3(b), a.w, b.w, st);
        }
        if (__ballot_sync(0xffffffffu, ray >= 0) == 0) break;
        trav_steps(S, st, pend, ray >= 0, cap, ntri);
        const bool fin = ray >= 0 && st.node < 0 && pend < 0;
        bool flag = false;
        if (fin) {
            float u = 0.0f, v = 0.0f;
            if (st.slot >= 0)
                flag = hit_needs_refine(S.tris + 3 * st.slot, st.o, st.d, st.tbest, refine_factor, uv != nullptr, u, v);
            __stcs(tri + ray, out_slot ? st.slot : st.best);
            __stcs(tout + ray, st.best >= 0 ? st.tbest : __int_as_float(0x7f800000));
            if (uv) __stcs(uv + ray, make_float2(u, v));
        }
        const uint32_t fm = __ballot_sync(0xffffffffu, flag);
        if (fm) {
            const int leader = __ffs(fm) - 1;
            unsigned long long b = 0;
            if (lane == leader) b = atomicAdd(ctr + 1, (unsigned long long)__popc(fm));
            b = __shfl_sync(0xffffffffu, b, leader);
            if (flag) rlist[b + __popc(fm & lt)] = make_int2((int)ray, st.slot);
        }
        if (fin) ray = -1;
        if (wq.done) {  // no rays left to take: a ray left alone in the warp is walked by all lanes
            const uint32_t act = __ballot_sync(0xffffffffu, ray >= 0);
            if (act && !(act & (act - 1))) {
                st = coop_walk(S.tris, S.nnodes, S.status, st, pend, __ffs(act) - 1, cap).st;
                pend = -1;
            }
        }
    }
}

// Closest hit by stack-based near-first traversal of the same tree in its child-pair layout
// (StackWalk), the kind of traversal the paper measures the multiple-threaded BVH against
// (Fig. 4; the stack-based kernels of Aila & Laine 2009), with the same work distribution, leaf
// test, output and FP64 refinement list as k_trace.
__global__ void __launch_bounds__(kTraceThreads, GSP_TRACE_MIN_BLOCKS)
k_trace_stack(DevScene S, const float4* __restrict__ rays, int64_t n, int32_t* __restrict__ tri,
              float* __restrict__ tout, float2* __restrict__ uv, unsigned long long* __restrict__ ctr,
              int2* __restrict__ rlist, float refine_factor) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    WarpQueue<> wq;
    wq.init((int32_t)n);
    Trav st;
    st.slot = -1;
    const int32_t cap = trav_cap(S);
    int32_t ray = -1;
    StackWalk w;
    w.node = kWalkDone;
    w.sp = 0;
    while (true) {
        const int32_t got = wq.take(ray < 0, ctr);
        if (got >= 0) {
            ray = got;
            const float4 a = __ldcs(rays + 2 * (int64_t)ray), b = __ldcs(rays + 2 * (int64_t)ray + 1);
            trav_init(S, f3(a), f3(b), a.w, b.w, st);
            stack_init(S, w);
        }
        if (__ballot_sync(0xffffffffu, ray >= 0) == 0) break;
        stack_steps(S, st, w, ray >= 0, cap);
        const bool fin = ray >= 0 && w.node == kWalkDone;
        bool flag = false;
        if (fin) {
            float u = 0.0f, v = 0.0f;
            if (st.slot >= 0)
                flag = hit_needs_refine(S.tris + 3 * st.slot, st.o, st.d, st.tbest, refine_factor, uv != nullptr, u, v);
            __stcs(tri + ray, st.best);
            __stcs(tout + ray, st.best >= 0 ? st.tbest : __int_as_float(0x7f800000));
            if (uv) __stcs(uv + ray, make_float2(u, v));
        }
        const uint32_t fm = __ballot_sync(0xffffffffu, flag);
        if (fm) {
            const int leader = __ffs(fm) - 1;
            unsigned long long b = 0;
            if (lane == leader) b = atomicAdd(ctr + 1, (unsigned long long)__popc(fm));
            b = __shfl_sync(0xffffffffu, b, leader);
            if (flag) rlist[b + __popc(fm & lt)] = make_int2((int)ray, st.slot);
        }
        if (fin) ray = -1;
    }
}

// FP64 re-evaluation of the listed hits (their rays are rare; full warps keep the FP64 pipe busy).
__global__ void __launch_bounds__(256)
k_refine(DevScene S, const float4* __restrict__ rays, const int2* __restrict__ rlist,
         const unsigned long long* __restrict__ ctr, float* __restrict__ tout, float2* __restrict__ uv) {
    const int64_t cnt = (int64_t)ctr[1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const int2 e = rlist[i];
        const float4 a = __ldg(rays + 2 * (int64_t)e.x), b = __ldg(rays + 2 * (int64_t)e.x + 1);
        Hit h;
        h.t = tout[e.x];
        h.u = h.v = 0.0f;
        h.id = 0;
        if (refine_hit(S.tris + 3 * (int64_t)e.y, f3(a), f3(b), h)) {
            tout[e.x] = h.t;
            if (uv) uv[e.x] = make_float2(h.u, h.v);
        }
    }
}

__global__ void k_zero_u64x2(unsigned long long* p) {
    p[0] = 0ull;
    p[1] = 0ull;
}

__global__ void k_zero_u64(unsigned long long* p) { *p = 0ull; }

// out[k * ndraw + j] = draw j of stream (seed, scene, domain, pass, ids[k])
__global__ void k_rng_fill(uint64_t seed, uint32_t scene, uint32_t domain, uint32_t pass,
                           const uint64_t* __restrict__ ids, int64_t n, int32_t ndraw, float* __restrict__ out) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        Rng r = rng_seed(seed, scene, domain, pass, ids[k]);
        for (int32_t j = 0; j < ndraw; ++j) out[k * ndraw + j] = rng_next(r);
    }
}

}  // namespace gspd

int gsp_trace_grid(int device) {
    static int cached[64] = {0};
    if (device >= 0 && device < 64 && cached[device]) return cached[device];
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gspd::k_trace, kTraceThreads, 0);
    int g = std::max(1, sms) * std::max(1, per_sm);
    if (device >= 0 && device < 64) cached[device] = g;
    return g;
}

// One closest-hit call on device buffers: counters zeroed, k_trace, FP64 refinement of the
// flagged hits. ctr (2 u64) and rlist (n entries) belong to this call's stream.
// With e0 and e1 (gsp_trace_time_launches), the two events bracket the k_trace launch alone.
static void launch_trace(const gsp_scene* s, const float4* rays, int64_t n, int32_t* tri, float* t, float2* uv,
                         unsigned long long* ctr, int2* rlist, cudaStream_t st, cudaEvent_t e0 = nullptr,
                         cudaEvent_t e1 = nullptr) {
    NvtxRange nvtx("gsp: closest hit");
    const gspd::DevScene S = gsp_dev_scene(s);
    gspd::k_zero_u64x2<<<1, 1, 0, st>>>(ctr);
    const int grid = gsp_trace_grid(s->ctx->device);
    if (e0) cudaEventRecord(e0, st);
    gspd::k_trace<<<grid, kTraceThreads, 0, st>>>(S, rays, n, nullptr, tri, t, uv, ctr, rlist, GSP_REFINE_FACTOR, 0);
    if (e1) cudaEventRecord(e1, st);
    gspd::k_refine<<<std::max(1, grid / 2), 256, 0, st>>>(S, rays, rlist, ctr, t, uv);
}

cudaError_t gsp_trace_queue(const gsp_scene* s, const float4* rays, int64_t max_n, const uint32_t* d_n, int32_t* tri,
                            float* t, float refine_factor, bool zero_counters, bool out_slot, unsigned long long* ctr,
                            int2* rlist, cudaStream_t st) {
    const gspd::DevScene S = gsp_dev_scene(s);
    const int grid = gsp_trace_grid(s->ctx->device);
    const bool list = refine_factor < INFINITY;
    if (list || zero_counters) gspd::k_zero_u64x2<<<1, 1, 0, st>>>(ctr);
    gspd::k_trace<<<grid, kTraceThreads, 0, st>>>(S, rays, max_n, d_n, tri, t, nullptr, ctr, rlist, refine_factor,
                                                  out_slot ? 1 : 0);
    if (list) gspd::k_refine<<<std::max(1, grid / 2), 256, 0, st>>>(S, rays, rlist, ctr, t, nullptr);
    return cudaGetLastError();
}

gspd::DevScene gsp_dev_scene(const gsp_scene* s) {
    gspd::DevScene d;
    d.nodes = s->d_nodes;
    d.tris = s->d_tris;
    d.bin = s->d_bin;
    d.bin_root = s->bvh.bin_root;
    d.step_limit = s->step_limit;
    d.shade = s->d_shade;
    d.nlo = s->d_nlo;
    d.mats = s->d_mats;
    d.attr = s->d_attr;
    d.texels = s->d_texels;
    d.mtex = s->d_mtex;
    d.nnodes = s->bvh.nnodes;
    d.stride = s->bvh.stride;
    d.link_sets = s->bvh.link_sets;
    d.status = s->ctx->d_status;
    return d;
}

extern "C" {

const char* gsp_status_string(gsp_status s) {
    switch (s) {
        case GSP_OK: return "ok";
        case GSP_ERR_INVALID_ARG: return "invalid argument";
        case GSP_ERR_OOM: return "out of memory";
        case GSP_ERR_CUDA: return "CUDA runtime error";
        case GSP_ERR_TRAVERSAL_LIMIT: return "traversal exceeded its step limit (corrupt BVH links)";
        case GSP_ERR_TIMEOUT: return "bounded device wait timed out";
        case GSP_ERR_NOT_BUILT: return "scene has no BVH";
        case GSP_ERR_BAD_STATE: return "call order violated";
        case GSP_ERR_IO: return "checkpoint I/O failed";
        case GSP_ERR_OVERFLOW: return "device buffer overflow";
        default: return "unknown status";
    }
}

const char* gsp_last_error_message(void) { return g_last_error.c_str(); }

gsp_status gsp_context_create(int32_t device, gsp_context** out) {
    if (!out) return GSP_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    GSP_CUDA_TRY(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(device));
    gsp_context* c = new (std::nothrow) gsp_context;
    if (!c) return GSP_ERR_OOM;
    c->device = device;
    cudaError_t e = cudaMalloc(&c->d_status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int32_t));
    if (e != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return gsp_cuda_fail(e);
    }
    *out = c;
    return GSP_OK;
}

void gsp_context_destroy(gsp_context* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaFree(ctx->d_status);
    cudaFree(ctx->grid_scratch);
    delete ctx;
}

gsp_status gsp_context_sync(gsp_context* ctx) {
    if (!ctx) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(ctx->device));
    GSP_CUDA_TRY(cudaDeviceSynchronize());
    int32_t st = 0;
    GSP_CUDA_TRY(cudaMemcpy(&st, ctx->d_status, sizeof st, cudaMemcpyDeviceToHost));
    if (st != 0) GSP_CUDA_TRY(cudaMemset(ctx->d_status, 0, sizeof(int32_t)));
    return st;
}

static void trace_events_free(gsp_scene* s) {
    for (cudaEvent_t e : s->tev)
        if (e) cudaEventDestroy(e);
    s->tev.clear();
    s->tev_used = 0;
}

static void host_lanes_free(gsp_scene* s) {
    for (auto& L : s->lanes) {
        if (L.st) cudaStreamDestroy(L.st);
        if (L.done) cudaEventDestroy(L.done);
        cudaFree(L.d_rays);
        cudaFree(L.d_tri);
        cudaFree(L.d_t);
        cudaFree(L.d_uv);
        cudaFree(L.d_ctr);
        cudaFree(L.d_rlist);
        cudaFreeHost(L.h_in);
        cudaFreeHost(L.h_out);
        L = gsp_scene::HostLane{};
    }
    s->lane_cap = 0;
}

static void scene_free_bvh(gsp_scene* s) {
    cudaFree(s->d_nodes);
    cudaFree(s->d_tris);
    cudaFree(s->d_bin);
    s->d_nodes = nullptr;
    s->d_tris = nullptr;
    s->d_bin = nullptr;
    s->built = false;
}


void gsp_scene_destroy(gsp_scene* s) {
    if (!s) return;
    if (s->ctx) {
        cudaSetDevice(s->ctx->device);
        scene_free_bvh(s);
        trace_events_free(s);
        cudaFree(s->d_shade);
        cudaFree(s->d_nlo);
        cudaFree(s->d_mats);
        cudaFree(s->d_counter);
        cudaFree(s->d_rlist);
        cudaFree(s->d_attr);
        cudaFree(s->d_texels);
        cudaFree(s->d_mtex);
        host_lanes_free(s);
    }
    delete s;
}

gsp_status gsp_scene_upload(gsp_context* ctx, const float* verts, int64_t nv, const int32_t* tris,
                            int64_t nt, const int32_t* tri_mat, const gsp_material* mats,
                            int32_t nmat, const gsp_camera* cam, gsp_scene** out) {
    if (!verts || !tris || !mats || !out || nv <= 0 || nt <= 0 || nmat < 1 || nmat > 64)
        return GSP_ERR_INVALID_ARG;
    *out = nullptr;
    if (nt >= (int64_t(1) << 28) || nv >= (int64_t(1) << 31)) return GSP_ERR_INVALID_ARG;
    for (int64_t i = 0; i < 3 * nv; ++i)
        if (!std::isfinite(verts[i])) return GSP_ERR_INVALID_ARG;
    for (int64_t i = 0; i < 3 * nt; ++i)
        if (tris[i] < 0 || tris[i] >= nv) return GSP_ERR_INVALID_ARG;
    if (tri_mat)
        for (int64_t i = 0; i < nt; ++i)
            if (tri_mat[i] < 0 || tri_mat[i] >= nmat) return GSP_ERR_INVALID_ARG;
    for (int32_t m = 0; m < nmat; ++m) {
        if (mats[m].type < GSP_DIFFUSE || mats[m].type > GSP_EMITTER) return GSP_ERR_INVALID_ARG;
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(mats[m].albedo[k]) || !std::isfinite(mats[m].emission[k]) ||
                mats[m].emission[k] < 0.0f)
                return GSP_ERR_INVALID_ARG;
        if (mats[m].type == GSP_DIELECTRIC && !(mats[m].ior > 0.0f)) return GSP_ERR_INVALID_ARG;
    }
    if (cam && (cam->width <= 0 || cam->height <= 0 || !(cam->vfov_deg > 0.0f) ||
                !(cam->vfov_deg < 180.0f)))
        return GSP_ERR_INVALID_ARG;
    if (ctx) GSP_CUDA_TRY(cudaSetDevice(ctx->device));
    gsp_scene* s = new (std::nothrow) gsp_scene;
    if (!s) return GSP_ERR_OOM;
    s->ctx = ctx;
    s->nv = nv;
    s->nt = nt;
    s->nmat = nmat;
    s->verts.assign(verts, verts + 3 * nv);
    s->tris.assign(tris, tris + 3 * nt);
    s->tri_mat = tri_mat ? std::vector<int32_t>(tri_mat, tri_mat + nt) : std::vector<int32_t>(nt, 0);
    s->mats.assign(mats, mats + nmat);
    if (cam) { s->has_cam = true; s->cam = *cam; }
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nv; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], (double)verts[3 * i + k]);
            hi[k] = std::max(hi[k], (double)verts[3 * i + k]);
        }
    s->extent = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                          (hi[2] - lo[2]) * (hi[2] - lo[2]));
    // shading record per triangle: unit geometric normal (computed in FP64) + material
    std::vector<float4> shade(nt), nlo(nt);
    for (int64_t i = 0; i < nt; ++i) {
        const float* a = verts + 3 * (int64_t)tris[3 * i];
        const float* b = verts + 3 * (int64_t)tris[3 * i + 1];
        const float* c = verts + 3 * (int64_t)tris[3 * i + 2];
        double e1[3], e2[3];
        for (int k = 0; k < 3; ++k) { e1[k] = (double)b[k] - a[k]; e2[k] = (double)c[k] - a[k]; }
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        double il = len > 0 ? 1.0 / len : 0.0;
        int32_t m = s->tri_mat[i];
        float mf;
        std::memcpy(&mf, &m, 4);
        const double u[3] = {n[0] * il, n[1] * il, n[2] * il};
        shade[i] = float4{(float)u[0], (float)u[1], (float)u[2], mf};
        nlo[i] = float4{(float)(u[0] - (double)shade[i].x), (float)(u[1] - (double)shade[i].y),
                        (float)(u[2] - (double)shade[i].z), 0.0f};
    }
    std::vector<float4> mt(2 * nmat);
    for (int32_t m = 0; m < nmat; ++m) {
        float tf;
        std::memcpy(&tf, &mats[m].type, 4);
        mt[2 * m] = float4{mats[m].albedo[0], mats[m].albedo[1], mats[m].albedo[2], tf};
        mt[2 * m + 1] = float4{mats[m].emission[0], mats[m].emission[1], mats[m].emission[2], mats[m].ior};
    }
    if (!ctx) {  // host-only scene: BVH build, export and host walk only
        *out = s;
        return GSP_OK;
    }
    cudaError_t e = cudaMalloc(&s->d_shade, nt * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_nlo, nt * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_mats, 2 * nmat * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_counter, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(s->d_shade, shade.data(), nt * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_nlo, nlo.data(), nt * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->d_mats, mt.data(), 2 * nmat * sizeof(float4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        gsp_scene_destroy(s);
        return gsp_cuda_fail(e);
    }
    *out = s;
    return GSP_OK;
}

gsp_status gsp_scene_set_materials(gsp_scene* s, const gsp_material* mats, int32_t nmat) {
    if (!s || !mats || nmat != s->nmat) return GSP_ERR_INVALID_ARG;
    for (int32_t m = 0; m < nmat; ++m) {
        if (mats[m].type < GSP_DIFFUSE || mats[m].type > GSP_EMITTER) return GSP_ERR_INVALID_ARG;
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(mats[m].albedo[k]) || !std::isfinite(mats[m].emission[k]) || mats[m].emission[k] < 0.0f)
                return GSP_ERR_INVALID_ARG;
        if (mats[m].type == GSP_DIELECTRIC && !(mats[m].ior > 0.0f)) return GSP_ERR_INVALID_ARG;
    }
    s->mats.assign(mats, mats + nmat);
    if (!s->ctx) return GSP_OK;
    std::vector<float4> mt(2 * nmat);
    for (int32_t m = 0; m < nmat; ++m) {
        float tf;
        std::memcpy(&tf, &mats[m].type, 4);
        mt[2 * m] = float4{mats[m].albedo[0], mats[m].albedo[1], mats[m].albedo[2], tf};
        mt[2 * m + 1] = float4{mats[m].emission[0], mats[m].emission[1], mats[m].emission[2], mats[m].ior};
    }
    GSP_CUDA_TRY(cudaSetDevice(s->ctx->device));
    GSP_NO_PENDING_ERROR("gsp_scene_set_materials");
    GSP_CUDA_TRY(cudaMemcpy(s->d_mats, mt.data(), mt.size() * sizeof(float4), cudaMemcpyHostToDevice));
    return GSP_OK;
}

gsp_status gsp_scene_set_step_limit(gsp_scene* s, int32_t max_box_tests) {
    if (!s || max_box_tests < 0) return GSP_ERR_INVALID_ARG;
    s->step_limit = max_box_tests;
    return GSP_OK;
}

gsp_status gsp_scene_set_attributes(gsp_scene* s, const float* normals, const float* texcoords) {
    if (!s) return GSP_ERR_INVALID_ARG;
    const int64_t nv = s->nv, nt = s->nt;
    if (normals)
        for (int64_t v = 0; v < nv; ++v) {
            const float* n = normals + 3 * v;
            if (!std::isfinite(n[0]) || !std::isfinite(n[1]) || !std::isfinite(n[2]) ||
                (double)n[0] * n[0] + (double)n[1] * n[1] + (double)n[2] * n[2] == 0.0)
                return GSP_ERR_INVALID_ARG;
        }
    if (texcoords)
        for (int64_t i = 0; i < 2 * nv; ++i)
            if (!std::isfinite(texcoords[i])) return GSP_ERR_INVALID_ARG;
    if (!texcoords)
        for (const auto& t : s->tex)
            if (!t.empty()) {
                gsp_set_last_error("gsp_scene_set_attributes: remove the scene's textures before its texture coordinates");
                return GSP_ERR_BAD_STATE;
            }
    if (s->ctx) {  // a host-only scene has no device copy and makes no CUDA call
        GSP_CUDA_TRY(cudaSetDevice(s->ctx->device));
        GSP_NO_PENDING_ERROR("gsp_scene_set_attributes");
        cudaFree(s->d_attr);
        s->d_attr = nullptr;
    }
    s->has_texcoords = false;
    if (!normals && !texcoords) return GSP_OK;
    s->has_texcoords = texcoords != nullptr;
    if (!s->ctx) return GSP_OK;
    // gathered per triangle so that a hit reads its shading data with four aligned loads
    std::vector<float4> rec(4 * (size_t)nt);
    const int32_t flags = normals ? 1 : 0;
    float ff;
    std::memcpy(&ff, &flags, 4);
    for (int64_t i = 0; i < nt; ++i) {
        float t3[3];
        for (int k = 0; k < 3; ++k) {
            const int64_t v = s->tris[3 * i + k];
            const float* n = normals ? normals + 3 * v : nullptr;
            rec[4 * i + k] = float4{n ? n[0] : 0.0f, n ? n[1] : 0.0f, n ? n[2] : 0.0f, texcoords ? texcoords[2 * v] : 0.0f};
            t3[k] = texcoords ? texcoords[2 * v + 1] : 0.0f;
        }
        rec[4 * i + 3] = float4{t3[0], t3[1], t3[2], ff};
    }
    GSP_CUDA_TRY(cudaMalloc(&s->d_attr, rec.size() * sizeof(float4)));
    GSP_CUDA_TRY(cudaMemcpy(s->d_attr, rec.data(), rec.size() * sizeof(float4), cudaMemcpyHostToDevice));
    return GSP_OK;
}

gsp_status gsp_scene_set_texture(gsp_scene* s, int32_t material, const float* rgb, int32_t width, int32_t height) {
    if (!s || material < 0 || material >= s->nmat) return GSP_ERR_INVALID_ARG;
    if (rgb) {
        if (s->mats[material].type != GSP_DIFFUSE || width < 1 || height < 1 || width > 16384 || height > 16384 ||
            (int64_t)width * height > (int64_t(1) << 26))
            return GSP_ERR_INVALID_ARG;
        for (int64_t i = 0; i < 3 * (int64_t)width * height; ++i)
            if (!std::isfinite(rgb[i]) || rgb[i] < 0.0f) return GSP_ERR_INVALID_ARG;
        if (!s->has_texcoords) {
            gsp_set_last_error("gsp_scene_set_texture: the scene has no texture coordinates (gsp_scene_set_attributes)");
            return GSP_ERR_BAD_STATE;
        }
        int64_t others = 0;  // texel offsets are int32
        for (int32_t m = 0; m < (int32_t)s->tex.size(); ++m)
            if (m != material) others += (int64_t)s->tex[m].size();
        if (others + (int64_t)width * height > INT32_MAX) return GSP_ERR_INVALID_ARG;
    }
    s->tex.resize(s->nmat);
    s->tex_size.resize(s->nmat, int2{0, 0});
    std::vector<float4>& t = s->tex[material];
    t.clear();
    s->tex_size[material] = int2{0, 0};
    if (rgb) {
        t.resize((size_t)width * height);
        for (size_t i = 0; i < t.size(); ++i) t[i] = float4{rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], 0.0f};
        s->tex_size[material] = int2{width, height};
    }
    if (!s->ctx) return GSP_OK;
    GSP_CUDA_TRY(cudaSetDevice(s->ctx->device));
    GSP_NO_PENDING_ERROR("gsp_scene_set_texture");
    cudaFree(s->d_texels);
    cudaFree(s->d_mtex);
    s->d_texels = nullptr;
    s->d_mtex = nullptr;
    int64_t total = 0;
    std::vector<int4> mt(s->nmat, int4{0, 0, 0, 0});
    for (int32_t m = 0; m < s->nmat; ++m) {
        mt[m] = int4{(int32_t)total, s->tex_size[m].x, s->tex_size[m].y, 0};
        total += (int64_t)s->tex[m].size();
    }
    if (total == 0) return GSP_OK;  // no material has a texture: kernels skip the lookup
    GSP_CUDA_TRY(cudaMalloc(&s->d_texels, total * sizeof(float4)));
    GSP_CUDA_TRY(cudaMalloc(&s->d_mtex, mt.size() * sizeof(int4)));
    for (int32_t m = 0; m < s->nmat; ++m)
        if (!s->tex[m].empty())
            GSP_CUDA_TRY(cudaMemcpy(s->d_texels + mt[m].x, s->tex[m].data(), s->tex[m].size() * sizeof(float4),
                                    cudaMemcpyHostToDevice));
    GSP_CUDA_TRY(cudaMemcpy(s->d_mtex, mt.data(), mt.size() * sizeof(int4), cudaMemcpyHostToDevice));
    return GSP_OK;
}

gsp_status gsp_build_bvh(gsp_scene* s, const gsp_bvh_params* params, gsp_bvh_stats* stats) {
    if (!s) return GSP_ERR_INVALID_ARG;
    gsp_bvh_params p{16, 4, 7, 6};
    if (params) p = *params;
    if (p.bins < 2 || p.bins > 64 || p.max_leaf < 1 || p.max_leaf > 7 || p.leaf_threshold < 1 ||
        p.leaf_threshold > p.max_leaf || (p.link_sets != 1 && p.link_sets != 6))
        return GSP_ERR_INVALID_ARG;
    HostBVH bvh;
    NvtxRange nvtx("gsp: host SAH build + threading");
    std::string err = bvh_build_host(s->verts.data(), s->nv, s->tris.data(), s->nt, p, bvh);
    if (!err.empty()) {
        gsp_set_last_error(err);
        return GSP_ERR_INVALID_ARG;
    }
    size_t nb = bvh.nodes.size() * sizeof(float4), tb = bvh.tris.size() * sizeof(float4);
    const size_t bb = std::max<size_t>(1, bvh.bin.size()) * sizeof(float4);
    if (s->ctx) {
        GSP_CUDA_TRY(cudaSetDevice(s->ctx->device));
        scene_free_bvh(s);
        GSP_CUDA_TRY(cudaMalloc(&s->d_nodes, nb));
        GSP_CUDA_TRY(cudaMalloc(&s->d_tris, tb));
        GSP_CUDA_TRY(cudaMemcpy(s->d_nodes, bvh.nodes.data(), nb, cudaMemcpyHostToDevice));
        GSP_CUDA_TRY(cudaMemcpy(s->d_tris, bvh.tris.data(), tb, cudaMemcpyHostToDevice));
        GSP_CUDA_TRY(cudaMalloc(&s->d_bin, bb));
        if (!bvh.bin.empty())
            GSP_CUDA_TRY(cudaMemcpy(s->d_bin, bvh.bin.data(), bvh.bin.size() * sizeof(float4), cudaMemcpyHostToDevice));
    }
    s->bvh = std::move(bvh);
    s->built = true;
    s->device_bytes = (int64_t)(nb + tb) + s->nt * (int64_t)sizeof(float4);  // MTBVH + triangles + shading
    if (stats) {
        stats->nodes = s->bvh.nnodes;
        stats->leaves = s->bvh.nleaves;
        stats->depth = s->bvh.depth;
        stats->link_sets = s->bvh.link_sets;
        stats->build_ms = s->bvh.build_ms;
        stats->thread_ms = s->bvh.thread_ms;
        stats->device_bytes = s->device_bytes;
    }
    return GSP_OK;
}

gsp_status gsp_trace_closest_hit(gsp_scene* s, const float* d_rays, int64_t n, int32_t* d_tri,
                                 float* d_t, float* d_uv, void* stream) {
    if (!s || n < 0) return GSP_ERR_INVALID_ARG;
    if (!s->ctx) return GSP_ERR_INVALID_ARG;  // host-only scene
    if (!s->built) return GSP_ERR_NOT_BUILT;
    if (n == 0) return GSP_OK;
    if (!d_rays || !d_tri || !d_t || n > INT32_MAX) return GSP_ERR_INVALID_ARG;
    if (((uintptr_t)d_rays & 15) || ((uintptr_t)d_uv & 7)) return GSP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    GSP_CUDA_TRY(cudaSetDevice(s->ctx->device));
    GSP_NO_PENDING_ERROR("gsp_trace_closest_hit");
    if (n > s->rlist_cap) {  // refine list sized for the largest batch seen (worst case: every ray)
        GSP_CUDA_TRY(cudaStreamSynchronize(st));
        cudaFree(s->d_rlist);
        s->d_rlist = nullptr;
        s->rlist_cap = 0;
        GSP_CUDA_TRY(cudaMalloc(&s->d_rlist, (size_t)n * sizeof(int2)));
        s->rlist_cap = n;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (2 * s->tev_used < (int64_t)s->tev.size()) {
        e0 = s->tev[2 * s->tev_used];
        e1 = s->tev[2 * s->tev_used + 1];
        ++s->tev_used;
    }
    launch_trace(s, (const float4*)d_rays, n, d_tri, d_t, (float2*)d_uv, s->d_counter, s->d_rlist, st, e0, e1);
    GSP_CUDA_TRY(cudaGetLastError());
    return GSP_OK;
}

gsp_status gsp_trace_time_launches(gsp_scene* s, int64_t n) {
    if (!s || !s->ctx || n < 0 || n > (int64_t(1) << 20)) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(s->ctx->device));
    GSP_NO_PENDING_ERROR("gsp_trace_time_launches");
    trace_events_free(s);
    s->tev.assign((size_t)(2 * n), nullptr);
    for (cudaEvent_t& e : s->tev) {
        const cudaError_t ce = cudaEventCreate(&e);
        if (ce != cudaSuccess) {
            trace_events_free(s);
            return gsp_cuda_fail(ce);
        }
    }
    return GSP_OK;
}

gsp_status gsp_trace_launch_times(gsp_scene* s, float* h_ms, int64_t capacity, int64_t* count) {
    if (!s || !s->ctx || capacity < 0 || (capacity > 0 && !h_ms) || !count) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(s->ctx->device));
    const int64_t m = s->tev_used;
    for (int64_t i = 0; i < std::min(m, capacity); ++i) {
        GSP_CUDA_TRY(cudaEventSynchronize(s->tev[2 * i + 1]));
        GSP_CUDA_TRY(cudaEventElapsedTime(&h_ms[i], s->tev[2 * i], s->tev[2 * i + 1]));
    }
    *count = m;
    s->tev_used = 0;
    return GSP_OK;
}

#ifndef GSP_HOST_CHUNK
#define GSP_HOST_CHUNK (1 << 20)  // rays per chunk of the staged pipeline
#endif

// (Re)allocates the host-tracing lanes for `cap` rays each; the ray and staging buffers only when
// `staged` (the mapped path reads the caller's rays in place).
static gsp_status host_lanes_reserve(gsp_scene* s, int64_t cap, bool staged) {
    const bool have_in = s->lanes[0].d_rays != nullptr;
    if (s->lane_cap >= cap && (!staged || have_in)) return GSP_OK;
    cap = std::max(cap, s->lane_cap);
    GSP_CUDA_TRY(cudaDeviceSynchronize());
    host_lanes_free(s);
    for (auto& L : s->lanes) {
        GSP_CUDA_TRY(cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking));
        GSP_CUDA_TRY(cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming));
        if (staged || have_in) {
            GSP_CUDA_TRY(cudaMalloc(&L.d_rays, (size_t)cap * 2 * sizeof(float4)));
            GSP_CUDA_TRY(cudaMallocHost(&L.h_in, (size_t)cap * 32));
            GSP_CUDA_TRY(cudaMallocHost(&L.h_out, (size_t)cap * 16));
        }
        GSP_CUDA_TRY(cudaMalloc(&L.d_tri, (size_t)cap * sizeof(int32_t)));
        GSP_CUDA_TRY(cudaMalloc(&L.d_t, (size_t)cap * sizeof(float)));
        GSP_CUDA_TRY(cudaMalloc(&L.d_uv, (size_t)cap * sizeof(float2)));
        GSP_CUDA_TRY(cudaMalloc(&L.d_ctr, 2 * sizeof(unsigned long long)));
        GSP_CUDA_TRY(cudaMalloc(&L.d_rlist, (size_t)cap * sizeof(int2)));
    }
    s->lane_cap = cap;
    return GSP_OK;
}

// Closest hits for host buffers. Page-locked buffers that the device can address: the rays are
// split in two halves on two streams; k_trace reads each half's rays from host memory itself (the
// transfer spreads over the traversal) and writes the hits to device buffers, which are copied
// back while the other half is traced. Measured alternatives were slower on GB300 (4,194,304
// rays): the traversal also writing its 4-byte results to host memory (3,390 Mrays/s against
// 3,560 for one part), a copy of the rays before the traversal (2,640), copy-engine pipelines
// of 2^17-2^20-ray chunks (1,240-2,940), and copying 50-100 % of the rays by copy engine while
// the rest is traced in place (3,000-3,230). Other buffers: chunks through page-locked
// staging buffers on three streams, the host filling and draining them while the device works
// on other chunks.
gsp_status gsp_trace_closest_hit_host(gsp_scene* s, const float* h_rays, int64_t n, int32_t* h_tri, float* h_t,
                                      float* h_uv) {
    if (!s || n < 0) return GSP_ERR_INVALID_ARG;
    if (!s->ctx) return GSP_ERR_INVALID_ARG;
    if (!s->built) return GSP_ERR_NOT_BUILT;
    if (n == 0) return GSP_OK;
    if (!h_rays || !h_tri || !h_t || n > INT32_MAX) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(s->ctx->device));
    GSP_NO_PENDING_ERROR("gsp_trace_closest_hit_host");
    // page-locked host memory that the device can address directly (NULL if it cannot)
    auto mapped = [](const void* p) -> const void* {
        cudaPointerAttributes a{};
        if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
    };
    const float4* m_rays = (const float4*)mapped(h_rays);
    if (m_rays && !((uintptr_t)m_rays & 15) && mapped(h_tri) && mapped(h_t) && (!h_uv || mapped(h_uv))) {
        constexpr int kParts = 2;
        const int64_t per = (n + kParts - 1) / kParts;
        gsp_status e = host_lanes_reserve(s, per, false);
        if (e != GSP_OK) return e;
        for (int k = 0; k < kParts; ++k) {
            const int64_t off = k * per, m = std::min(per, n - off);
            if (m <= 0) break;
            auto& L = s->lanes[k];
            launch_trace(s, m_rays + 2 * off, m, L.d_tri, L.d_t, h_uv ? L.d_uv : nullptr, L.d_ctr, L.d_rlist, L.st);
            GSP_CUDA_TRY(cudaMemcpyAsync(h_tri + off, L.d_tri, (size_t)m * 4, cudaMemcpyDeviceToHost, L.st));
            GSP_CUDA_TRY(cudaMemcpyAsync(h_t + off, L.d_t, (size_t)m * 4, cudaMemcpyDeviceToHost, L.st));
            if (h_uv)
                GSP_CUDA_TRY(cudaMemcpyAsync(h_uv + 2 * off, L.d_uv, (size_t)m * 8, cudaMemcpyDeviceToHost, L.st));
        }
        for (int k = 0; k < kParts; ++k) GSP_CUDA_TRY(cudaStreamSynchronize(s->lanes[k].st));
        GSP_CUDA_TRY(cudaGetLastError());
        return GSP_OK;
    }
    const int64_t chunk = std::min<int64_t>(GSP_HOST_CHUNK, n);
    gsp_status e = host_lanes_reserve(s, chunk, true);
    if (e != GSP_OK) return e;
    const int64_t cap = s->lane_cap;
    const int64_t nchunks = (n + chunk - 1) / chunk;
    std::vector<int64_t> pending(gsp_scene::kHostLanes, -1);  // chunk whose results wait in staging
    auto drain = [&](int k) -> cudaError_t {                    // copy a staged chunk's results out
        if (pending[k] < 0) return cudaSuccess;
        cudaError_t ce = cudaEventSynchronize(s->lanes[k].done);
        if (ce != cudaSuccess) return ce;
        const int64_t off = pending[k] * chunk, m = std::min(chunk, n - off);
        const char* o = (const char*)s->lanes[k].h_out;
        std::memcpy(h_tri + off, o, (size_t)m * 4);
        std::memcpy(h_t + off, o + (size_t)cap * 4, (size_t)m * 4);
        if (h_uv) std::memcpy(h_uv + 2 * off, o + (size_t)cap * 8, (size_t)m * 8);
        pending[k] = -1;
        return cudaSuccess;
    };
    for (int64_t c = 0; c < nchunks; ++c) {
        const int k = (int)(c % gsp_scene::kHostLanes);
        auto& L = s->lanes[k];
        const int64_t off = c * chunk, m = std::min(chunk, n - off);
        GSP_CUDA_TRY(drain(k));  // the lane's staging buffers are free again
        GSP_CUDA_TRY(cudaEventSynchronize(L.done));
        std::memcpy(L.h_in, h_rays + off * 8, (size_t)m * 32);
        GSP_CUDA_TRY(cudaMemcpyAsync(L.d_rays, L.h_in, (size_t)m * 32, cudaMemcpyHostToDevice, L.st));
        launch_trace(s, L.d_rays, m, L.d_tri, L.d_t, h_uv ? L.d_uv : nullptr, L.d_ctr, L.d_rlist, L.st);
        char* o = (char*)L.h_out;
        GSP_CUDA_TRY(cudaMemcpyAsync(o, L.d_tri, (size_t)m * 4, cudaMemcpyDeviceToHost, L.st));
        GSP_CUDA_TRY(cudaMemcpyAsync(o + (size_t)cap * 4, L.d_t, (size_t)m * 4, cudaMemcpyDeviceToHost, L.st));
        if (h_uv) GSP_CUDA_TRY(cudaMemcpyAsync(o + (size_t)cap * 8, L.d_uv, (size_t)m * 8, cudaMemcpyDeviceToHost, L.st));
        pending[k] = c;
        GSP_CUDA_TRY(cudaEventRecord(L.done, L.st));
    }
    for (int k = 0; k < gsp_scene::kHostLanes; ++k) {
        GSP_CUDA_TRY(drain(k));
        GSP_CUDA_TRY(cudaStreamSynchronize(s->lanes[k].st));
    }
    GSP_CUDA_TRY(cudaGetLastError());
    return GSP_OK;
}

gsp_status gsp_trace_closest_hit_stack(gsp_scene* s, const float* d_rays, int64_t n, int32_t* d_tri,
                                 float* d_t, float* d_uv, void* stream) {
    if (!s || n < 0) return GSP_ERR_INVALID_ARG;
    if (!s->ctx) return GSP_ERR_INVALID_ARG;  // host-only scene
    if (!s->built) return GSP_ERR_NOT_BUILT;
    if (s->bvh.depth >= gspd::kStackDepth) {
        gsp_set_last_error("gsp_trace_closest_hit_stack: the tree is deeper than the traversal stack (64)");
        return GSP_ERR_INVALID_ARG;
    }
    if (n == 0) return GSP_OK;
    if (!d_rays || !d_tri || !d_t || n > INT32_MAX) return GSP_ERR_INVALID_ARG;
    if (((uintptr_t)d_rays & 15) || ((uintptr_t)d_uv & 7)) return GSP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    GSP_CUDA_TRY(cudaSetDevice(s->ctx->device));
    GSP_NO_PENDING_ERROR("gsp_trace_closest_hit_stack");
    if (n > s->rlist_cap) {  // refine list sized for the largest batch seen (worst case: every ray)
        GSP_CUDA_TRY(cudaStreamSynchronize(st));
        cudaFree(s->d_rlist);
        s->d_rlist = nullptr;
        s->rlist_cap = 0;
        GSP_CUDA_TRY(cudaMalloc(&s->d_rlist, (size_t)n * sizeof(int2)));
        s->rlist_cap = n;
    }
    const gspd::DevScene S = gsp_dev_scene(s);
    gspd::k_zero_u64x2<<<1, 1, 0, st>>>(s->d_counter);
    const int grid = gsp_trace_grid(s->ctx->device);
    gspd::k_trace_stack<<<grid, kTraceThreads, 0, st>>>(S, (const float4*)d_rays, n, d_tri, d_t, (float2*)d_uv,
                                                        s->d_counter, s->d_rlist, GSP_REFINE_FACTOR);
    gspd::k_refine<<<std::max(1, grid / 2), 256, 0, st>>>(S, (const float4*)d_rays, s->d_rlist, s->d_counter, d_t,
                                                          (float2*)d_uv);
    GSP_CUDA_TRY(cudaGetLastError());
    return GSP_OK;
}

gsp_status gsp_rng_fill(gsp_context* ctx, uint64_t seed, uint32_t scene, uint32_t domain, uint32_t pass,
                        const uint64_t* d_ids, int64_t n, int32_t ndraw, float* d_out, void* stream) {
    if (!ctx || n < 0 || ndraw < 0 || (n > 0 && (!d_ids || !d_out))) return GSP_ERR_INVALID_ARG;
    if (n == 0 || ndraw == 0) return GSP_OK;
    GSP_CUDA_TRY(cudaSetDevice(ctx->device));
    GSP_NO_PENDING_ERROR("gsp_rng_fill");
    const int64_t nb = std::min<int64_t>((n + 255) / 256, 65535);
    gspd::k_rng_fill<<<(unsigned)nb, 256, 0, (cudaStream_t)stream>>>(seed, scene, domain, pass, d_ids, n, ndraw, d_out);
    GSP_CUDA_TRY(cudaGetLastError());
    return GSP_OK;
}

gsp_status gsp_bvh_host_walk(gsp_scene* s, const float* h_rays, int64_t n, int32_t* h_tri,
                             float* h_t, int32_t* h_visits, int32_t* h_tests) {
    if (!s || n < 0 || (n > 0 && !h_rays)) return GSP_ERR_INVALID_ARG;
    if (!s->built) return GSP_ERR_NOT_BUILT;
    bvh_host_walk(s->bvh, h_rays, n, h_tri, h_t, h_visits, h_tests);
    return GSP_OK;
}

gsp_status gsp_bvh_export(gsp_scene* s, int32_t set, float* h_nodes, float* h_tris, int64_t* nodes_out) {
    if (!s) return GSP_ERR_INVALID_ARG;
    if (!s->built) return GSP_ERR_NOT_BUILT;
    if (set < 0 || set >= s->bvh.link_sets) return GSP_ERR_INVALID_ARG;
    if (nodes_out) *nodes_out = s->bvh.nnodes;
    if (h_nodes)
        std::memcpy(h_nodes, s->bvh.nodes.data() + (size_t)set * s->bvh.stride * 2,
                    s->bvh.nnodes * 2 * sizeof(float4));
    if (h_tris) std::memcpy(h_tris, s->bvh.tris.data(), s->bvh.tris.size() * sizeof(float4));
    return GSP_OK;
}

}  // extern "C"

void gsp_scene_adopt_bvh(gsp_scene* s, HostBVH&& bvh, float4* d_nodes, float4* d_tris, float4* d_bin) {
    scene_free_bvh(s);
    s->d_nodes = d_nodes;
    s->d_tris = d_tris;
    s->d_bin = d_bin;
    s->device_bytes = (int64_t)((bvh.nodes.size() + bvh.tris.size()) * sizeof(float4)) + s->nt * (int64_t)sizeof(float4);
    s->bvh = std::move(bvh);
    s->built = true;
}
