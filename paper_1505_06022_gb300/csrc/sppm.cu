// sppm.cu -- stochastic progressive photon mapping on the device (Sec. 2, 3.3, 3.4): the host
// side (renderer state, pass orchestration, gradient replay, batches, autotuners, checkpoints).
// The kernels are in sppm_paths.cuh (eye and photon passes, path kernels) and sppm_gather.cuh
// (deposit, gather and progressive update, adjoint).
//
// One pass = eye pass (first non-specular hit per pixel; emission seen directly is recorded as
// the pass's direct term), photon pass (whole paths, or one bounce per thread with path
// regeneration), hash-grid deposit, and the fused range query + progressive update (which also
// folds the pass's direct term into the pixel state). The eye and photon passes are emission
// kernels, optional wavefront steps, and one persistent path kernel (k_paths; k_paths_multi for
// a batch of renderers); several passes overlap on three streams (passes_overlapped: two
// tracing streams, one per trace set, and the caller's stream for the deposits and gathers).
//
// Device layout (all library-owned, sized at creation):
//   pixel state   st0[p] = {tau.rgb, N}, st1[p] = {direct.rgb, R}          32 B / pixel
//   trace sets    two (both made at creation), each:
//     hit points  hx[p] = {x.xyz, material or -1}, hn[p] = {n_s.xyz, 0},
//                 hf[p] = {w * albedo / pi, 0}, hd[p] = {direct.rgb, 0}     64 B / pixel
//     photons     slot s: {x.xyz, id}, {flux.rgb, octahedral direction}    32 B / deposit
//                 path k owns slots [k*32, k*32+32) (one slot per thread in REGEN mode)
//     queues      eye and photon wavefront queues, two of each (ping-pong), their lengths,
//                 the path kernel's work counter, the wavefront steps' trace counters
//   exact grid    bucket-sorted SoA copies spos[], spay[] + bucket starts bstart[T+1]
//   stochastic    entry[T] = min(random depth bits << 32 | slot), ecount[T], one table per trace set
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "devcommon.cuh"
#include "gsp_internal.h"
#include "launch.h"
#include "persist.cuh"
#include "scan_sort.h"
#include "sppm_gather.cuh"
#include "sppm_paths.cuh"

// ============================================================================================
// host side
// ============================================================================================
using namespace gspd;

int64_t gsp_grid_scratch_words(int64_t n, int64_t T);
gsp_status gsp_grid_build_with(const float4* pos, int64_t n, float cell_h, int64_t T, uint32_t* order,
                               uint32_t* bstart, uint32_t* scratch, cudaStream_t st, bool skip_invalid);

static_assert(kWorkCounts == GSP_WORK_COUNTS && kWorkEyeRays == GSP_WORK_EYE_RAYS &&
                  kWorkPhotonRays == GSP_WORK_PHOTON_RAYS && kWorkNodes == GSP_WORK_NODE_VISITS &&
                  kWorkTris == GSP_WORK_TRI_TESTS && kWorkDeposits == GSP_WORK_DEPOSITS &&
                  kWorkHits == GSP_WORK_HIT_POINTS && kWorkScanned == GSP_WORK_PHOTONS_SCANNED &&
                  kWorkHitsScanned == GSP_WORK_HIT_POINTS_SCANNED,
              "the work counters of the kernels are the ones gsp.h names");

struct gsp_sppm {
    gsp_scene* scene = nullptr;
    gsp_sppm_params P{};
    int32_t w = 0, h = 0;
    int64_t npix = 0, np = 0, T = 0, slot_cap = 0;
    int32_t tbits = 0, slots_per_path = 0;
    float inv_h = 0;
    CamDev cam{};
    int32_t nemit = 0;
    float4* d_emit = nullptr;
    float* d_cdf = nullptr;
    float4 *st0 = nullptr, *st1 = nullptr;
    // The tracing of a pass: its path queues and counters, and the outputs its deposit and gather
    // read. Two sets, so that the tracing of pass i + 1 runs while pass i is gathered and while
    // the longest paths of pass i are still being traced (gsp_sppm_pass with several passes);
    // both sets are made at creation in exact mode (else on first use). hx .. rlist alias the set
    // in use.
    struct TraceBuf {
        float4 *hx = nullptr, *hn = nullptr, *hf = nullptr, *hd = nullptr, *slots = nullptr;
        uint32_t* pcount = nullptr;
        float4* hw = nullptr;     // gradient replay: eye throughput per hit point
        int32_t* smat = nullptr;  // gradient replay: material under each deposit
        PathQ q[2]{};             // photon wavefront queues, ping-pong (np entries; full paths only)
        PathQ qe[2]{};            // eye wavefront queues (npix entries)
        uint32_t* qctr = nullptr;  // [16]: eye queue lengths 4..6, photon 8..10, path-kernel work 12, regen 13
        unsigned long long* tctr = nullptr;  // closest-hit counters of the wavefront steps
        int2* rlist = nullptr;               // their FP64 refinement list (qcap entries)
        unsigned long long* entry = nullptr;  // stochastic hashing: the pass's table (T entries)
        uint32_t* ecount = nullptr;
    } tb[2];
    int cur = 0;
    float4 *hx = nullptr, *hn = nullptr, *hf = nullptr, *hd = nullptr;
    float4* slots = nullptr;
    uint32_t* pcount = nullptr;
    PathQ *q = nullptr, *qe = nullptr;
    uint32_t* qctr = nullptr;
    unsigned long long* tctr = nullptr;
    int2* rlist = nullptr;
    cudaStream_t tstream[2] = {nullptr, nullptr};  // tracing streams of overlapped passes, one per set
    cudaEvent_t ev_start = nullptr, ev_traced[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
    uint32_t *poff = nullptr, *counters = nullptr;
    uint32_t *keys[2] = {nullptr, nullptr}, *vals[2] = {nullptr, nullptr};
    uint32_t *hist = nullptr, *scan_tmp = nullptr, *bcount = nullptr, *bstart = nullptr;
    float4 *spos = nullptr, *spay = nullptr;
    unsigned long long* entry = nullptr;
    uint32_t* ecount = nullptr;
    float4 *ro = nullptr, *rd = nullptr, *rphi = nullptr;
    unsigned long long* started = nullptr;
    uint32_t* last_order = nullptr;  // sorted slot order of the last exact pass
    uint32_t* heavy = nullptr;  // exact gather: hit points with long queries (k_gather_heavy), npix entries
    unsigned long long* work = nullptr;  // work counters (kWorkCounts), see gsp_sppm_count_work
    bool count_work = false;
    // tuning
    int32_t gather_lanes = 8;  // lanes per hit point in the exact gather (set at creation)
    int32_t traversal = GSP_TRAVERSAL_MTBVH;  // of the path kernel
    int64_t qcap = 0;
    int32_t eye_steps = 0;      // eye wavefront steps before the persistent path kernel
    int32_t photon_steps = 0;   // photon wavefront steps before the persistent path kernel
    float refine_factor = 0.0f; // 0: every SPPM hit takes the refined (plane) distance
    // gradient (pass replay) buffers, allocated by gsp_sppm_enable_grad
    bool grad = false;
    int32_t grad_max_passes = 0, emit_mat = -1;
    float* rhist = nullptr;            // [max passes][npix] gather radius
    float4* shist = nullptr;           // [max passes][npix] gathered flux sum
    float4 *hw = nullptr, *badj = nullptr;  // hw aliases the trace buffers in use
    int32_t* smat = nullptr;                 // alias as hw
    double* gacc = nullptr;            // [nmat * 3 + 3]
    uint32_t *hp_order = nullptr, *hp_bstart = nullptr, *hp_scratch = nullptr;
    float4* hp_rec = nullptr;  // hit points in grid order for the adjoint gather (3 float4 each)
    int64_t hp_T = 0;
    int64_t passes = 0;
    std::vector<void*> allocs;
};

namespace {

template <class T>
cudaError_t alloc(gsp_sppm* r, T** p, int64_t count) {
    *p = nullptr;
    if (count <= 0) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)p, (size_t)count * sizeof(T));
    if (e == cudaSuccess) r->allocs.push_back((void*)*p);
    return e;
}

void free_all(gsp_sppm* r) {
    for (void* p : r->allocs) cudaFree(p);
    r->allocs.clear();
}

void use_buf(gsp_sppm* r, int j) {
    r->cur = j;
    r->hw = r->tb[j].hw;
    r->smat = r->tb[j].smat;
    r->hx = r->tb[j].hx;
    r->hn = r->tb[j].hn;
    r->hf = r->tb[j].hf;
    r->hd = r->tb[j].hd;
    r->slots = r->tb[j].slots;
    r->pcount = r->tb[j].pcount;
    r->q = r->tb[j].q;
    r->qe = r->tb[j].qe;
    r->qctr = r->tb[j].qctr;
    r->tctr = r->tb[j].tctr;
    r->rlist = r->tb[j].rlist;
    r->entry = r->tb[j].entry;
    r->ecount = r->tb[j].ecount;
}

// The path queues and counters of trace set j.
template <class AllocF>
void alloc_trace_queues(gsp_sppm* r, int j, AllocF&& A) {
    const int64_t nq = r->P.photon_mode == GSP_FULL_PATH ? r->np : 0;
    auto& t = r->tb[j];
    for (int b = 0; b < 2; ++b) {
        A(&t.q[b].ray, 2 * nq);
        A(&t.q[b].w, nq);
        A(&t.q[b].rng, nq);
        A(&t.q[b].meta, nq);
        A(&t.q[b].tri, nq);
        A(&t.q[b].t, nq);
        A(&t.qe[b].ray, 2 * r->npix);
        A(&t.qe[b].w, r->npix);
        A(&t.qe[b].rng, r->npix);
        A(&t.qe[b].meta, r->npix);
        A(&t.qe[b].tri, r->npix);
        A(&t.qe[b].t, r->npix);
    }
    A(&t.qctr, 16);
    A(&t.tctr, 2);
    A(&t.rlist, r->qcap);
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

extern "C" {

static gsp_status ensure_second_buffer(gsp_sppm* r);

gsp_status gsp_sppm_create(gsp_scene* s, const gsp_sppm_params* params, gsp_sppm** out) {
    if (!s || !params || !out) return GSP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!s->ctx || !s->has_cam) return GSP_ERR_INVALID_ARG;
    if (!s->built) return GSP_ERR_NOT_BUILT;
    GSP_NO_PENDING_ERROR("gsp_sppm_create");
    gsp_sppm_params P = *params;
    if (P.photons_per_pass <= 0 || P.photons_per_pass > (int64_t(1) << 27)) return GSP_ERR_INVALID_ARG;
    if (!(P.alpha > 0.0f && P.alpha <= 1.0f) || !(P.r0 > 0.0f) || !(P.rr_continue > 0.0f && P.rr_continue <= 1.0f) ||
        !(P.eps >= 0.0f) || P.max_eye_depth < 0 || P.max_eye_depth > 64 || P.max_photon_depth < 1 ||
        P.max_photon_depth > kSlotsPerPath || (P.photon_mode != GSP_FULL_PATH && P.photon_mode != GSP_REGEN) ||
        (P.hash_mode != GSP_EXACT && P.hash_mode != GSP_STOCHASTIC))
        return GSP_ERR_INVALID_ARG;
    if (P.cell_h == 0.0f) P.cell_h = 2.0f * P.r0;
    // the range query visits at most three cells per axis: exact mode needs h >= R (R <= r0);
    // stochastic hashing's estimator is defined with h >= 2 r0
    if (!(P.cell_h >= 0.25f * P.r0) || !std::isfinite(P.cell_h) ||
        (P.hash_mode == GSP_STOCHASTIC && P.cell_h < 2.0f * P.r0))
        return GSP_ERR_INVALID_ARG;
    if (P.table_size == 0) {
        P.table_size = 1;
        while (P.table_size < 2 * P.photons_per_pass) P.table_size *= 2;
    }
    if (P.table_size < 1 || P.table_size > (int64_t(1) << 30) || (P.table_size & (P.table_size - 1)))
        return GSP_ERR_INVALID_ARG;
    // emitting triangles: probability proportional to area * mean emission
    std::vector<int64_t> etri;
    std::vector<double> cdf;
    double acc = 0.0;
    for (int64_t i = 0; i < s->nt; ++i) {
        const gsp_material& m = s->mats[s->tri_mat[i]];
        if (!(m.type == GSP_DIFFUSE || m.type == GSP_EMITTER)) continue;
        if (!(std::max({m.emission[0], m.emission[1], m.emission[2]}) > 0.0f)) continue;
        const float* a = &s->verts[3 * (int64_t)s->tris[3 * i]];
        const float* b = &s->verts[3 * (int64_t)s->tris[3 * i + 1]];
        const float* c = &s->verts[3 * (int64_t)s->tris[3 * i + 2]];
        double e1[3], e2[3];
        for (int k = 0; k < 3; ++k) { e1[k] = (double)b[k] - a[k]; e2[k] = (double)c[k] - a[k]; }
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double area = 0.5 * std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(area > 0.0)) continue;
        acc += area * ((double)m.emission[0] + m.emission[1] + m.emission[2]) / 3.0;
        cdf.push_back(acc);
        etri.push_back(i);
    }
    if (etri.empty()) return GSP_ERR_INVALID_ARG;
    const int32_t ne = (int32_t)etri.size();
    std::vector<float4> emit(5 * (size_t)ne);
    std::vector<float> cdff(ne);
    for (int32_t j = 0; j < ne; ++j) {
        const int64_t i = etri[j];
        const gsp_material& m = s->mats[s->tri_mat[i]];
        const float* a = &s->verts[3 * (int64_t)s->tris[3 * i]];
        const float* b = &s->verts[3 * (int64_t)s->tris[3 * i + 1]];
        const float* c = &s->verts[3 * (int64_t)s->tris[3 * i + 2]];
        double e1[3], e2[3];
        for (int k = 0; k < 3; ++k) { e1[k] = (double)b[k] - a[k]; e2[k] = (double)c[k] - a[k]; }
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        // flux of a path started here: Le * pi * sum(area * mean Le) / mean Le (the probability
        // of picking the triangle times the density of its point cancels its own area)
        double mean = ((double)m.emission[0] + m.emission[1] + m.emission[2]) / 3.0;
        double scale = M_PI * acc / mean;
        emit[5 * j] = float4{a[0], a[1], a[2], 0.0f};
        emit[5 * j + 1] = float4{(float)e1[0], (float)e1[1], (float)e1[2], 0.0f};
        emit[5 * j + 2] = float4{(float)e2[0], (float)e2[1], (float)e2[2], 0.0f};
        emit[5 * j + 3] = float4{(float)(n[0] / len), (float)(n[1] / len), (float)(n[2] / len), 0.0f};
        emit[5 * j + 4] = float4{(float)(m.emission[0] * scale), (float)(m.emission[1] * scale),
                                 (float)(m.emission[2] * scale), 0.0f};
        cdff[j] = (float)(cdf[j] / acc);
    }
    GSP_CUDA_TRY(cudaSetDevice(s->ctx->device));
    gsp_sppm* r = new (std::nothrow) gsp_sppm;
    if (!r) return GSP_ERR_OOM;
    r->scene = s;
    r->P = P;
    r->w = s->cam.width;
    r->h = s->cam.height;
    r->npix = (int64_t)r->w * r->h;
    r->np = P.photons_per_pass;
    r->T = P.table_size;
    while ((int64_t(1) << r->tbits) < r->T) ++r->tbits;
    r->inv_h = 1.0f / P.cell_h;
    r->slots_per_path = P.photon_mode == GSP_FULL_PATH ? kSlotsPerPath : 1;
    r->slot_cap = r->np * r->slots_per_path;
    r->nemit = ne;
    {  // camera basis in FP64, passed on as double-float pairs
        const gsp_camera& c = s->cam;
        double eye[3] = {c.eye[0], c.eye[1], c.eye[2]}, f[3], rt[3], up[3];
        for (int k = 0; k < 3; ++k) f[k] = (double)c.look[k] - eye[k];
        double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        for (int k = 0; k < 3; ++k) f[k] /= fl;
        double u0[3] = {c.up[0], c.up[1], c.up[2]};
        rt[0] = f[1] * u0[2] - f[2] * u0[1];
        rt[1] = f[2] * u0[0] - f[0] * u0[2];
        rt[2] = f[0] * u0[1] - f[1] * u0[0];
        double rl = std::sqrt(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]);
        for (int k = 0; k < 3; ++k) rt[k] /= rl;
        up[0] = rt[1] * f[2] - rt[2] * f[1];
        up[1] = rt[2] * f[0] - rt[0] * f[2];
        up[2] = rt[0] * f[1] - rt[1] * f[0];
        r->cam.eye = make_float3((float)eye[0], (float)eye[1], (float)eye[2]);
        // each FP64 value as a double-float pair: hi its FP32 rounding, lo that of the remainder
        auto split3 = [](const double* v, float3& hi, float3& lo) {
            hi = make_float3((float)v[0], (float)v[1], (float)v[2]);
            lo = make_float3((float)(v[0] - (double)hi.x), (float)(v[1] - (double)hi.y), (float)(v[2] - (double)hi.z));
        };
        split3(f, r->cam.fwd_hi, r->cam.fwd_lo);
        split3(rt, r->cam.right_hi, r->cam.right_lo);
        split3(up, r->cam.up_hi, r->cam.up_lo);
        const double th = std::tan((double)c.vfov_deg * M_PI / 180.0 / 2.0), aspect = (double)c.width / (double)c.height;
        r->cam.th_hi = (float)th;
        r->cam.th_lo = (float)(th - (double)r->cam.th_hi);
        r->cam.aspect_hi = (float)aspect;
        r->cam.aspect_lo = (float)(aspect - (double)r->cam.aspect_hi);
        r->cam.w = c.width;
        r->cam.h = c.height;
    }
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, int64_t n) { if (e == cudaSuccess) e = alloc(r, p, n); };
    A(&r->d_emit, 5 * (int64_t)ne);
    A(&r->d_cdf, ne);
    A(&r->st0, r->npix);
    A(&r->st1, r->npix);
    A(&r->tb[0].hx, r->npix);
    A(&r->tb[0].hn, r->npix);
    A(&r->tb[0].hf, r->npix);
    A(&r->tb[0].hd, r->npix);
    A(&r->tb[0].slots, 2 * r->slot_cap);
    A(&r->tb[0].pcount, r->np);
    use_buf(r, 0);
    A(&r->poff, r->np);
    A(&r->counters, 16);
    A(&r->started, 1);
    A(&r->work, kWorkCounts);
    const int64_t scan_tmp = std::max({gsp_scan_temp_elems(r->np), gsp_scan_temp_elems(r->T),
                                       gsp_scan_temp_elems(gsp_sort_hist_elems())});
    A(&r->scan_tmp, scan_tmp);
    if (P.hash_mode == GSP_EXACT) {
        for (int b = 0; b < 2; ++b) {
            A(&r->keys[b], r->slot_cap);
            A(&r->vals[b], r->slot_cap);
        }
        A(&r->hist, gsp_sort_hist_elems());
        A(&r->bcount, r->T);
        A(&r->bstart, r->T + 1);
        A(&r->spos, r->slot_cap);
        A(&r->spay, r->slot_cap);
        // the heavy-query split pays on large images; on small ones its extra launch costs more
        if (r->npix >= kHeavyMinPixels) A(&r->heavy, r->npix);
    } else {
        A(&r->tb[0].entry, r->T);  // one table per trace set, so that passes overlap
        A(&r->tb[0].ecount, r->T);
    }
    r->qcap = std::max(r->npix, P.photon_mode == GSP_FULL_PATH ? r->np : (int64_t)0);
    // gather lanes per hit point: a small image's gather has too few hit points to fill the GPU
    // with 8 lanes each (a 64x64 pass: 0.183 against 0.200 ms with 16)
    r->gather_lanes = r->npix < kGatherWideBelow ? 16 : 8;
    r->eye_steps = 0;     // no wavefront steps: the persistent path kernel (per-lane refill)
    r->photon_steps = 0;  // traces every bounce; a step costs a closest-hit launch over the whole
                          // queue plus a shade launch, and waits for its slowest ray
    alloc_trace_queues(r, 0, A);
    use_buf(r, 0);
    if (P.photon_mode == GSP_REGEN) {
        A(&r->ro, r->np);
        A(&r->rd, r->np);
        A(&r->rphi, r->np);
    }
    if (e == cudaSuccess) e = cudaMemcpy(r->d_emit, emit.data(), emit.size() * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->d_cdf, cdff.data(), cdff.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_init_state<<<blocks(r->npix, 256), 256>>>(r->st0, r->st1, r->npix, P.r0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemset(r->started, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(r->counters, 0, 16 * sizeof(uint32_t));
    if (e == cudaSuccess && r->ro) {
        e = cudaMemset(r->ro, 0, r->np * sizeof(float4));
        if (e == cudaSuccess) e = cudaMemset(r->rd, 0, r->np * sizeof(float4));
        if (e == cudaSuccess) e = cudaMemset(r->rphi, 0, r->np * sizeof(float4));
    }
    // several passes are traced into both trace sets: the second one is made now, so that no
    // pass allocates
    if (e == cudaSuccess) {
        const gsp_status se = ensure_second_buffer(r);
        if (se != GSP_OK) {
            gsp_sppm_destroy(r);
            return se;
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_all(r);
        delete r;
        return gsp_cuda_fail(e);
    }
    *out = r;
    return GSP_OK;
}

void gsp_sppm_destroy(gsp_sppm* r) {
    if (!r) return;
    cudaSetDevice(r->scene->ctx->device);
    for (cudaStream_t t : r->tstream)
        if (t) cudaStreamDestroy(t);
    for (cudaEvent_t ev : {r->ev_start, r->ev_traced[0], r->ev_traced[1], r->ev_free[0], r->ev_free[1]})
        if (ev) cudaEventDestroy(ev);
    free_all(r);
    delete r;
}

static PassDev pass_params(const gsp_sppm* r, int64_t pass) {
    PassDev P;
    P.seed = r->P.seed;
    P.scene_id = r->P.scene_id;
    P.pass = (uint32_t)pass;
    P.pass_dev = nullptr;
    P.alpha = r->P.alpha;
    P.rr = r->P.rr_continue;
    P.eps = r->P.eps;
    P.inv_h = r->inv_h;
    P.max_eye = r->P.max_eye_depth;
    P.max_photon = r->P.max_photon_depth;
    P.tmask = (uint32_t)(r->T - 1);
    P.np = r->np;
    P.tri_is_id = r->refine_factor > 0.0f && !r->scene->d_attr ? 1 : 0;  // as eye_front / photon_front
    P.work = r->count_work ? r->work : nullptr;
    return P;
}

// Renderer counters (uint32): [0] deposits of the pass, [7] first pass index of a replayed graph,
// [10] hit points listed for k_gather_heavy, [11] out-of-range pixels of a state given to
// gsp_sppm_set_state.
// Per trace set (qctr): [4..6] eye queue lengths, [8..10] photon queue lengths (three each, used
// in rotation), [12] work counter of k_paths, [13] work counter of k_photon_regen.
static int sm_count(int device) {
    static int cached[64] = {0};
    if (device < 0 || device >= 64) device = 0;
    if (!cached[device]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
        cached[device] = std::max(1, v);
    }
    return cached[device];
}

// Grid-stride kernels over a queue whose length is on the device: 4 blocks of 256 per SM.
static unsigned shade_blocks(int64_t n, int device) {
    return (unsigned)std::min<int64_t>(blocks(n, 256), 4 * (int64_t)sm_count(device));
}

// Exact gather with `lanes` lanes per hit point (1, 4, 8 or 16).
static void launch_gather_exact(int lanes, const GatherDev& G, const PassDev& P, int64_t npix, cudaStream_t st) {
    switch (lanes) {
        case 1: k_gather_exact<1><<<blocks(npix, 128), 128, 0, st>>>(G, P); break;
        case 4: k_gather_exact<4><<<blocks(npix * 4, 128), 128, 0, st>>>(G, P); break;
        case 16: k_gather_exact<16><<<blocks(npix * 16, 128), 128, 0, st>>>(G, P); break;
        default: k_gather_exact<8><<<blocks(npix * 8, 128), 128, 0, st>>>(G, P); break;
    }
}

// Grid of a persistent path kernel (k_paths, or k_paths_multi when multi, of the given
// instantiation): resident blocks on every SM, but no more warps than items.
static int path_grid(int64_t items, int device, bool stack, bool shade, bool multi = false) {
    static int per_sm[2][2][2][64] = {};
    static int sms[64] = {0};
    if (device < 0 || device >= 64) device = 0;
    int& ps = per_sm[multi][stack][shade][device];
    if (!ps) {
        const void* const kernels[2][2][2] = {
            {{(const void*)k_paths<false, false, false>, (const void*)k_paths<false, true, false>},
             {(const void*)k_paths<true, false, false>, (const void*)k_paths<true, true, false>}},
            {{(const void*)k_paths_multi<false, false>, (const void*)k_paths_multi<false, true>},
             {(const void*)k_paths_multi<true, false>, (const void*)k_paths_multi<true, true>}}};
        int b = 0;
        cudaDeviceGetAttribute(&sms[device], cudaDevAttrMultiProcessorCount, device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernels[multi][stack][shade], kTraceThreads, 0);
        ps = std::max(1, b);
    }
    const int64_t full = (int64_t)std::max(1, sms[device]) * ps;
    const int64_t need = (items + kTraceThreads - 1) / kTraceThreads;
    return (int)std::max<int64_t>(1, std::min(full, need));
}

// Eye pass up to the persistent kernel: primary rays, then eye_steps wavefront steps. Returns in
// b the queue holding the paths still going (none if b > max_eye_depth).
static gsp_status eye_front(gsp_sppm* r, const PassDev& P, const EyeOut& O, cudaStream_t st, int& b) {
    gsp_scene* s = r->scene;
    const DevScene S = gsp_dev_scene(s);
    uint32_t* qn = r->qctr + 4;
    unsigned long long* tctr = r->tctr;
    // 0: every hit is refined in the shade kernel (always with per-vertex shading data, which
    // needs the hit's triangle slot for its barycentrics)
    const bool list = r->refine_factor > 0.0f && !s->d_attr;
    const float rf = list ? r->refine_factor : INFINITY;
    k_eye_emit<<<blocks(r->npix, 256), 256, 0, st>>>(r->cam, P, r->qe[0], O, qn, tctr, r->qctr + 12);
    for (b = 0; b < r->eye_steps && b <= r->P.max_eye_depth; ++b) {
        const PathQ& cur = r->qe[b & 1];
        GSP_CUDA_TRY(gsp_trace_queue(s, cur.ray, r->npix, qn + b % 3, cur.tri, cur.t, rf, false, !list, tctr, r->rlist, st));
        if (S.attr)
            k_eye_shade<true><<<shade_blocks(r->npix, s->ctx->device), 256, 0, st>>>(S, P, cur, r->qe[(b + 1) & 1], O, qn, b, tctr);
        else
            k_eye_shade<false><<<shade_blocks(r->npix, s->ctx->device), 256, 0, st>>>(S, P, cur, r->qe[(b + 1) & 1], O, qn, b, tctr);
    }
    return GSP_OK;
}

// Photon pass up to the persistent kernel: emission and photon_steps wavefront steps of whole
// paths (b = the queue still going; none if b >= max_photon_depth), or the one-bounce-per-thread
// pass of Sec. 3.3 (b = -1).
static gsp_status photon_front(gsp_sppm* r, const PassDev& P, const DepositDev& D, cudaStream_t st, int& b) {
    gsp_scene* s = r->scene;
    const DevScene S = gsp_dev_scene(s);
    uint32_t* qn = r->qctr + 8;
    unsigned long long* tctr = r->tctr;
    const bool list = r->refine_factor > 0.0f && !s->d_attr;
    const float rf = list ? r->refine_factor : INFINITY;
    const EmitDev E{r->d_emit, r->d_cdf, r->nemit};
    if (D.stochastic) {
        k_fill_u64<<<1024, 256, 0, st>>>(r->entry, r->T, ~0ull);
        GSP_CUDA_TRY(cudaMemsetAsync(r->ecount, 0, r->T * sizeof(uint32_t), st));
    }
    b = -1;
    if (r->P.photon_mode == GSP_FULL_PATH) {
        k_photon_emit<<<blocks(r->np, 256), 256, 0, st>>>(E, P, r->q[0], r->pcount, qn, tctr, r->qctr + 12);
        for (b = 0; b < r->photon_steps && b < r->P.max_photon_depth; ++b) {
            const PathQ& cur = r->q[b & 1];
            GSP_CUDA_TRY(gsp_trace_queue(s, cur.ray, r->np, qn + b % 3, cur.tri, cur.t, rf, false, !list, tctr, r->rlist, st));
            if (S.attr)
                k_photon_shade<true><<<shade_blocks(r->np, s->ctx->device), 256, 0, st>>>(S, P, D, cur, r->q[(b + 1) & 1], qn, b, tctr);
            else
                k_photon_shade<false><<<shade_blocks(r->np, s->ctx->device), 256, 0, st>>>(S, P, D, cur, r->q[(b + 1) & 1], qn, b, tctr);
        }
    } else {
        RegenDev R{r->ro, r->rd, r->rphi, r->started};
        GSP_CUDA_TRY(cudaMemsetAsync(r->qctr + 13, 0, sizeof(uint32_t), st));
        const bool stack = r->traversal == GSP_TRAVERSAL_STACK;
        const unsigned grid = (unsigned)path_grid(r->np, r->scene->ctx->device, stack, false);
        if (stack)
            S.attr ? k_photon_regen<true, true, false><<<grid, kTraceThreads, 0, st>>>(S, E, P, D, R, r->qctr + 13)
                   : k_photon_regen<true, false, false><<<grid, kTraceThreads, 0, st>>>(S, E, P, D, R, r->qctr + 13);
        else if (P.work)  // counting the work (never with the stack walk)
            S.attr ? k_photon_regen<false, true, true><<<grid, kTraceThreads, 0, st>>>(S, E, P, D, R, r->qctr + 13)
                   : k_photon_regen<false, false, true><<<grid, kTraceThreads, 0, st>>>(S, E, P, D, R, r->qctr + 13);
        else
            S.attr ? k_photon_regen<false, true, false><<<grid, kTraceThreads, 0, st>>>(S, E, P, D, R, r->qctr + 13)
                   : k_photon_regen<false, false, false><<<grid, kTraceThreads, 0, st>>>(S, E, P, D, R, r->qctr + 13);
    }
    return GSP_OK;
}

// Eye and photon passes of one pass (Sec. 2): both fronts, then one persistent kernel finishes
// the eye and photon paths still going.
// Both fronts of a pass; J describes the paths still going (J.nchunks == 0: none).
static gsp_status paths_front(gsp_sppm* r, const PassDev& P, const EyeOut& O, const DepositDev& D, cudaStream_t st,
                              PathJob& J) {
    int be = 0, bp = -1;
    gsp_status e = eye_front(r, P, O, st, be);
    if (e == GSP_OK) e = photon_front(r, P, D, st, bp);
    if (e != GSP_OK) return e;
    const bool eye_left = be <= r->P.max_eye_depth;
    const bool ph_left = bp >= 0 && bp < r->P.max_photon_depth;
    J.S = gsp_dev_scene(r->scene);
    J.P = P;
    J.qe = r->qe[be & 1];
    J.qp = r->q[ph_left ? bp & 1 : 0];
    J.O = O;
    J.D = D;
    J.ne_ptr = eye_left ? r->qctr + 4 + be % 3 : nullptr;
    J.np_ptr = ph_left ? r->qctr + 8 + bp % 3 : nullptr;
    J.first_chunk = 0;
    const int64_t items = (eye_left ? r->npix : 0) + (ph_left ? r->np : 0);
    J.nchunks = (int32_t)((items + kMultiChunk - 1) / kMultiChunk);
    return GSP_OK;
}

static gsp_status stage_paths(gsp_sppm* r, const PassDev& P, const EyeOut& O, const DepositDev& D, cudaStream_t st) {
    NvtxRange nvtx("gsp: eye + photon paths");
    PathJob J;
    gsp_status e = paths_front(r, P, O, D, st, J);
    if (e != GSP_OK) return e;
    if (J.nchunks > 0) {
        const bool stack = r->traversal == GSP_TRAVERSAL_STACK;
        const unsigned grid = (unsigned)path_grid((int64_t)J.nchunks * kMultiChunk, r->scene->ctx->device, stack, J.S.attr != nullptr);
        if (stack)
            J.S.attr ? k_paths<true, true, false><<<grid, kTraceThreads, 0, st>>>(J.S, P, J.qe, O, J.ne_ptr, J.qp, D, J.np_ptr, r->qctr + 12)
                     : k_paths<true, false, false><<<grid, kTraceThreads, 0, st>>>(J.S, P, J.qe, O, J.ne_ptr, J.qp, D, J.np_ptr, r->qctr + 12);
        else if (P.work)  // counting the work (never with the stack walk)
            J.S.attr ? k_paths<false, true, true><<<grid, kTraceThreads, 0, st>>>(J.S, P, J.qe, O, J.ne_ptr, J.qp, D, J.np_ptr, r->qctr + 12)
                     : k_paths<false, false, true><<<grid, kTraceThreads, 0, st>>>(J.S, P, J.qe, O, J.ne_ptr, J.qp, D, J.np_ptr, r->qctr + 12);
        else
            J.S.attr ? k_paths<false, true, false><<<grid, kTraceThreads, 0, st>>>(J.S, P, J.qe, O, J.ne_ptr, J.qp, D, J.np_ptr, r->qctr + 12)
                     : k_paths<false, false, false><<<grid, kTraceThreads, 0, st>>>(J.S, P, J.qe, O, J.ne_ptr, J.qp, D, J.np_ptr, r->qctr + 12);
    }
    GSP_CUDA_TRY(cudaGetLastError());
    return GSP_OK;
}

// Exact hash grid of the pass's deposits: compaction in id order, stable sort by bucket,
// bucket starts, sorted SoA copies.
static gsp_status stage_deposit(gsp_sppm* r, const PassDev& P, cudaStream_t st) {
    uint32_t* d_total = r->counters;  // deposits this pass
    GSP_CUDA_TRY(gsp_scan_u32(r->pcount, r->poff, r->np, d_total, r->scan_tmp, st));
    GSP_CUDA_TRY(cudaMemsetAsync(r->bcount, 0, r->T * sizeof(uint32_t), st));
    k_compact<<<blocks(r->np, 256), 256, 0, st>>>(r->slots, r->pcount, r->poff, r->np, r->slots_per_path, r->inv_h,
                                                  P.tmask, r->keys[0], r->vals[0], r->bcount);
    GSP_CUDA_TRY(gsp_scan_u32(r->bcount, r->bstart, r->T, r->bstart + r->T, r->scan_tmp, st));
    uint32_t *ko = nullptr, *vo = nullptr;
    GSP_CUDA_TRY(gsp_radix_sort_u32(r->keys[0], r->vals[0], r->keys[1], r->vals[1], d_total, r->tbits, r->hist,
                                    r->scan_tmp, st, &ko, &vo));
    r->last_order = vo;
    k_permute<<<1024, 256, 0, st>>>(r->slots, vo, d_total, r->spos, r->spay);
    GSP_CUDA_TRY(cudaGetLastError());
    return GSP_OK;
}

// The pass's deposits in path order, without the hash grid: the list the adjoint's photon loop
// walks (a grid would only order it).
static gsp_status stage_deposit_list(gsp_sppm* r, cudaStream_t st) {
    uint32_t* d_total = r->counters;
    GSP_CUDA_TRY(gsp_scan_u32(r->pcount, r->poff, r->np, d_total, r->scan_tmp, st));
    k_compact<<<blocks(r->np, 256), 256, 0, st>>>(r->slots, r->pcount, r->poff, r->np, r->slots_per_path, 0.0f, 0u,
                                                  nullptr, r->vals[0], nullptr);
    r->last_order = r->vals[0];
    k_permute<<<1024, 256, 0, st>>>(r->slots, r->vals[0], d_total, r->spos, r->spay);
    GSP_CUDA_TRY(cudaGetLastError());
    return GSP_OK;
}

// One pass on stream st. In graph mode (a pass captured once and replayed) the pass index is read
// from the device counter counters[7], which the pass advances itself, and the host count is left
// to the caller.
// Tracing half of a pass: eye and photon passes into the trace buffers in use.
static gsp_status trace_half(gsp_sppm* r, const PassDev& P, cudaStream_t st) {
    const EyeOut O{r->hx, r->hn, r->hf, r->hd, nullptr};
    const DepositDev D{r->slots, r->pcount, r->entry, r->ecount, r->P.hash_mode == GSP_STOCHASTIC ? 1 : 0, nullptr};
    return stage_paths(r, P, O, D, st);
}

// Gather half of a pass: deposit (exact mode) and the fused range query + progressive update.
static gsp_status gather_half(gsp_sppm* r, const PassDev& P, cudaStream_t st) {
    NvtxRange nvtx("gsp: deposit + gather");
    GatherDev G{};
    G.hx = r->hx;
    G.hn = r->hn;
    G.hf = r->hf;
    G.hd = r->hd;
    G.st0 = r->st0;
    G.st1 = r->st1;
    G.npix = r->npix;
    G.rhist = r->grad ? r->rhist : nullptr;
    G.shist = r->grad ? r->shist : nullptr;
    if (r->P.hash_mode == GSP_STOCHASTIC) {
        G.slots = r->slots;
        G.entry = r->entry;
        G.ecount = r->ecount;
        // deposit count for diagnostics
        GSP_CUDA_TRY(gsp_scan_u32(r->pcount, r->poff, r->np, r->counters, r->scan_tmp, st));
        k_gather_stoch<<<blocks(r->npix, 128), 128, 0, st>>>(G, P);
    } else {
        gsp_status e = stage_deposit(r, P, st);
        if (e != GSP_OK) return e;
        G.spos = r->spos;
        G.spay = r->spay;
        G.bstart = r->bstart;
        // long queries are listed by k_gather_exact and served by whole blocks (counters[10] counts them)
        if (r->heavy) {
            G.heavy = r->heavy;
            G.nheavy = r->counters + 10;
            GSP_CUDA_TRY(cudaMemsetAsync(G.nheavy, 0, sizeof(uint32_t), st));
        }
        launch_gather_exact(r->gather_lanes, G, P, r->npix, st);
        if (r->heavy) k_gather_heavy<<<2 * sm_count(r->scene->ctx->device), kHeavyThreads, 0, st>>>(G, P);
    }
    if (P.work) k_work_add<<<1, 1, 0, st>>>(P.work + kWorkDeposits, r->counters);
    GSP_CUDA_TRY(cudaGetLastError());
    return GSP_OK;
}

#ifndef GSP_ADJ_LANES
#define GSP_ADJ_LANES 8
#endif

static gsp_status check_grad_room(gsp_sppm* r, int64_t npasses) {
    if (r->grad && r->passes + npasses > r->grad_max_passes) {
        gsp_set_last_error("gsp_sppm_pass: more passes than gsp_sppm_enable_grad reserved radius history for");
        return GSP_ERR_OVERFLOW;
    }
    return GSP_OK;
}

static gsp_status sppm_one_pass(gsp_sppm* r, cudaStream_t st, bool graph = false) {
    PassDev P = pass_params(r, r->passes);
    if (graph) {
        P.pass_dev = r->counters + 7;
        P.pass = 0;
    }
    gsp_status e = check_grad_room(r, graph ? 0 : 1);
    if (e == GSP_OK) e = trace_half(r, P, st);
    if (e == GSP_OK) e = gather_half(r, P, st);
    if (e != GSP_OK) return e;
    if (graph) k_add_u32<<<1, 1, 0, st>>>(r->counters + 7, 1u);
    GSP_CUDA_TRY(cudaGetLastError());
    if (!graph) r->passes += 1;
    return GSP_OK;
}

// The second set of trace buffers, the tracing streams and their events (at creation in exact
// mode, else on first use).
static gsp_status ensure_second_buffer(gsp_sppm* r) {
    if (r->tb[1].hx && r->tb[1].qctr && (!r->grad || r->tb[1].hw) &&
        (r->P.hash_mode != GSP_STOCHASTIC || r->tb[1].entry))
        return GSP_OK;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, int64_t n) {
        if (e == cudaSuccess && !*p) e = alloc(r, p, n);
    };
    A(&r->tb[1].hx, r->npix);
    A(&r->tb[1].hn, r->npix);
    A(&r->tb[1].hf, r->npix);
    A(&r->tb[1].hd, r->npix);
    A(&r->tb[1].slots, 2 * r->slot_cap);
    A(&r->tb[1].pcount, r->np);
    if (r->grad) {
        A(&r->tb[1].hw, r->npix);
        A(&r->tb[1].smat, r->slot_cap);
    }
    if (r->P.hash_mode == GSP_STOCHASTIC) {
        A(&r->tb[1].entry, r->T);
        A(&r->tb[1].ecount, r->T);
    }
    if (!r->tb[1].qctr) alloc_trace_queues(r, 1, A);
    for (cudaStream_t& t : r->tstream)
        if (e == cudaSuccess && !t) e = cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&r->ev_start, &r->ev_traced[0], &r->ev_traced[1], &r->ev_free[0], &r->ev_free[1]})
        if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return gsp_cuda_fail(e);
    use_buf(r, r->cur);
    return GSP_OK;
}

// Several passes, pass i traced on tracing stream i % 2 into trace set i % 2 while the caller's
// stream deposits and gathers the pass before: the tracing of pass i + 1 starts as soon as its
// set has been gathered (pass i - 1), so it runs beside the long tail of pass i's path kernel,
// when only the longest paths are still going, and beside pass i's sort and gather. Events order
// each set's reuse (and, with paths carried from pass to pass, the tracing itself); results are
// those of one pass after the other. Exact hashing only (stochastic hashing shares its table
// between the two halves).
static gsp_status passes_overlapped(gsp_sppm* r, int32_t npasses, cudaStream_t st) {
    gsp_status se = ensure_second_buffer(r);
    if (se != GSP_OK) return se;
    // the tracing streams start after everything the caller queued before
    GSP_CUDA_TRY(cudaEventRecord(r->ev_start, st));
    for (cudaStream_t t : r->tstream) GSP_CUDA_TRY(cudaStreamWaitEvent(t, r->ev_start, 0));
    const bool chained = r->P.photon_mode == GSP_REGEN;  // photon paths continue into the next pass
    for (int32_t i = 0; i < npasses; ++i) {
        const int j = i & 1;
        use_buf(r, j);
        const PassDev P = pass_params(r, r->passes);
        if (i >= 2) GSP_CUDA_TRY(cudaStreamWaitEvent(r->tstream[j], r->ev_free[j], 0));  // pass i - 2 gathered
        if (chained && i >= 1) GSP_CUDA_TRY(cudaStreamWaitEvent(r->tstream[j], r->ev_traced[j ^ 1], 0));
        gsp_status e = trace_half(r, P, r->tstream[j]);
        if (e != GSP_OK) return e;
        GSP_CUDA_TRY(cudaEventRecord(r->ev_traced[j], r->tstream[j]));
        GSP_CUDA_TRY(cudaStreamWaitEvent(st, r->ev_traced[j], 0));
        e = gather_half(r, P, st);
        if (e != GSP_OK) return e;
        GSP_CUDA_TRY(cudaEventRecord(r->ev_free[j], st));
        r->passes += 1;
    }
    return GSP_OK;
}

gsp_status gsp_sppm_tune(gsp_sppm* r, int32_t eye_steps, int32_t photon_steps, float refine_factor,
                         int32_t gather_lanes, int32_t traversal) {
    if (!r || eye_steps < 0 || eye_steps > 64 || photon_steps < 0 || photon_steps > kSlotsPerPath ||
        !(refine_factor >= 0.0f) ||
        (gather_lanes != 0 && gather_lanes != 1 && gather_lanes != 4 && gather_lanes != 8 && gather_lanes != 16) ||
        (traversal != 0 && traversal != GSP_TRAVERSAL_MTBVH && traversal != GSP_TRAVERSAL_STACK) ||
        (traversal == GSP_TRAVERSAL_STACK && r->scene->bvh.depth >= kStackDepth))
        return GSP_ERR_INVALID_ARG;
    if (r->count_work && (eye_steps || photon_steps || traversal == GSP_TRAVERSAL_STACK)) {
        gsp_set_last_error("gsp_sppm_tune: work is counted in the persistent stackless path kernels only");
        return GSP_ERR_BAD_STATE;
    }
    r->eye_steps = eye_steps;
    r->photon_steps = photon_steps;
    r->refine_factor = refine_factor;
    if (gather_lanes) r->gather_lanes = gather_lanes;
    if (traversal) r->traversal = traversal;
    return GSP_OK;
}

gsp_status gsp_sppm_count_work(gsp_sppm* r, int32_t on, uint64_t* h_counts) {
    if (!r) return GSP_ERR_INVALID_ARG;
    if (on && (r->eye_steps || r->photon_steps || r->traversal == GSP_TRAVERSAL_STACK)) {
        gsp_set_last_error("gsp_sppm_count_work: work is counted in the persistent stackless path kernels only "
                           "(no wavefront steps, traversal GSP_TRAVERSAL_MTBVH)");
        return GSP_ERR_BAD_STATE;
    }
    GSP_CUDA_TRY(cudaSetDevice(r->scene->ctx->device));
    GSP_CUDA_TRY(cudaDeviceSynchronize());
    if (h_counts)
        GSP_CUDA_TRY(cudaMemcpy(h_counts, r->work, kWorkCounts * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    GSP_CUDA_TRY(cudaMemset(r->work, 0, kWorkCounts * sizeof(unsigned long long)));
    r->count_work = on != 0;
    return GSP_OK;
}

gsp_status gsp_sppm_pass(gsp_sppm* r, int32_t npasses, void* stream) {
    if (!r || npasses < 0) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(r->scene->ctx->device));
    GSP_NO_PENDING_ERROR("gsp_sppm_pass");
    gsp_status s = check_grad_room(r, npasses);
    if (s != GSP_OK) return s;
    if (npasses >= 2) return passes_overlapped(r, npasses, (cudaStream_t)stream);
    for (int32_t i = 0; i < npasses; ++i) {
        s = sppm_one_pass(r, (cudaStream_t)stream);
        if (s != GSP_OK) return s;
    }
    return GSP_OK;
}

gsp_status gsp_sppm_enable_grad(gsp_sppm* r, int32_t max_passes) {
    if (!r || max_passes < 1) return GSP_ERR_INVALID_ARG;
    if (r->passes != 0 || r->grad) return GSP_ERR_BAD_STATE;
    if (r->P.photon_mode != GSP_FULL_PATH || r->P.hash_mode != GSP_EXACT || r->scene->nmat > kMaxGradMats) {
        gsp_set_last_error("gsp_sppm_enable_grad: needs whole photon paths, the exact hash grid and at most 64 materials");
        return GSP_ERR_INVALID_ARG;
    }
    int em = -1;
    for (int32_t m = 0; m < r->scene->nmat; ++m) {
        const gsp_material& mt = r->scene->mats[m];
        if ((mt.type == GSP_DIFFUSE || mt.type == GSP_EMITTER) &&
            std::max({mt.emission[0], mt.emission[1], mt.emission[2]}) > 0.0f) {
            if (em >= 0) {
                gsp_set_last_error("gsp_sppm_enable_grad: needs exactly one emitting material");
                return GSP_ERR_INVALID_ARG;
            }
            em = m;
        }
    }
    GSP_CUDA_TRY(cudaSetDevice(r->scene->ctx->device));
    r->hp_T = 1;
    while (r->hp_T < 2 * r->npix) r->hp_T *= 2;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, int64_t n) { if (e == cudaSuccess) e = alloc(r, p, n); };
    A(&r->rhist, (int64_t)max_passes * r->npix);
    A(&r->shist, (int64_t)max_passes * r->npix);
    for (int j = 0; j < 2; ++j)
        if (r->tb[j].hx) {
            A(&r->tb[j].hw, r->npix);
            A(&r->tb[j].smat, r->slot_cap);
        }
    A(&r->badj, r->slot_cap);
    A(&r->gacc, (int64_t)kMaxGradMats * 3 + 3);
    A(&r->hp_order, r->npix);
    A(&r->hp_bstart, r->hp_T + 1);
    A(&r->hp_scratch, gsp_grid_scratch_words(r->npix, r->hp_T));
    A(&r->hp_rec, 3 * r->npix);
    if (e != cudaSuccess) return gsp_cuda_fail(e);
    r->grad = true;
    r->grad_max_passes = max_passes;
    r->emit_mat = em;
    use_buf(r, r->cur);
    return GSP_OK;
}

gsp_status gsp_render_grad(gsp_sppm* r, const float* d_dloss_dimg, float* d_grad_albedo, float* d_grad_emission,
                           void* stream) {
    if (!r || !d_dloss_dimg || !d_grad_albedo || !d_grad_emission) return GSP_ERR_INVALID_ARG;
    if (!r->grad || r->passes < 1) return GSP_ERR_BAD_STATE;
    GSP_CUDA_TRY(cudaSetDevice(r->scene->ctx->device));
    GSP_NO_PENDING_ERROR("gsp_render_grad");
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t nmat = r->scene->nmat;
    GSP_CUDA_TRY(cudaMemsetAsync(r->gacc, 0, ((size_t)kMaxGradMats * 3 + 3) * sizeof(double), st));
    const float hp_cell = 2.0f * r->P.r0;
    const int grid = 4 * sm_count(r->scene->ctx->device);
    // Pass i + 1 is replayed on the other tracing stream into the other trace set while the adjoint
    // kernels of pass i run on the caller's stream (the same double buffering as gsp_sppm_pass).
    gsp_status e = ensure_second_buffer(r);
    if (e != GSP_OK) return e;
    GSP_CUDA_TRY(cudaEventRecord(r->ev_start, st));
    for (cudaStream_t t : r->tstream) GSP_CUDA_TRY(cudaStreamWaitEvent(t, r->ev_start, 0));
    for (int64_t i = 0; i < r->passes; ++i) {
        const int j = (int)(i & 1);
        use_buf(r, j);
        // replay pass i from its PRNG counters: the same hit points, photons and radii
        NvtxRange nvtx("gsp: adjoint pass");
        const PassDev P = pass_params(r, i);
        const EyeOut O{r->hx, r->hn, r->hf, r->hd, r->hw};
        const DepositDev D{r->slots, r->pcount, nullptr, nullptr, 0, r->smat};
        if (i >= 2) GSP_CUDA_TRY(cudaStreamWaitEvent(r->tstream[j], r->ev_free[j], 0));
        e = stage_paths(r, P, O, D, r->tstream[j]);
        if (e != GSP_OK) return e;
        GSP_CUDA_TRY(cudaEventRecord(r->ev_traced[j], r->tstream[j]));
        GSP_CUDA_TRY(cudaStreamWaitEvent(st, r->ev_traced[j], 0));
        e = stage_deposit_list(r, st);
        if (e != GSP_OK) return e;
        e = gsp_grid_build_with(r->hx, r->npix, hp_cell, r->hp_T, r->hp_order, r->hp_bstart, r->hp_scratch, st, true);
        if (e != GSP_OK) return e;
        AdjDev A;
        A.hx = r->hx;
        A.hn = r->hn;
        A.hf = r->hf;
        A.hw = r->hw;
        A.rhist = r->rhist + (size_t)i * r->npix;
        A.g = d_dloss_dimg;
        A.hp_order = r->hp_order;
        A.hp_bstart = r->hp_bstart;
        A.hp_mask = (uint32_t)(r->hp_T - 1);
        A.inv_hp = 1.0f / hp_cell;
        A.rmax = r->P.r0;
        A.spos = r->spos;
        A.spay = r->spay;
        A.order = r->last_order;
        A.d_total = r->counters;
        A.badj = r->badj;
        A.work = r->count_work ? r->work : nullptr;
        A.hp_rec = r->hp_rec;
        if (A.work) k_work_add<<<1, 1, 0, st>>>(A.work + kWorkDeposits, r->counters);
        k_adj_hp_records<<<blocks(r->npix, 256), 256, 0, st>>>(A, r->npix, r->hp_rec);
        k_adj_photons<GSP_ADJ_LANES><<<grid * GSP_ADJ_LANES, 128, 0, st>>>(A);
        k_adj_pixels<<<grid, 256, 0, st>>>(r->hx, r->hw, A.rhist, r->shist + (size_t)i * r->npix, d_dloss_dimg,
                                           r->npix, r->gacc, nmat);
        k_adj_paths<<<grid, 128, 0, st>>>(r->slots, r->pcount, r->smat, r->badj, r->scene->d_mats, r->np, r->gacc,
                                          nmat);
        GSP_CUDA_TRY(cudaEventRecord(r->ev_free[j], st));
    }
    const double ne = (double)r->passes * (double)r->np;
    k_adj_emission<<<256, 256, 0, st>>>(r->st0, r->st1, d_dloss_dimg, r->npix, 1.0f / (float)r->passes, ne,
                                        r->gacc + (size_t)nmat * 3);
    const gsp_material& em = r->scene->mats[r->emit_mat];
    k_adj_finalize<<<1, 256, 0, st>>>(r->gacc, nmat, 1.0 / (M_PI * ne),
                                      make_float4(em.emission[0], em.emission[1], em.emission[2], 0.0f), d_grad_albedo,
                                      d_grad_emission);
    GSP_CUDA_TRY(cudaGetLastError());
    return GSP_OK;
}

}  // extern "C"

struct gsp_batch {
    std::vector<gsp_sppm*> rs;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins, joins2;  // per renderer: ends of its branches (first, second pass)
    cudaEvent_t fork = nullptr, paths[2] = {nullptr, nullptr};
    cudaStream_t cap = nullptr;   // private stream the graphs are captured on (never the legacy stream)
    cudaStream_t cap2 = nullptr;  // the second pass's path launch in a two-pass graph
    cudaGraphExec_t exec = nullptr;   // one pass
    cudaGraphExec_t exec2 = nullptr;  // fused: two passes, the second traced beside the first
    int32_t device = 0;
    bool fused = true;           // all renderers' paths in one persistent launch (k_paths_multi)
    PathJob* d_jobs = nullptr;   // fused: job tables, [0, n) one-pass graph, [n, 3n) two-pass graph
    uint32_t* d_ctr = nullptr;   // fused: the path kernel's work counters (one per table)
    std::vector<DevScene> captured;  // each renderer's scene as the graphs baked it in
};

// Whether every renderer's scene still has the device description the graphs were captured
// with (a new BVH, new shading data or a new step limit changes it; replaying would then read
// freed or stale buffers).
static bool batch_scenes_unchanged(const gsp_batch* b) {
    if (b->captured.size() != b->rs.size()) return false;
    for (size_t i = 0; i < b->rs.size(); ++i) {
        const DevScene x = gsp_dev_scene(b->rs[i]->scene), &y = b->captured[i];
        if (x.nodes != y.nodes || x.tris != y.tris || x.shade != y.shade || x.nlo != y.nlo || x.mats != y.mats ||
            x.bin != y.bin || x.attr != y.attr || x.texels != y.texels || x.mtex != y.mtex || x.nnodes != y.nnodes ||
            x.stride != y.stride || x.link_sets != y.link_sets || x.bin_root != y.bin_root ||
            x.step_limit != y.step_limit || x.status != y.status)
            return false;
    }
    return true;
}

static void batch_note_scenes(gsp_batch* b) {
    b->captured.clear();
    for (gsp_sppm* r : b->rs) b->captured.push_back(gsp_dev_scene(r->scene));
}

static void batch_drop_graphs(gsp_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->exec2) cudaGraphExecDestroy(b->exec2);
    b->exec = b->exec2 = nullptr;
}

static void batch_free(gsp_batch* b) {
    batch_drop_graphs(b);
    for (auto s : b->streams) cudaStreamDestroy(s);
    for (auto e : b->joins) cudaEventDestroy(e);
    for (auto e : b->joins2) cudaEventDestroy(e);
    for (cudaEvent_t e : {b->fork, b->paths[0], b->paths[1]})
        if (e) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->cap2) cudaStreamDestroy(b->cap2);
    cudaFree(b->d_jobs);
    cudaFree(b->d_ctr);
    delete b;
}

// Back to the state of a new renderer (radii r0, nothing gathered, no pass run).
static cudaError_t reset_state(gsp_sppm* t, cudaStream_t st) {
    t->passes = 0;
    k_init_state<<<blocks(t->npix, 256), 256, 0, st>>>(t->st0, t->st1, t->npix, t->P.r0);
    cudaError_t e = cudaMemsetAsync(t->started, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess && t->rd) e = cudaMemsetAsync(t->rd, 0, t->np * sizeof(float4), st);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

// Fused form of batch passes: the eye and photon fronts of every renderer in parallel branches,
// then ONE persistent k_paths_multi launch over all renderers' remaining paths, then the
// deposits and gathers in parallel branches. K = 2 captures two passes into one graph, pass k in
// trace set k: the second pass's fronts and path launch depend on nothing of the first, so its
// paths fill the SMs that the first path launch's tail leaves idle; each renderer's second gather
// follows its first. The job tables hold only pointers and device counters, so they are written
// once, after the capture.
static gsp_status batch_capture_fused(gsp_batch* b, cudaStream_t st, int K, cudaGraphExec_t* out) {
    const int n = (int)b->rs.size();
    if (!b->d_jobs) {
        GSP_CUDA_TRY(cudaMalloc(&b->d_jobs, 3 * (size_t)n * sizeof(PathJob)));
        GSP_CUDA_TRY(cudaMalloc(&b->d_ctr, 3 * sizeof(uint32_t)));
    }
    if (K == 2)
        for (gsp_sppm* r : b->rs) {  // both trace sets (made outside the capture)
            gsp_status se = ensure_second_buffer(r);
            if (se != GSP_OK) return se;
        }
    bool stack = true, shade = false;  // one launch for all: shading code if any scene has shading data
    for (gsp_sppm* r : b->rs) {
        stack = stack && r->traversal == GSP_TRAVERSAL_STACK;
        shade = shade || r->scene->d_attr != nullptr;
    }
    const size_t base = K == 2 ? (size_t)n : 0;  // job tables and counters of this graph
    std::vector<PathJob> jobs((size_t)K * n);
    std::vector<PassDev> passes((size_t)K * n);
    std::vector<int32_t> total(K, 0);
    GSP_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    gsp_status e = GSP_OK;
    cudaError_t ce = cudaEventRecord(b->fork, st);
    for (int i = 0; i < n && ce == cudaSuccess; ++i) ce = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
    if (ce == cudaSuccess && K == 2) ce = cudaStreamWaitEvent(b->cap2, b->fork, 0);
    // fronts: per renderer, pass 0 then pass 1 on its branch
    for (int k = 0; k < K && ce == cudaSuccess && e == GSP_OK; ++k)
        for (int i = 0; i < n && ce == cudaSuccess && e == GSP_OK; ++i) {
            gsp_sppm* r = b->rs[i];
            use_buf(r, k);
            PassDev& P = passes[(size_t)k * n + i];
            P = pass_params(r, r->passes);
            P.pass_dev = r->counters + 7;
            P.pass = (uint32_t)k;
            const EyeOut O{r->hx, r->hn, r->hf, r->hd, nullptr};
            const DepositDev D{r->slots, r->pcount, r->entry, r->ecount, r->P.hash_mode == GSP_STOCHASTIC ? 1 : 0,
                               nullptr};
            e = paths_front(r, P, O, D, b->streams[i], jobs[(size_t)k * n + i]);
            if (e == GSP_OK) ce = cudaEventRecord((k == 0 ? b->joins : b->joins2)[i], b->streams[i]);
        }
    // one path launch per pass, pass 1's on its own stream
    for (int k = 0; k < K && ce == cudaSuccess && e == GSP_OK; ++k) {
        cudaStream_t ps = k == 0 ? st : b->cap2;
        for (int i = 0; i < n && ce == cudaSuccess; ++i) ce = cudaStreamWaitEvent(ps, (k == 0 ? b->joins : b->joins2)[i], 0);
        for (int i = 0; i < n; ++i) {
            PathJob& J = jobs[(size_t)k * n + i];
            J.first_chunk = total[k];
            total[k] += J.nchunks;
        }
        uint32_t* ctr = b->d_ctr + (K == 2 ? 1 + k : 0);
        const PathJob* jt = b->d_jobs + base + (size_t)k * n;
        if (ce == cudaSuccess && total[k] > 0) {
            ce = cudaMemsetAsync(ctr, 0, sizeof(uint32_t), ps);
            const unsigned grid = (unsigned)path_grid((int64_t)total[k] * kMultiChunk, b->device, stack, shade, true);
            if (ce == cudaSuccess) {
                if (stack)
                    shade ? k_paths_multi<true, true><<<grid, kTraceThreads, 0, ps>>>(jt, n, total[k], ctr)
                          : k_paths_multi<true, false><<<grid, kTraceThreads, 0, ps>>>(jt, n, total[k], ctr);
                else
                    shade ? k_paths_multi<false, true><<<grid, kTraceThreads, 0, ps>>>(jt, n, total[k], ctr)
                          : k_paths_multi<false, false><<<grid, kTraceThreads, 0, ps>>>(jt, n, total[k], ctr);
                ce = cudaGetLastError();
            }
        }
        if (ce == cudaSuccess) ce = cudaEventRecord(b->paths[k], ps);
    }
    // deposits and gathers: per renderer, pass 0 then pass 1 on its branch
    for (int k = 0; k < K && ce == cudaSuccess && e == GSP_OK; ++k)
        for (int i = 0; i < n && ce == cudaSuccess && e == GSP_OK; ++i) {
            gsp_sppm* r = b->rs[i];
            use_buf(r, k);
            ce = cudaStreamWaitEvent(b->streams[i], b->paths[k], 0);
            if (ce == cudaSuccess) e = gather_half(r, passes[(size_t)k * n + i], b->streams[i]);
            if (ce == cudaSuccess && e == GSP_OK && k == K - 1) {
                k_add_u32<<<1, 1, 0, b->streams[i]>>>(r->counters + 7, (uint32_t)K);
                ce = cudaEventRecord(b->joins[i], b->streams[i]);
                if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, b->joins[i], 0);
            }
        }
    if (ce == cudaSuccess && e == GSP_OK && K == 2) ce = cudaStreamWaitEvent(st, b->paths[1], 0);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(st, &g);
    if (ce == cudaSuccess) ce = ee;
    if (ce == cudaSuccess && e == GSP_OK) ce = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    if (ce == cudaSuccess && e == GSP_OK)
        ce = cudaMemcpy(b->d_jobs + base, jobs.data(), jobs.size() * sizeof(PathJob), cudaMemcpyHostToDevice);
    if (e != GSP_OK) return e;
    if (ce != cudaSuccess) return gsp_cuda_fail(ce);
    return GSP_OK;
}

// One pass of every renderer captured as a single CUDA graph: a branch per renderer, forked
// from and joined to the capturing stream, so the scenes' kernels overlap on the GPU.
static gsp_status batch_capture(gsp_batch* b, cudaStream_t st) {
    if (b->fused) return batch_capture_fused(b, st, 1, &b->exec);
    GSP_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    gsp_status e = GSP_OK;
    cudaError_t ce = cudaEventRecord(b->fork, st);
    for (size_t i = 0; i < b->rs.size() && ce == cudaSuccess && e == GSP_OK; ++i) {
        ce = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
        if (ce == cudaSuccess) e = sppm_one_pass(b->rs[i], b->streams[i], true);
        if (ce == cudaSuccess && e == GSP_OK) ce = cudaEventRecord(b->joins[i], b->streams[i]);
        if (ce == cudaSuccess && e == GSP_OK) ce = cudaStreamWaitEvent(st, b->joins[i], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(st, &g);
    if (ce == cudaSuccess) ce = ee;
    if (ce == cudaSuccess && e == GSP_OK) ce = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != GSP_OK) return e;
    if (ce != cudaSuccess) return gsp_cuda_fail(ce);
    return GSP_OK;
}

// Two-pass graphs need exact hashing everywhere: a stochastic pass resets its hash table in its
// fronts, which the previous pass's photons may still be filling.
static bool batch_pairs(const gsp_batch* b) {
    if (!b->fused) return false;
    for (const gsp_sppm* r : b->rs)
        if (r->P.hash_mode != GSP_EXACT) return false;
    return true;
}

extern "C" {

gsp_status gsp_batch_create(gsp_sppm* const* renderers, int32_t n, gsp_batch** out) {
    if (!renderers || n < 1 || !out) return GSP_ERR_INVALID_ARG;
    *out = nullptr;
    const int32_t dev = renderers[0] ? renderers[0]->scene->ctx->device : -1;
    for (int32_t i = 0; i < n; ++i) {
        if (!renderers[i] || renderers[i]->scene->ctx->device != dev) return GSP_ERR_INVALID_ARG;
        for (int32_t j = 0; j < i; ++j)
            if (renderers[j]->scene == renderers[i]->scene) {  // a scene's trace scratch is shared
                gsp_set_last_error("gsp_batch_create: renderers of one batch need distinct scenes");
                return GSP_ERR_INVALID_ARG;
            }
    }
    GSP_CUDA_TRY(cudaSetDevice(dev));
    gsp_batch* b = new (std::nothrow) gsp_batch;
    if (!b) return GSP_ERR_OOM;
    b->device = dev;
    b->rs.assign(renderers, renderers + n);
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (cudaEvent_t* ev : {&b->paths[0], &b->paths[1]})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking);
    for (int32_t i = 0; i < n && e == cudaSuccess; ++i) {
        cudaStream_t s = nullptr;
        cudaEvent_t j = nullptr, j2 = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->streams.push_back(s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
        if (e == cudaSuccess) b->joins.push_back(j);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j2, cudaEventDisableTiming);
        if (e == cudaSuccess) b->joins2.push_back(j2);
    }
    (void)gsp_trace_grid(dev);  // fill the launch-size cache outside any capture
    if (e != cudaSuccess) {
        batch_free(b);
        return gsp_cuda_fail(e);
    }
    *out = b;
    return GSP_OK;
}

gsp_status gsp_batch_tune(gsp_batch* b, int32_t fused) {
    if (!b || fused < 0 || fused > 1) return GSP_ERR_INVALID_ARG;
    if (b->fused != (fused == 1)) {
        cudaSetDevice(b->device);
        batch_drop_graphs(b);  // captured again at the next gsp_batch_pass
    }
    b->fused = fused == 1;
    return GSP_OK;
}

void gsp_batch_destroy(gsp_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    batch_free(b);
}

gsp_status gsp_batch_pass(gsp_batch* b, int32_t npasses, void* stream) {
    if (!b || npasses < 0) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(b->device));
    GSP_NO_PENDING_ERROR("gsp_batch_pass");
    cudaStream_t st = (cudaStream_t)stream;
    for (gsp_sppm* r : b->rs) {
        if (r->grad && r->passes + npasses > r->grad_max_passes) return GSP_ERR_OVERFLOW;
        if (r->count_work) {
            gsp_set_last_error("gsp_batch_pass: a renderer counts its work (batched passes are not counted)");
            return GSP_ERR_BAD_STATE;
        }
    }
    if (npasses == 0) return GSP_OK;
    if ((b->exec || b->exec2) && !batch_scenes_unchanged(b)) batch_drop_graphs(b);
    // pairs of passes as two-pass graphs where they apply, the rest one pass per graph
    const int32_t pairs = batch_pairs(b) ? npasses / 2 : 0, singles = npasses - 2 * pairs;
    if (pairs > 0 && !b->exec2) {
        gsp_status e = batch_capture_fused(b, b->cap, 2, &b->exec2);  // capture runs nothing
        if (e != GSP_OK) return e;
        batch_note_scenes(b);
    }
    if (singles > 0 && !b->exec) {
        gsp_status e = batch_capture(b, b->cap);  // capture runs nothing; the graph launches on st
        if (e != GSP_OK) return e;
        batch_note_scenes(b);
    }
    for (gsp_sppm* r : b->rs) k_store_u32<<<1, 1, 0, st>>>(r->counters + 7, (uint32_t)r->passes);
    for (int32_t k = 0; k < pairs; ++k) GSP_CUDA_TRY(cudaGraphLaunch(b->exec2, st));
    for (int32_t k = 0; k < singles; ++k) GSP_CUDA_TRY(cudaGraphLaunch(b->exec, st));
    for (gsp_sppm* r : b->rs) r->passes += npasses;
    GSP_CUDA_TRY(cudaGetLastError());
    return GSP_OK;
}

// The autotuners keep their current choice unless a candidate is clearly faster: a renderer's
// trials are a few short passes from a fresh state, whose timings vary by a few percent and whose
// radii are those of a render's first passes, so it asks for 3 %; a batch's trials are whole-batch
// passes of many milliseconds, steady to well under a percent, so it asks for 1 %.
constexpr float kTuneMargin = 0.97f;
constexpr float kBatchTuneMargin = 0.99f;

gsp_status gsp_batch_autotune(gsp_batch* b, int32_t trial_passes, gsp_tune_result* out) {
    if (!b || trial_passes < 1) return GSP_ERR_INVALID_ARG;
    for (gsp_sppm* r : b->rs)
        if (r->passes != 0 || r->grad || r->count_work) return GSP_ERR_BAD_STATE;
    GSP_CUDA_TRY(cudaSetDevice(b->device));
    GSP_NO_PENDING_ERROR("gsp_batch_autotune");
    cudaStream_t st = b->cap;
    cudaEvent_t a = nullptr, z = nullptr;
    cudaError_t ce = cudaEventCreate(&a);
    if (ce == cudaSuccess) ce = cudaEventCreate(&z);
    gsp_status e = GSP_OK;
    // cf: hash cell edge of the exact-mode renderers as a multiple of each one's r0 (0: the edge
    // each had before tuning); a stochastic renderer's cell edge is part of its estimate and stays
    struct Cand { int32_t es, ps, gl, tr; bool fused; float cf; };
    const Cand start{b->rs[0]->eye_steps, b->rs[0]->photon_steps, b->rs[0]->gather_lanes, b->rs[0]->traversal,
                     b->fused, 0.0f};
    std::vector<float> cell0;
    bool any_exact = false;
    for (gsp_sppm* r : b->rs) {
        cell0.push_back(r->P.cell_h);
        any_exact = any_exact || r->P.hash_mode == GSP_EXACT;
    }
    bool stack_ok = true;
    for (gsp_sppm* r : b->rs) stack_ok = stack_ok && r->scene->bvh.depth < kStackDepth;
    Cand pick = start;
    float best = INFINITY, first = INFINITY;
    int32_t ncand = 0;
    auto apply = [&](const Cand& c) {
        for (size_t i = 0; i < b->rs.size(); ++i) {
            gsp_sppm* r = b->rs[i];
            r->eye_steps = c.es;
            r->photon_steps = c.ps;
            r->gather_lanes = c.gl;
            r->traversal = c.tr;
            if (r->P.hash_mode == GSP_EXACT) {
                r->P.cell_h = c.cf > 0.0f ? c.cf * r->P.r0 : cell0[i];
                r->inv_h = 1.0f / r->P.cell_h;
            }
        }
        b->fused = c.fused;
        batch_drop_graphs(b);
    };
    // Each candidate: capture its graph, one untimed graph launch, then trial_passes timed passes
    // the way gsp_batch_pass runs them (two-pass graphs where they apply), then every renderer
    // back to its initial state.
    auto trial = [&](const Cand& c) {
        if (ce != cudaSuccess || e != GSP_OK) return;
        apply(c);
        const bool two = batch_pairs(b) && trial_passes >= 2;
        e = two ? batch_capture_fused(b, st, 2, &b->exec2) : batch_capture(b, st);
        cudaGraphExec_t g = two ? b->exec2 : b->exec;
        const int32_t per = two ? 2 : 1, launches = (trial_passes + per - 1) / per;
        for (int32_t k = 0; k <= launches && e == GSP_OK && ce == cudaSuccess; ++k) {
            if (k == 1) ce = cudaEventRecord(a, st);
            for (gsp_sppm* r : b->rs) k_store_u32<<<1, 1, 0, st>>>(r->counters + 7, (uint32_t)(k * per));
            if (ce == cudaSuccess) ce = cudaGraphLaunch(g, st);
        }
        if (ce == cudaSuccess && e == GSP_OK) ce = cudaEventRecord(z, st);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(z);
        float ms = 0.0f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, a, z);
        for (gsp_sppm* r : b->rs)
            if (ce == cudaSuccess) ce = reset_state(r, st);
        ms /= (float)(launches * per);
        if (ncand++ == 0) first = ms;
        if (ms < best * kBatchTuneMargin) {  // a clear gain only (kBatchTuneMargin)
            best = ms;
            pick = c;
        }
    };
    trial(start);
    const bool full = b->rs[0]->P.photon_mode == GSP_FULL_PATH;
    for (int32_t es : {0, 1})
        for (int32_t ps : full ? std::vector<int32_t>{0, 1, 2} : std::vector<int32_t>{0})
            if (es != start.es || ps != start.ps) trial({es, ps, start.gl, start.tr, start.fused, 0.0f});
    const Cand steps = pick;
    if (any_exact)  // the exact-mode cell edge (a multiple of each renderer's r0)
        for (float cf : {2.0f, 1.5f, 1.0f, 0.75f}) trial({steps.es, steps.ps, start.gl, start.tr, start.fused, cf});
    const Cand cell = pick;
    for (int32_t gl : {4, 8, 16})
        if (gl != start.gl) trial({cell.es, cell.ps, gl, start.tr, start.fused, cell.cf});
    const Cand lanes = pick;
    for (int32_t tr : {GSP_TRAVERSAL_MTBVH, GSP_TRAVERSAL_STACK})
        if (tr != start.tr && (tr != GSP_TRAVERSAL_STACK || stack_ok))
            trial({lanes.es, lanes.ps, lanes.gl, tr, start.fused, lanes.cf});
    // last: one fused path launch for all renderers, or a path launch per renderer; with the
    // steps searched again for the other form (the best split moves)
    const Cand form = pick;
    for (int32_t es : {0, 1})
        for (int32_t ps : full ? std::vector<int32_t>{0, 1, 2} : std::vector<int32_t>{0})
            trial({es, ps, form.gl, form.tr, !form.fused, form.cf});
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (a) cudaEventDestroy(a);
    if (z) cudaEventDestroy(z);
    apply(pick);  // captured again at the next gsp_batch_pass
    if (e != GSP_OK) return e;
    if (ce != cudaSuccess) return gsp_cuda_fail(ce);
    if (out) {
        out->eye_steps = pick.es;
        out->photon_steps = pick.ps;
        out->cell_h = b->rs[0]->P.cell_h;
        out->ms_per_pass = best;
        out->first_ms_per_pass = first;
        out->candidates = ncand;
        out->gather_lanes = pick.gl;
        out->traversal = pick.tr;
        out->fused = pick.fused ? 1 : 0;
    }
    return GSP_OK;
}

gsp_status gsp_sppm_autotune(gsp_sppm* r, int32_t trial_passes, gsp_tune_result* out) {
    if (!r || trial_passes < 1) return GSP_ERR_INVALID_ARG;
    if (r->count_work) {
        gsp_set_last_error("gsp_sppm_autotune: the renderer counts its work (its settings must stay put)");
        return GSP_ERR_BAD_STATE;
    }
    GSP_CUDA_TRY(cudaSetDevice(r->scene->ctx->device));
    GSP_NO_PENDING_ERROR("gsp_sppm_autotune");
    gsp_sppm* t = nullptr;
    gsp_sppm_params P = r->P;
    gsp_status e = gsp_sppm_create(r->scene, &P, &t);
    if (e != GSP_OK) return e;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, z = nullptr;
    cudaError_t ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreate(&a);
    if (ce == cudaSuccess) ce = cudaEventCreate(&z);
    struct Cand { int32_t es, ps; float cell; int32_t gl, tr; };
    int32_t ncand = 0;
    float best = INFINITY, first = INFINITY;
    Cand pick{r->eye_steps, r->photon_steps, r->P.cell_h, r->gather_lanes, r->traversal};
    // Each candidate starts from a fresh state (radii r0), runs one untimed pass and times
    // trial_passes more, so every candidate sees the same radii. Several passes are timed the
    // way gsp_sppm_pass runs them (overlapped), which changes which settings win:
    // the overlap hides the path kernel's tail.
    const bool overlap = trial_passes >= 2;
    if (overlap) e = ensure_second_buffer(t);
    auto trial = [&](const Cand& c) {
        if (ce != cudaSuccess || e != GSP_OK) return;
        t->eye_steps = c.es;
        t->photon_steps = c.ps;
        t->inv_h = 1.0f / c.cell;
        t->gather_lanes = c.gl;
        t->traversal = c.tr;
        ce = reset_state(t, st);
        if (ce != cudaSuccess) return;
        e = sppm_one_pass(t, st);
        if (e != GSP_OK) return;
        ce = cudaEventRecord(a, st);
        if (overlap)
            e = passes_overlapped(t, trial_passes, st);
        else
            for (int32_t k = 0; k < trial_passes && e == GSP_OK; ++k) e = sppm_one_pass(t, st);
        if (ce == cudaSuccess) ce = cudaEventRecord(z, st);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(z);
        float ms = 0.0f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, a, z);
        ms /= (float)trial_passes;
        if (ncand++ == 0) first = ms;
        if (ms < best * kTuneMargin) {  // a clear gain only: trial timings vary by a few percent
            best = ms;
            pick = c;
        }
    };
    // stage 1: wavefront steps at the renderer's cell edge; stage 2: the cell edge (exact mode)
    const bool full = r->P.photon_mode == GSP_FULL_PATH;
    const int32_t gl0 = r->gather_lanes, tr0 = r->traversal;
    trial({r->eye_steps, r->photon_steps, r->P.cell_h, gl0, tr0});  // the current settings first
    for (int32_t es : {0, 1, 2})
        for (int32_t ps : full ? std::vector<int32_t>{0, 1, 2, 4} : std::vector<int32_t>{0})
            if (es != r->eye_steps || ps != r->photon_steps) trial({es, ps, r->P.cell_h, gl0, tr0});
    if (r->P.hash_mode == GSP_EXACT) {
        // stage 2: the cell edge; stage 3: lanes per hit point in the gather
        const Cand steps = pick;
        for (float c : {2.0f, 1.5f, 1.0f, 0.75f, 0.5f})
            if (c * r->P.r0 != r->P.cell_h) trial({steps.es, steps.ps, c * r->P.r0, gl0, tr0});
        const Cand cell = pick;
        for (int32_t gl : {1, 4, 8, 16})
            if (gl != gl0) trial({cell.es, cell.ps, cell.cell, gl, tr0});
    }
    // last stage: the path kernel's traversal
    const Cand lanes = pick;
    for (int32_t tr : {GSP_TRAVERSAL_MTBVH, GSP_TRAVERSAL_STACK})
        if (tr != tr0 && (tr != GSP_TRAVERSAL_STACK || r->scene->bvh.depth < kStackDepth))
            trial({lanes.es, lanes.ps, lanes.cell, lanes.gl, tr});
    if (st) cudaStreamDestroy(st);
    if (a) cudaEventDestroy(a);
    if (z) cudaEventDestroy(z);
    gsp_sppm_destroy(t);
    if (e != GSP_OK) return e;
    if (ce != cudaSuccess) return gsp_cuda_fail(ce);
    r->eye_steps = pick.es;
    r->photon_steps = pick.ps;
    r->gather_lanes = pick.gl;
    r->traversal = pick.tr;
    r->inv_h = 1.0f / pick.cell;
    r->P.cell_h = pick.cell;
    if (out) {
        out->eye_steps = pick.es;
        out->photon_steps = pick.ps;
        out->cell_h = pick.cell;
        out->ms_per_pass = best;
        out->first_ms_per_pass = first;
        out->candidates = ncand;
        out->gather_lanes = pick.gl;
        out->traversal = pick.tr;
    }
    return GSP_OK;
}

// ---- checkpoint -------------------------------------------------------------------------------
// File: "GSPPMCK1", then a header of int64 fields {version, npix, np, passes, photon_mode,
// hash_mode, grad passes recorded}, the creation parameters (raw gsp_sppm_params), then the
// arrays: pixel state st0, st1 (npix float4 each); in REGEN mode the per-thread path state
// ro, rd, rphi (np float4 each) and the started-path count; with gradients the recorded radii
// and flux sums of the passes so far.
static const char kCkMagic[8] = {'G', 'S', 'P', 'P', 'M', 'C', 'K', '1'};

static bool ck_write(FILE* f, const void* d_src, size_t bytes, std::vector<char>& buf) {
    buf.resize(bytes);
    if (bytes) {
        const cudaError_t e = cudaMemcpy(buf.data(), d_src, bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            (void)gsp_cuda_fail(e);  // message and last error; the call reports GSP_ERR_IO
            return false;
        }
    }
    return fwrite(buf.data(), 1, bytes, f) == bytes;
}

// One section of a checkpoint read into host memory; copied to d_dst only once every section of
// the file has been read (a short or corrupt file leaves the renderer as it was).
struct CkSection {
    void* d_dst;
    std::vector<char> data;
};

// Whether a pixel state (st0 = {tau, N}, st1 = {direct, R}) holds only values a render can reach:
// N finite and >= 0, R finite in (0, r0], tau and the direct sums finite and >= 0.
static bool state_in_range(const float4* st0, const float4* st1, int64_t npix, float r0) {
    auto fin = [](float v) { return std::isfinite(v) && v >= 0.0f; };
    for (int64_t p = 0; p < npix; ++p) {
        const float4 a = st0[p], b = st1[p];
        if (!(fin(a.x) && fin(a.y) && fin(a.z) && fin(a.w) && fin(b.x) && fin(b.y) && fin(b.z) &&
              std::isfinite(b.w) && b.w > 0.0f && b.w <= r0))
            return false;
    }
    return true;
}

static bool ck_read(FILE* f, void* d_dst, size_t bytes, std::vector<CkSection>& out) {
    CkSection c{d_dst, std::vector<char>(bytes)};
    if (fread(c.data.data(), 1, bytes, f) != bytes) return false;
    out.push_back(std::move(c));
    return true;
}

gsp_status gsp_sppm_save(gsp_sppm* r, const char* path) {
    if (!r || !path) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(r->scene->ctx->device));
    GSP_CUDA_TRY(cudaDeviceSynchronize());
    FILE* f = fopen(path, "wb");
    if (!f) return GSP_ERR_IO;
    const int64_t hdr[7] = {1, r->npix, r->np, r->passes, r->P.photon_mode, r->P.hash_mode,
                            r->grad ? r->passes : 0};
    std::vector<char> buf;
    bool ok = fwrite(kCkMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof hdr, 1, f) == 1 &&
              fwrite(&r->P, sizeof r->P, 1, f) == 1 && ck_write(f, r->st0, r->npix * sizeof(float4), buf) &&
              ck_write(f, r->st1, r->npix * sizeof(float4), buf);
    if (ok && r->P.photon_mode == GSP_REGEN)
        ok = ck_write(f, r->ro, r->np * sizeof(float4), buf) && ck_write(f, r->rd, r->np * sizeof(float4), buf) &&
             ck_write(f, r->rphi, r->np * sizeof(float4), buf) && ck_write(f, r->started, sizeof(unsigned long long), buf);
    if (ok && r->grad && r->passes > 0)
        ok = ck_write(f, r->rhist, (size_t)r->passes * r->npix * sizeof(float), buf) &&
             ck_write(f, r->shist, (size_t)r->passes * r->npix * sizeof(float4), buf);
    ok = (fclose(f) == 0) && ok;
    return ok ? GSP_OK : GSP_ERR_IO;
}

gsp_status gsp_sppm_load(gsp_sppm* r, const char* path) {
    if (!r || !path) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(r->scene->ctx->device));
    GSP_CUDA_TRY(cudaDeviceSynchronize());
    FILE* f = fopen(path, "rb");
    if (!f) return GSP_ERR_IO;
    char magic[8];
    int64_t hdr[7];
    gsp_sppm_params P, mine = r->P;
    std::vector<CkSection> sec;
    gsp_status st = GSP_OK;
    const bool read_ok = fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCkMagic, 8) == 0 &&
                         fread(hdr, sizeof hdr, 1, f) == 1 && fread(&P, sizeof P, 1, f) == 1;
    // In exact mode the cell edge is an execution setting (the autotuner changes it): ignore it.
    if (read_ok && P.hash_mode == GSP_EXACT) P.cell_h = mine.cell_h;
    if (!read_ok) {
        st = GSP_ERR_IO;
    } else if (hdr[0] != 1 || hdr[1] != r->npix || hdr[2] != r->np || hdr[4] != r->P.photon_mode ||
               hdr[5] != r->P.hash_mode || std::memcmp(&P, &mine, sizeof P) != 0 || hdr[3] < 0 ||
               (hdr[6] > 0 && (!r->grad || hdr[6] > r->grad_max_passes)) || (r->grad && hdr[6] != hdr[3])) {
        gsp_set_last_error("gsp_sppm_load: the checkpoint was written by a renderer with other parameters");
        st = GSP_ERR_BAD_STATE;
    } else {
        bool ok = ck_read(f, r->st0, r->npix * sizeof(float4), sec) && ck_read(f, r->st1, r->npix * sizeof(float4), sec);
        if (ok && r->P.photon_mode == GSP_REGEN)
            ok = ck_read(f, r->ro, r->np * sizeof(float4), sec) && ck_read(f, r->rd, r->np * sizeof(float4), sec) &&
                 ck_read(f, r->rphi, r->np * sizeof(float4), sec) &&
                 ck_read(f, r->started, sizeof(unsigned long long), sec);
        if (ok && hdr[6] > 0)
            ok = ck_read(f, r->rhist, (size_t)hdr[6] * r->npix * sizeof(float), sec) &&
                 ck_read(f, r->shist, (size_t)hdr[6] * r->npix * sizeof(float4), sec);
        ok = ok && fgetc(f) == EOF;  // nothing may follow the last section
        if (!ok) {
            gsp_set_last_error("gsp_sppm_load: the checkpoint is short or has trailing data; the renderer is unchanged");
            st = GSP_ERR_IO;
        } else if (!state_in_range((const float4*)sec[0].data.data(), (const float4*)sec[1].data.data(), r->npix,
                                   r->P.r0)) {
            gsp_set_last_error("gsp_sppm_load: the checkpoint's pixel state is out of range (N < 0, R outside (0, r0] "
                               "or values not finite); the renderer is unchanged");
            st = GSP_ERR_IO;
        }
    }
    fclose(f);
    if (st != GSP_OK) return st;
    // the whole file has been read: only now is the renderer's state replaced
    for (const CkSection& c : sec)
        if (!c.data.empty()) GSP_CUDA_TRY(cudaMemcpy(c.d_dst, c.data.data(), c.data.size(), cudaMemcpyHostToDevice));
    r->passes = hdr[3];
    return GSP_OK;
}

gsp_status gsp_sppm_image(gsp_sppm* r, float* d_rgb, void* stream) {
    if (!r || !d_rgb) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(r->scene->ctx->device));
    GSP_NO_PENDING_ERROR("gsp_sppm_image");
    const float inv_p = r->passes > 0 ? 1.0f / (float)r->passes : 0.0f;
    const double ne_host = (double)r->passes * (double)r->np;
    k_image<<<blocks(r->npix, 256), 256, 0, (cudaStream_t)stream>>>(
        r->st0, r->st1, r->npix, inv_p, ne_host, r->P.photon_mode == GSP_REGEN ? r->started : nullptr, d_rgb);
    GSP_CUDA_TRY(cudaGetLastError());
    return GSP_OK;
}

gsp_status gsp_sppm_state(gsp_sppm* r, float* d_N, float* d_R, float* d_tau, float* d_direct,
                          double* h_counts, void* stream) {
    if (!r) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(r->scene->ctx->device));
    GSP_NO_PENDING_ERROR("gsp_sppm_state");
    cudaStream_t st = (cudaStream_t)stream;
    if (d_N || d_R || d_tau || d_direct) {
        k_state<<<blocks(r->npix, 256), 256, 0, st>>>(r->st0, r->st1, r->npix, d_N, d_R, d_tau, d_direct);
        GSP_CUDA_TRY(cudaGetLastError());
    }
    if (h_counts) {
        double ne = (double)r->passes * (double)r->np;
        if (r->P.photon_mode == GSP_REGEN) {
            unsigned long long v = 0;
            GSP_CUDA_TRY(cudaMemcpyAsync(&v, r->started, sizeof v, cudaMemcpyDeviceToHost, st));
            GSP_CUDA_TRY(cudaStreamSynchronize(st));
            ne = (double)v;
        }
        h_counts[0] = (double)r->passes;
        h_counts[1] = ne;
    }
    return GSP_OK;
}

gsp_status gsp_sppm_set_state(gsp_sppm* r, const float* d_N, const float* d_R, const float* d_tau,
                              const float* d_direct, int64_t passes, void* stream) {
    if (!r || !d_N || !d_R || !d_tau || !d_direct || passes < 0 || passes > UINT32_MAX) return GSP_ERR_INVALID_ARG;
    if (r->P.photon_mode != GSP_FULL_PATH || r->grad) {
        gsp_set_last_error("gsp_sppm_set_state: whole photon paths only, and not with gradients enabled");
        return GSP_ERR_BAD_STATE;
    }
    GSP_CUDA_TRY(cudaSetDevice(r->scene->ctx->device));
    GSP_NO_PENDING_ERROR("gsp_sppm_set_state");
    // every value is checked before any is taken (a radius above r0 would make a gather visit
    // cells without bound): counters[11] counts the pixels out of range
    const cudaStream_t st = (cudaStream_t)stream;
    GSP_CUDA_TRY(cudaMemsetAsync(r->counters + 11, 0, sizeof(uint32_t), st));
    k_check_state<<<blocks(r->npix, 256), 256, 0, st>>>(r->npix, d_N, d_R, d_tau, d_direct, r->P.r0, r->counters + 11);
    uint32_t bad = 0;
    GSP_CUDA_TRY(cudaMemcpyAsync(&bad, r->counters + 11, sizeof bad, cudaMemcpyDeviceToHost, st));
    GSP_CUDA_TRY(cudaStreamSynchronize(st));
    if (bad) {
        gsp_set_last_error("gsp_sppm_set_state: N must be finite and >= 0, R finite in (0, r0], tau and the direct "
                           "sums finite and >= 0; the renderer is unchanged");
        return GSP_ERR_INVALID_ARG;
    }
    k_set_state<<<blocks(r->npix, 256), 256, 0, st>>>(r->st0, r->st1, r->npix, d_N, d_R, d_tau, d_direct);
    GSP_CUDA_TRY(cudaGetLastError());
    r->passes = passes;
    return GSP_OK;
}

int64_t gsp_sppm_last_deposits(gsp_sppm* r, uint32_t* h_ids, int64_t capacity) {
    if (!r) return GSP_ERR_INVALID_ARG;
    cudaError_t ce = cudaSetDevice(r->scene->ctx->device);
    if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
    uint32_t total = 0;
    if (ce == cudaSuccess) ce = cudaMemcpy(&total, r->counters, sizeof total, cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return gsp_cuda_fail(ce);
    if (!h_ids) return (int64_t)total;
    if (capacity < (int64_t)total) return GSP_ERR_INVALID_ARG;
    // ids of every deposit: walk the per-path counts on the host
    std::vector<uint32_t> cnt(r->np);
    std::vector<float4> rec(2 * (size_t)r->slot_cap);
    ce = cudaMemcpy(cnt.data(), r->pcount, r->np * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaMemcpy(rec.data(), r->slots, rec.size() * sizeof(float4), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return gsp_cuda_fail(ce);
    int64_t k = 0;
    for (int64_t pth = 0; pth < r->np; ++pth)
        for (uint32_t i = 0; i < cnt[pth]; ++i) {
            const int64_t slot = pth * r->slots_per_path + i;
            uint32_t id;
            std::memcpy(&id, &rec[2 * slot].w, 4);
            if (k < capacity) h_ids[k] = id;
            ++k;
        }
    std::sort(h_ids, h_ids + k);
    return k;
}

}  // extern "C"

// Scratch (uint32 words) of a hash-grid build over n points with T buckets: key/value
// ping-pong buffers, the radix histogram, scan partials and the device copy of n.
int64_t gsp_grid_scratch_words(int64_t n, int64_t T) { return gsp_grid_scratch_words_c(n, T); }

// Exact hash grid of n points: keys -> counts -> in-place bucket scan -> stable radix sort.
gsp_status gsp_grid_build_with(const float4* pos, int64_t n, float cell_h, int64_t T, uint32_t* order,
                               uint32_t* bstart, uint32_t* scratch, cudaStream_t st, bool skip_invalid) {
    int tbits = 0;
    while ((int64_t(1) << tbits) < T) ++tbits;
    if (skip_invalid) ++tbits;  // the key T of skipped points needs one more bit
    uint32_t* ka = scratch;
    uint32_t* va = ka + n;
    uint32_t* kb = va + n;
    uint32_t* vb = kb + n;
    uint32_t* hist = vb + n;
    uint32_t* nbuf = hist + gsp_sort_hist_elems();
    uint32_t* tmp = nbuf + 64;
    GSP_CUDA_TRY(cudaMemsetAsync(bstart, 0, (size_t)T * sizeof(uint32_t), st));
    k_store_u32<<<1, 1, 0, st>>>(nbuf, (uint32_t)n);
    if (n > 0)
        k_grid_keys<<<(unsigned)std::min<int64_t>(blocks(n, 256), 4096), 256, 0, st>>>(
            pos, n, 1.0f / cell_h, (uint32_t)(T - 1), ka, va, bstart, skip_invalid ? 1 : 0);
    GSP_CUDA_TRY(gsp_scan_u32(bstart, bstart, T, bstart + T, tmp, st));
    uint32_t *ko = nullptr, *vo = nullptr;
    GSP_CUDA_TRY(gsp_radix_sort_u32(ka, va, kb, vb, nbuf, tbits, hist, tmp, st, &ko, &vo));
    if (n > 0) GSP_CUDA_TRY(cudaMemcpyAsync(order, vo, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    GSP_CUDA_TRY(cudaGetLastError());
    return GSP_OK;
}

static gsp_status grid_args_ok(const float* d_pos, int64_t n, float cell_h, int64_t T, const uint32_t* d_order,
                               const uint32_t* d_bstart) {
    if (n < 0 || n > INT32_MAX || !(cell_h > 0.0f) || !std::isfinite(cell_h) || T < 1 || T > (int64_t(1) << 30) ||
        (T & (T - 1)) || !d_bstart || (n > 0 && (!d_pos || !d_order)) || ((uintptr_t)d_pos & 15))
        return GSP_ERR_INVALID_ARG;
    return GSP_OK;
}

extern "C" {

gsp_status gsp_hash_grid_build(gsp_context* ctx, const float* d_pos, int64_t n, float cell_h, int64_t table_size,
                               uint32_t* d_order, uint32_t* d_bstart, void* stream) {
    if (!ctx) return GSP_ERR_INVALID_ARG;
    gsp_status a = grid_args_ok(d_pos, n, cell_h, table_size, d_order, d_bstart);
    if (a != GSP_OK) return a;
    GSP_CUDA_TRY(cudaSetDevice(ctx->device));
    GSP_NO_PENDING_ERROR("gsp_hash_grid_build");
    const int64_t words = gsp_grid_scratch_words(n, table_size);
    if (words > ctx->grid_words) {  // grow the context's scratch (first use or a larger build)
        GSP_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
        cudaFree(ctx->grid_scratch);
        ctx->grid_scratch = nullptr;
        ctx->grid_words = 0;
        GSP_CUDA_TRY(cudaMalloc(&ctx->grid_scratch, (size_t)words * sizeof(uint32_t)));
        ctx->grid_words = words;
    }
    return gsp_grid_build_with((const float4*)d_pos, n, cell_h, table_size, d_order, d_bstart, ctx->grid_scratch,
                               (cudaStream_t)stream, false);
}

gsp_status gsp_sppm_sync(gsp_sppm* r) {
    if (!r) return GSP_ERR_INVALID_ARG;
    return gsp_context_sync(r->scene->ctx);
}

}  // extern "C"
