// sppm.cu -- stochastic progressive photon mapping on the device (Sec. 2, 3.3, 3.4).
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
//   trace sets    two (both made at creation in exact mode), each:
//     hit points  hx[p] = {x.xyz, material or -1}, hn[p] = {n_s.xyz, 0},
//                 hf[p] = {w * albedo / pi, 0}, hd[p] = {direct.rgb, 0}     64 B / pixel
//     photons     slot s: {x.xyz, id}, {flux.rgb, octahedral direction}    32 B / deposit
//                 path k owns slots [k*32, k*32+32) (one slot per thread in REGEN mode)
//     queues      eye and photon wavefront queues, two of each (ping-pong), their lengths,
//                 the path kernel's work counter, the wavefront steps' trace counters
//   exact grid    bucket-sorted SoA copies spos[], spay[] + bucket starts bstart[T+1]
//   stochastic    entry[T] = min(random depth bits << 32 | slot), ecount[T]
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

namespace gspd {

constexpr float kPi = 3.14159265358979323846f;
constexpr int kSlotsPerPath = 32;

struct CamDev {
    float3 eye;
    double3 fwd, right, up;
    double th, aspect;
    int32_t w, h;
};

struct EmitDev {
    const float4* __restrict__ geo;  // 5 per emitter: v0, e1, e2, n, flux
    const float* __restrict__ cdf;
    int32_t n;
};

struct PassDev {
    int32_t tri_is_id;  // wavefront hits: 1 = upload-order triangle index, 0 = leaf-ordered slot
    const uint32_t* pass_dev;  // if set, the pass index is read here (replayed CUDA graphs)
    uint64_t seed;
    uint32_t scene_id, pass;
    float alpha, rr, eps, inv_h;
    int32_t max_eye, max_photon;
    uint32_t tmask;
    int64_t np;
};

// The pass index; in a replayed graph the device counter holds the graph's first pass and
// P.pass the pass's place in the graph.
__device__ __forceinline__ uint32_t pass_index(const PassDev& P) { return P.pass_dev ? *P.pass_dev + P.pass : P.pass; }

struct Material {
    float3 albedo, emission;
    int32_t type;
    float ior;
};

__device__ __forceinline__ Material load_mat(const DevScene& S, int32_t m) {
    const float4 a = __ldg(S.mats + 2 * m), b = __ldg(S.mats + 2 * m + 1);
    Material r;
    r.albedo = f3(a);
    r.type = __float_as_int(a.w);
    r.emission = f3(b);
    r.ior = b.w;
    return r;
}

__device__ __forceinline__ bool emits(const Material& m) {
    return (m.type == GSP_DIFFUSE || m.type == GSP_EMITTER) &&
           fmaxf(m.emission.x, fmaxf(m.emission.y, m.emission.z)) > 0.0f;
}

// Orthonormal basis about a unit vector (Duff et al., JCGT 2017).
__device__ __forceinline__ void onb(float3 n, float3& t1, float3& t2) {
    const float sign = copysignf(1.0f, n.z);
    const float a = -1.0f / (sign + n.z);
    const float b = n.x * n.y * a;
    t1 = make_float3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
    t2 = make_float3(b, sign + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ float3 cosine_dir(float3 n, float ua, float ub) {
    const float r = sqrtf(ua);
    const float z = sqrtf(fmaxf(0.0f, 1.0f - ua));
    float s, c;
    sincospif(2.0f * ub, &s, &c);  // angle 2 pi ub without rounding 2 pi ub first
    float3 t1, t2;
    onb(n, t1, t2);
    return madd3(n, z, madd3(t2, r * s, t1 * (r * c)));
}

__device__ __forceinline__ float3 reflect3(float3 d, float3 n) { return madd3(n, -2.0f * dot3(d, n), d); }

// Smooth dielectric: reflection with the exact unpolarised Fresnel probability, else refraction.
__device__ __forceinline__ float3 dielectric(float3 d, float3 n, float ior, float u) {
    const bool front = dot3(d, n) < 0.0f;
    const float3 nf = front ? n : n * -1.0f;
    const float n1 = front ? 1.0f : ior, n2 = front ? ior : 1.0f;
    const float eta = n1 / n2;
    const float cosi = -dot3(d, nf);
    const float k = 1.0f - eta * eta * (1.0f - cosi * cosi);
    if (k < 0.0f) return reflect3(d, nf);
    const float cost = sqrtf(k);
    const float rs = (n1 * cosi - n2 * cost) / (n1 * cosi + n2 * cost);
    const float rp = (n2 * cosi - n1 * cost) / (n2 * cosi + n1 * cost);
    const float F = 0.5f * (rs * rs + rp * rp);
    if (u < F) return reflect3(d, nf);
    return madd3(nf, __fmaf_rn(eta, cosi, -cost), d * eta);
}

// Octahedral unit-vector encoding, 2 x 16-bit snorm (Cigolle et al., JCGT 2014).
__device__ __forceinline__ uint32_t oct_encode(float3 v) {
    const float l1 = fabsf(v.x) + fabsf(v.y) + fabsf(v.z);
    float px = v.x / l1, py = v.y / l1;
    if (v.z < 0.0f) {
        const float ox = (1.0f - fabsf(py)) * copysignf(1.0f, px);
        const float oy = (1.0f - fabsf(px)) * copysignf(1.0f, py);
        px = ox;
        py = oy;
    }
    const int32_t qx = __float2int_rn(fminf(fmaxf(px, -1.0f), 1.0f) * 32767.0f);
    const int32_t qy = __float2int_rn(fminf(fmaxf(py, -1.0f), 1.0f) * 32767.0f);
    return ((uint32_t)(qx & 0xffff)) | ((uint32_t)(qy & 0xffff) << 16);
}

__device__ __forceinline__ float3 oct_decode(uint32_t e) {
    const float px = (float)(int16_t)(e & 0xffff) * (1.0f / 32767.0f);
    const float py = (float)(int16_t)(e >> 16) * (1.0f / 32767.0f);
    float3 v = make_float3(px, py, 1.0f - fabsf(px) - fabsf(py));
    const float t = fmaxf(-v.z, 0.0f);
    v.x += v.x >= 0.0f ? -t : t;
    v.y += v.y >= 0.0f ? -t : t;
    return normalize3(v);
}

// Teschner et al. 2003 spatial hash of an integer cell, 32-bit wraparound.
__device__ __forceinline__ uint32_t cell_hash(int32_t ix, int32_t iy, int32_t iz, uint32_t mask) {
    return (((uint32_t)ix * 73856093u) ^ ((uint32_t)iy * 19349663u) ^ ((uint32_t)iz * 83492791u)) & mask;
}

// Cell lattice shifted by 0.381966 of a cell so that axis-aligned walls at multiples of the
// cell size (e.g. a floor at 0) do not lie on cell boundaries.
constexpr float kCellOffset = 0.381966f;

__device__ __forceinline__ int32_t cell_of(float x, float inv_h) {
    return (int32_t)floorf(fmaf(x, inv_h, kCellOffset));
}

__device__ __forceinline__ uint32_t bucket_of(float3 x, float inv_h, uint32_t mask) {
    return cell_hash(cell_of(x.x, inv_h), cell_of(x.y, inv_h), cell_of(x.z, inv_h), mask);
}

// ------------------------------------------------------------------------------------------
// wavefront queues: a ray per entry plus the path state that continues after its hit
// ------------------------------------------------------------------------------------------
struct PathQ {
    float4* ray;   // 2 per entry: {o, tmin}, {d, tmax} (the closest-hit input layout)
    float4* w;     // eye: {throughput, pixel bits}; photon: {flux, path bits}
    int4* rng;     // PRNG state after the draws so far
    int32_t* meta; // depth | deposits << 8
    int32_t* tri;  // closest-hit output
    float* t;
};

// A wavefront hit given as a leaf-ordered triangle slot: t from the triangle's plane in
// double-float arithmetic (as in the persistent path kernel); returns the upload-order index.
__device__ __forceinline__ int32_t slot_refine(const DevScene& S, float3 o, float3 d, Hit& h) {
    h.slot = h.id;
    const int32_t id = __float_as_int(__ldg(S.tris + 3 * (int64_t)h.id).w);
    refine_plane(S.tris, S.shade, S.nlo, h.id, id, o, d, h.t);
    return id;
}

// Closest hit of a finished walk (trav_steps), t refined as above.
__device__ __forceinline__ Hit walk_hit(const DevScene& S, const Trav& st) {
    Hit h;
    h.id = st.best;
    h.t = st.tbest;
    h.u = h.v = 0.0f;
    h.slot = st.slot;
    if (st.slot >= 0) refine_plane(S.tris, S.shade, S.nlo, st.slot, h.id, st.o, st.d, h.t);
    return h;
}

// ------------------------------------------------------------------------------------------
// per-vertex shading data (Sec. 3.1's triangle: a normal and texture coordinates per vertex)
// ------------------------------------------------------------------------------------------
struct Surf {
    float3 ns;    // shading normal, in the geometric normal's hemisphere
    float3 tex;   // factor of a diffuse albedo (1 without a texture)
    bool smooth;  // ns blended from vertex normals
};

// Bilinear lookup with wrap-around of texture T = {first texel, w, h} at coordinates (s, t):
// texel (i, j) holds its value at the centre of [i/w, (i+1)/w) x [j/h, (j+1)/h).
__device__ __forceinline__ float3 tex_bilinear(const float4* __restrict__ texels, int4 T, float s, float t) {
    s = s - floorf(s);
    t = t - floorf(t);
    const float x = s * (float)T.y - 0.5f, y = t * (float)T.z - 0.5f;
    const float x0 = floorf(x), y0 = floorf(y);
    const float fx = x - x0, fy = y - y0;
    int i0 = (int)x0, j0 = (int)y0;  // -1 .. size - 1
    if (i0 < 0) i0 += T.y;
    if (j0 < 0) j0 += T.z;
    const int i1 = i0 + 1 == T.y ? 0 : i0 + 1, j1 = j0 + 1 == T.z ? 0 : j0 + 1;
    const float4* q = texels + T.x;
    const float3 a = f3(__ldg(q + (int64_t)j0 * T.y + i0)), b = f3(__ldg(q + (int64_t)j0 * T.y + i1));
    const float3 c = f3(__ldg(q + (int64_t)j1 * T.y + i0)), e = f3(__ldg(q + (int64_t)j1 * T.y + i1));
    const float gx = 1.0f - fx, gy = 1.0f - fy;
    return madd3(e, fx * fy, madd3(c, gx * fy, madd3(b, fx * gy, a * (gx * gy))));
}

// Shading from the per-vertex data of triangle `id` (vertices at leaf-ordered `slot`) for the
// hit of ray (o, d) with geometric unit normal n: barycentric weights (Moller-Trumbore's u, v
// for vertices 1 and 2; 1 - u - v for vertex 0), blended normal, texture lookup.
__device__ __forceinline__ Surf surface_attr(const float4* __restrict__ attr, const float4* __restrict__ tris,
                                          const float4* __restrict__ texels, const int4* __restrict__ mtex,
                                          int32_t slot, int32_t id, float3 o, float3 d, float3 n, bool diffuse,
                                          int32_t mid) {
    Surf sf;
    sf.ns = n;
    sf.tex = make_float3(1.0f, 1.0f, 1.0f);
    sf.smooth = false;
    const float4* tv = tris + 3 * (int64_t)slot;
    const float3 v0 = f3(__ldg(tv)), e1 = f3(__ldg(tv + 1)) - v0, e2 = f3(__ldg(tv + 2)) - v0;
    const float3 p = cross3(d, e2);
    const float f = 1.0f / dot3(e1, p);
    const float3 s0 = o - v0;
    const float b1 = f * dot3(s0, p), b2 = f * dot3(d, cross3(s0, e1)), b0 = 1.0f - b1 - b2;
    const float4* a = attr + 4 * (int64_t)id;
    const float4 a0 = __ldg(a), a1 = __ldg(a + 1), a2 = __ldg(a + 2), a3 = __ldg(a + 3);
    if (__float_as_int(a3.w) & 1) {
        float3 nb = madd3(f3(a2), b2, madd3(f3(a1), b1, f3(a0) * b0));
        const float l2 = dot3(nb, nb);
        if (l2 > 0.0f) {
            nb = nb * (1.0f / sqrtf(l2));
            sf.ns = dot3(nb, n) < 0.0f ? nb * -1.0f : nb;
            sf.smooth = true;
        }
    }
    if (mtex && diffuse) {
        const int4 T = __ldg(mtex + mid);
        if (T.y > 0) {
            const float s = __fmaf_rn(a2.w, b2, __fmaf_rn(a1.w, b1, a0.w * b0));
            const float t = __fmaf_rn(a3.z, b2, __fmaf_rn(a3.y, b1, a3.x * b0));
            sf.tex = tex_bilinear(texels, T, s, t);
        }
    }
    return sf;
}

// Shading at hit h of ray (o, d) with geometric unit normal n and material m (index mid).
// SHADE = false compiles the flat case only (kernels launched for scenes without shading data
// keep the registers of the plain path).
template <bool SHADE>
__device__ __forceinline__ Surf surface(const DevScene& S, const Hit& h, float3 o, float3 d, float3 n,
                                        const Material& m, int32_t mid) {
    if (SHADE && S.attr) return surface_attr(S.attr, S.tris, S.texels, S.mtex, h.slot, h.id, o, d, n, m.type == GSP_DIFFUSE, mid);
    Surf sf;
    sf.ns = n;
    sf.tex = make_float3(1.0f, 1.0f, 1.0f);
    sf.smooth = false;
    return sf;
}

// Appends the lanes with `keep` set to queue Q (warp-aggregated: one atomic per warp).
__device__ __forceinline__ void queue_push(const PathQ& Q, uint32_t* count, bool keep, float3 o, float tmin, float3 d,
                                           float3 w, int32_t tag, const Rng& rng, int32_t meta) {
    const uint32_t m = __ballot_sync(0xffffffffu, keep);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!keep) return;
    const uint32_t j = base + __popc(m & ((1u << lane) - 1u));
    Q.ray[2 * (size_t)j] = make_float4(o.x, o.y, o.z, tmin);
    Q.ray[2 * (size_t)j + 1] = make_float4(d.x, d.y, d.z, __int_as_float(0x7f800000));
    Q.w[j] = make_float4(w.x, w.y, w.z, __int_as_float(tag));
    Q.rng[j] = make_int4(rng.s[0], rng.s[1], rng.s[2], rng.s[3]);
    Q.meta[j] = meta;
}

__device__ __forceinline__ Rng rng_from(int4 v) {
    Rng r;
    r.s[0] = v.x;
    r.s[1] = v.y;
    r.s[2] = v.z;
    r.s[3] = v.w;
    return r;
}

// ------------------------------------------------------------------------------------------
// eye pass: jittered pinhole ray, specular chain, first non-specular hit (Sec. 2)
// ------------------------------------------------------------------------------------------
struct EyeOut {
    float4* __restrict__ hx;
    float4* __restrict__ hn;
    float4* __restrict__ hf;
    float4* __restrict__ hd;  // this pass's directly seen emission per pixel (added by the gather)
    float4* __restrict__ hw;  // optional: eye throughput w of each hit point (gradient replay)
};

// One eye-path interaction at a hit. Emission seen from the front is added to the pixel's
// direct term of this pass (one path per pixel, so no atomics);
// a diffuse hit records the hit point and ends the path; a mirror or dielectric bends the ray
// (returns true: the path continues from x along the new d).
template <bool SHADE>
__device__ __forceinline__ bool eye_interact(const DevScene& S, const PassDev& P, const EyeOut& O, int64_t p,
                                             const Hit& h, float3& o, float3& d, float3& w, Rng& rng) {
    const float4 sh = __ldg(S.shade + h.id);
    const float3 n = f3(sh);
    const int32_t mid = __float_as_int(sh.w);
    const Material m = load_mat(S, mid);
    const bool front = dot3(d, n) < 0.0f;
    if (front && emits(m)) {
        float4 v = O.hd[p];
        v.x += w.x * m.emission.x;
        v.y += w.y * m.emission.y;
        v.z += w.z * m.emission.z;
        O.hd[p] = v;
    }
    if (m.type == GSP_EMITTER) return false;
    const float3 x = madd3(d, h.t, o);
    const Surf sf = surface<SHADE>(S, h, o, d, n, m, mid);
    if (m.type == GSP_DIFFUSE) {
        const float3 ns = front ? n : n * -1.0f;
        const float3 wt = mul3(w, sf.tex);  // the hit point's weight without its albedo
        const float3 f = mul3(wt, m.albedo) * (1.0f / kPi);
        O.hx[p] = make_float4(x.x, x.y, x.z, __int_as_float(mid));
        O.hn[p] = make_float4(ns.x, ns.y, ns.z, 0.0f);
        O.hf[p] = make_float4(f.x, f.y, f.z, 0.0f);
        if (O.hw) O.hw[p] = make_float4(wt.x, wt.y, wt.z, 0.0f);
        return false;
    }
    if (m.type == GSP_MIRROR) {
        w = mul3(w, m.albedo);
        d = reflect3(d, sf.ns);
    } else {
        d = dielectric(d, sf.ns, m.ior, rng_next(rng));
    }
    o = x;
    return true;
}

// Primary rays: one per pixel, jittered inside the pixel; the queue starts in pixel order.
__global__ void __launch_bounds__(256)
k_eye_emit(CamDev C, PassDev P, PathQ Q, EyeOut O, uint32_t* __restrict__ qn, unsigned long long* __restrict__ trace_ctr,
           uint32_t* __restrict__ tail_ctr) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t npix = (int64_t)C.w * C.h;
    if (p == 0) {
        trace_ctr[0] = 0ull;
        qn[0] = (uint32_t)npix;
        qn[1] = 0;
        qn[2] = 0;
        *tail_ctr = 0;  // work counter of k_paths
    }
    if (p >= npix) return;
    const int px = (int)(p % C.w), py = (int)(p / C.w);
    Rng rng = rng_seed(P.seed, P.scene_id, 0u, pass_index(P), (uint64_t)p);
    const float u0 = rng_next(rng), u1 = rng_next(rng);
    // primary ray in FP64 (once per pixel), rounded once
    const double sx = (((double)px + u0) / (double)C.w * 2.0 - 1.0) * C.th * C.aspect;
    const double sy = (1.0 - ((double)py + u1) / (double)C.h * 2.0) * C.th;
    const double dx = C.fwd.x + C.right.x * sx + C.up.x * sy, dy = C.fwd.y + C.right.y * sx + C.up.y * sy,
                 dz = C.fwd.z + C.right.z * sx + C.up.z * sy;
    const double il = rsqrt(dx * dx + dy * dy + dz * dz);
    Q.ray[2 * p] = make_float4(C.eye.x, C.eye.y, C.eye.z, 0.0f);
    Q.ray[2 * p + 1] = make_float4((float)(dx * il), (float)(dy * il), (float)(dz * il), __int_as_float(0x7f800000));
    Q.w[p] = make_float4(1.0f, 1.0f, 1.0f, __int_as_float((int32_t)p));
    Q.rng[p] = make_int4(rng.s[0], rng.s[1], rng.s[2], rng.s[3]);
    Q.meta[p] = 0;
    O.hx[p] = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(-1));
    O.hd[p] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// Wavefront step b of the eye pass: shade the traced queue qn[b % 3], push continuing paths.
template <bool SHADE>
__global__ void __launch_bounds__(256)
k_eye_shade(DevScene S, PassDev P, PathQ cur, PathQ nxt, EyeOut O, uint32_t* __restrict__ qn, int b,
            unsigned long long* __restrict__ trace_ctr) {
    const uint32_t n = qn[b % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        qn[(b + 2) % 3] = 0;
        trace_ctr[0] = 0ull;  // for the next step's closest-hit launch
    }
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        bool keep = false;
        float3 o, d, w;
        Rng rng;
        int32_t p = 0, depth = 0;
        if (i < n) {
            const float4 a = cur.ray[2 * (size_t)i], c = cur.ray[2 * (size_t)i + 1], ww = cur.w[i];
            o = f3(a);
            d = f3(c);
            w = f3(ww);
            p = __float_as_int(ww.w);
            depth = cur.meta[i];
            rng = rng_from(cur.rng[i]);
            Hit h;
            h.id = cur.tri[i];
            h.t = cur.t[i];
            h.slot = -1;
            if (h.id >= 0 && !P.tri_is_id) h.id = slot_refine(S, o, d, h);
            if (h.id >= 0) {
                keep = eye_interact<SHADE>(S, P, O, p, h, o, d, w, rng) && depth + 1 <= P.max_eye;
            }
        }
        queue_push(nxt, qn + (b + 1) % 3, keep, o, P.eps, d, w, p, rng, depth + 1);
    }
}

// ------------------------------------------------------------------------------------------
// photon pass (Sec. 2 photon tracing; Sec. 3.3 one bounce per pass with regeneration)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void emit_photon(const EmitDev& E, Rng& rng, float3& o, float3& d, float3& phi) {
    const float u0 = rng_next(rng);
    int lo = 0, hi = E.n;  // first j with cdf[j] > u0
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(E.cdf + mid) > u0) hi = mid; else lo = mid + 1;
    }
    const int j = min(lo, E.n - 1);
    const float3 v0 = f3(__ldg(E.geo + 5 * j)), e1 = f3(__ldg(E.geo + 5 * j + 1)),
                 e2 = f3(__ldg(E.geo + 5 * j + 2)), n = f3(__ldg(E.geo + 5 * j + 3));
    phi = f3(__ldg(E.geo + 5 * j + 4));
    const float u1 = rng_next(rng), u2 = rng_next(rng);
    // point on the triangle in FP64 (once per path), rounded once
    const double su = sqrt((double)u1), b1 = su * (1.0 - (double)u2), b2 = su * (double)u2;
    o = make_float3((float)(v0.x + e1.x * b1 + e2.x * b2), (float)(v0.y + e1.y * b1 + e2.y * b2),
                    (float)(v0.z + e1.z * b1 + e2.z * b2));
    const float u3 = rng_next(rng), u4 = rng_next(rng);
    d = cosine_dir(n, u3, u4);
}

struct DepositDev {
    float4* __restrict__ slots;          // 2 float4 per slot
    uint32_t* __restrict__ pcount;       // deposits per path / thread
    unsigned long long* __restrict__ entry;  // stochastic: min key per bucket
    uint32_t* __restrict__ ecount;       // stochastic: photons per bucket
    int32_t stochastic;
    int32_t* __restrict__ smat;          // optional: material of each deposit's surface (gradient replay)
};

// One photon interaction at a hit. Returns false when the path ends.
template <bool SHADE>
__device__ __forceinline__ bool photon_bounce(const DevScene& S, const PassDev& P, const DepositDev& D,
                                              Rng& rng, const Hit& h, float3& o, float3& d, float3& phi,
                                              uint32_t id, uint32_t slot, uint32_t& ndep) {
    const float4 sh = __ldg(S.shade + h.id);
    const float3 n = f3(sh);
    const Material m = load_mat(S, __float_as_int(sh.w));
    if (m.type == GSP_EMITTER) return false;
    const float3 x = madd3(d, h.t, o);
    const Surf sf = surface<SHADE>(S, h, o, d, n, m, __float_as_int(sh.w));
    if (m.type == GSP_DIFFUSE) {
        if (D.smat) D.smat[slot] = __float_as_int(sh.w);
        float4* rec = D.slots + 2 * (size_t)slot;
        rec[0] = make_float4(x.x, x.y, x.z, __uint_as_float(id));
        rec[1] = make_float4(phi.x, phi.y, phi.z, __uint_as_float(oct_encode(d)));
        ++ndep;
        if (D.stochastic) {
            const float z = rng_next(rng);
            const uint32_t b = bucket_of(x, P.inv_h, P.tmask);
            const unsigned long long key = ((unsigned long long)__float_as_uint(z) << 32) | slot;
            atomicMin(D.entry + b, key);
            atomicAdd(D.ecount + b, 1u);
        }
        const float urr = rng_next(rng);
        if (!(urr < P.rr)) return false;
        phi = mul3(mul3(phi, m.albedo), sf.tex) * (1.0f / P.rr);
        const bool fr = dot3(d, n) < 0.0f;
        const float3 ns = fr ? sf.ns : sf.ns * -1.0f;
        const float ua = rng_next(rng), ub = rng_next(rng);
        d = cosine_dir(ns, ua, ub);
        // about a shading normal the direction can point into the surface: the path ends there
        if (sf.smooth && !(dot3(d, fr ? n : n * -1.0f) > 0.0f)) return false;
    } else if (m.type == GSP_MIRROR) {
        phi = mul3(phi, m.albedo);
        d = reflect3(d, sf.ns);
    } else {
        d = dielectric(d, sf.ns, m.ior, rng_next(rng));
    }
    o = x;
    return true;
}

// Photon paths: emission into the queue in path order (whole paths per pass).
__global__ void __launch_bounds__(256)
k_photon_emit(EmitDev E, PassDev P, PathQ Q, uint32_t* __restrict__ pcount, uint32_t* __restrict__ qn,
              unsigned long long* __restrict__ trace_ctr, uint32_t* __restrict__ tail_ctr) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) {
        trace_ctr[0] = 0ull;
        qn[0] = (uint32_t)P.np;
        qn[1] = 0;
        qn[2] = 0;
        *tail_ctr = 0;  // work counter of k_paths
    }
    if (k >= P.np) return;
    Rng rng = rng_seed(P.seed, P.scene_id, 1u, pass_index(P), (uint64_t)k);
    float3 o, d, phi;
    emit_photon(E, rng, o, d, phi);
    Q.ray[2 * k] = make_float4(o.x, o.y, o.z, P.eps);
    Q.ray[2 * k + 1] = make_float4(d.x, d.y, d.z, __int_as_float(0x7f800000));
    Q.w[k] = make_float4(phi.x, phi.y, phi.z, __int_as_float((int32_t)k));
    Q.rng[k] = make_int4(rng.s[0], rng.s[1], rng.s[2], rng.s[3]);
    Q.meta[k] = 0;
    pcount[k] = 0;
}

// Wavefront step b of the photon pass: shade the traced queue qn[b % 3] (deposit, Russian
// roulette, new direction) and push the paths that go on.
template <bool SHADE>
__global__ void __launch_bounds__(256)
k_photon_shade(DevScene S, PassDev P, DepositDev D, PathQ cur, PathQ nxt, uint32_t* __restrict__ qn, int b,
               unsigned long long* __restrict__ trace_ctr) {
    const uint32_t n = qn[b % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        qn[(b + 2) % 3] = 0;
        trace_ctr[0] = 0ull;  // for the next step's closest-hit launch
    }
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        bool keep = false;
        float3 o, d, phi;
        Rng rng;
        int32_t k = 0, depth = 0;
        uint32_t ndep = 0;
        if (i < n) {
            const float4 a = cur.ray[2 * (size_t)i], c = cur.ray[2 * (size_t)i + 1], ww = cur.w[i];
            o = f3(a);
            d = f3(c);
            phi = f3(ww);
            k = __float_as_int(ww.w);
            const int32_t meta = cur.meta[i];
            depth = meta & 0xff;
            ndep = (uint32_t)(meta >> 8);
            rng = rng_from(cur.rng[i]);
            Hit h;
            h.id = cur.tri[i];
            h.t = cur.t[i];
            h.slot = -1;
            if (h.id >= 0 && !P.tri_is_id) h.id = slot_refine(S, o, d, h);
            if (h.id >= 0) {
                const uint32_t id = (uint32_t)k * kSlotsPerPath + depth;
                const uint32_t slot = (uint32_t)k * kSlotsPerPath + ndep;
                const uint32_t before = ndep;
                keep = photon_bounce<SHADE>(S, P, D, rng, h, o, d, phi, id, slot, ndep) && depth + 1 < P.max_photon;
                if (ndep != before) D.pcount[k] = ndep;
            }
        }
        queue_push(nxt, qn + (b + 1) % 3, keep, o, P.eps, d, phi, k, rng, (depth + 1) | (int32_t)(ndep << 8));
    }
}

// The eye and photon paths left in their queues after the wavefront steps (all of them when
// there are none), finished by one persistent kernel: items [0, ne) are eye-queue entries,
// [ne, ne + nph) photon-queue entries. Each lane follows one path bounce by bounce and takes the
// next item as soon as its path ends (WarpQueue, counter *ctr), so the long specular eye paths,
// which start first, run beside the bulk of the photon work instead of after it. Eye entries
// have depth <= max_eye, photon entries depth < max_photon (the host launches accordingly).
// STACK: walk the child-pair layout with a stack (StackWalk) instead of the hit/miss links.
template <bool STACK, bool SHADE>
__global__ void __launch_bounds__(kTraceThreads, GSP_PATH_MIN_BLOCKS)
k_paths(DevScene S, PassDev P, PathQ qe, EyeOut O, const uint32_t* __restrict__ ne_ptr, PathQ qp, DepositDev D,
        const uint32_t* __restrict__ np_ptr, uint32_t* __restrict__ ctr) {
    const int32_t cap = trav_cap(S);
    const int32_t ne = ne_ptr ? (int32_t)*ne_ptr : 0;
    const int32_t nph = np_ptr ? (int32_t)*np_ptr : 0;
    WarpQueue wq;
    wq.init(ne + nph);
    Trav st;
    st.node = -1;
    st.slot = -1;
    int32_t i = -1, pend = -1, id = 0, depth = 0;
    uint32_t ndep = 0;
    bool eye = false;
    StackWalk sw;
    sw.node = kWalkDone;
    sw.sp = 0;
    float3 w = make_float3(0.0f, 0.0f, 0.0f);  // eye: throughput; photon: flux
    Rng rng;
    while (true) {
        const int32_t got = wq.take(i < 0, ctr);
        if (got >= 0) {
            i = got;
            eye = got < ne;
            const PathQ Q = eye ? qe : qp;
            const size_t j = (size_t)(eye ? got : got - ne);
            const float4 a = Q.ray[2 * j], c = Q.ray[2 * j + 1], ww = Q.w[j];
            const int32_t meta = Q.meta[j];
            w = f3(ww);
            id = __float_as_int(ww.w);
            rng = rng_from(Q.rng[j]);
            depth = eye ? meta : (meta & 0xff);
            ndep = eye ? 0u : (uint32_t)(meta >> 8);
            trav_init(S, f3(a), f3(c), eye ? a.w : P.eps, __int_as_float(0x7f800000), st);
            if (STACK) stack_init(S, sw);
        }
        if (__ballot_sync(0xffffffffu, i >= 0) == 0) break;
        if (STACK)
            stack_steps(S, st, sw, i >= 0, cap);
        else
            trav_steps(S, st, pend, i >= 0, cap);
        const bool walked = STACK ? sw.node == kWalkDone : (st.node < 0 && pend < 0);
        if (i >= 0 && walked) {
            const Hit h = walk_hit(S, st);
            float3 o = st.o, d = st.d;
            bool more = false;
            if (eye) {
                more = h.id >= 0 && eye_interact<SHADE>(S, P, O, id, h, o, d, w, rng) && ++depth <= P.max_eye;
            } else {
                if (h.id >= 0) {
                    const uint32_t pid = (uint32_t)id * kSlotsPerPath + depth;
                    const uint32_t slot = (uint32_t)id * kSlotsPerPath + ndep;
                    more = photon_bounce<SHADE>(S, P, D, rng, h, o, d, w, pid, slot, ndep) && ++depth < P.max_photon;
                }
                if (!more) D.pcount[id] = ndep;
            }
            if (more) {
                trav_init(S, o, d, P.eps, __int_as_float(0x7f800000), st);
                if (STACK) stack_init(S, sw);
            } else {
                i = -1;
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// the eye and photon paths of many renderers in one persistent launch (batched passes)
// ------------------------------------------------------------------------------------------
// One renderer's share of a fused launch: its scene, pass, queues and outputs, where its item
// counts live on the device, and its range of 64-item chunks in the launch's chunk sequence
// (sized by capacity; chunks past the pass's actual counts are skipped).
struct PathJob {
    DevScene S;
    PassDev P;
    PathQ qe, qp;
    EyeOut O;
    DepositDev D;
    const uint32_t* ne_ptr;  // null: no eye items
    const uint32_t* np_ptr;  // null: no photon items
    int32_t first_chunk, nchunks;
};

// Work distribution over the chunks of all jobs: as WarpQueue, but a chunk also names its job
// (found by binary search over the jobs' chunk ranges), and its items are that job's local
// item indices (eye items first, then photon items).
struct MultiQueue {
    int32_t total, static_end, pos, pend, job;
    bool done;

    __device__ __forceinline__ bool chunk(const PathJob* __restrict__ jobs, int32_t njobs, int32_t c) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].first_chunk <= c) lo = mid; else hi = mid - 1;
        }
        job = lo;
        const PathJob& J = jobs[lo];
        const int32_t items = (J.ne_ptr ? (int32_t)*J.ne_ptr : 0) + (J.np_ptr ? (int32_t)*J.np_ptr : 0);
        pos = (c - J.first_chunk) * kTraceChunk;
        pend = min(pos + kTraceChunk, items);
        return pos < pend;
    }

    __device__ __forceinline__ void init(const PathJob* __restrict__ jobs, int32_t njobs, int32_t total_chunks) {
        total = total_chunks;
        const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
        static_end = (int32_t)min(warps, (int64_t)total);
        const int32_t c = (int32_t)((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
        done = false;
        pos = pend = 0;
        job = 0;
        if (c < total) chunk(jobs, njobs, c);
    }

    // Lanes with `need` set receive the next item of some job (-1 when all are exhausted); the
    // job is `job` at the time of the return for every lane that received one in this call only
    // if no chunk change happened after its assignment, so it is returned per lane.
    __device__ __forceinline__ int32_t take(bool need, const PathJob* __restrict__ jobs, int32_t njobs, uint32_t* ctr,
                                            int32_t& item_job) {
        int32_t item = -1;
        const uint32_t lt = lanemask_lt();
        need = need && !done;
        uint32_t m = __ballot_sync(0xffffffffu, need);
        while (m) {
            while (pos >= pend) {
                uint32_t b = 0;
                if (static_end < total && (threadIdx.x & 31) == 0) b = atomicAdd(ctr, 1u);
                b = __shfl_sync(0xffffffffu, b, 0);
                const int64_t c = (int64_t)static_end + b;
                if (c >= total) {
                    done = true;
                    return item;
                }
                chunk(jobs, njobs, (int32_t)c);
            }
            const int take = min(__popc(m), pend - pos);
            const int rank = __popc(m & lt);
            if (need && rank < take) {
                item = pos + rank;
                item_job = job;
                need = false;
            }
            pos += take;
            m = __ballot_sync(0xffffffffu, need);
        }
        return item;
    }
};

template <bool STACK, bool SHADE>
__global__ void __launch_bounds__(kTraceThreads, GSP_PATH_MIN_BLOCKS)
k_paths_multi(const PathJob* __restrict__ jobs, int32_t njobs, int32_t total_chunks, uint32_t* __restrict__ ctr) {
    MultiQueue mq;
    mq.init(jobs, njobs, total_chunks);
    Trav st;
    st.node = -1;
    st.slot = -1;
    StackWalk sw;
    sw.node = kWalkDone;
    sw.sp = 0;
    int32_t i = -1, jb = 0, pend = -1, id = 0, depth = 0, cap = 0;
    uint32_t ndep = 0;
    bool eye = false;
    float3 w = make_float3(0.0f, 0.0f, 0.0f);  // eye: throughput; photon: flux
    Rng rng;
    while (true) {
        const int32_t got = mq.take(i < 0, jobs, njobs, ctr, jb);
        if (got >= 0) {
            const PathJob& J = jobs[jb];
            const int32_t ne = J.ne_ptr ? (int32_t)*J.ne_ptr : 0;
            i = got;
            eye = got < ne;
            const PathQ Q = eye ? J.qe : J.qp;
            const size_t j = (size_t)(eye ? got : got - ne);
            const float4 a = Q.ray[2 * j], c = Q.ray[2 * j + 1], ww = Q.w[j];
            const int32_t meta = Q.meta[j];
            w = f3(ww);
            id = __float_as_int(ww.w);
            rng = rng_from(Q.rng[j]);
            depth = eye ? meta : (meta & 0xff);
            ndep = eye ? 0u : (uint32_t)(meta >> 8);
            cap = trav_cap(J.S);
            trav_init(J.S, f3(a), f3(c), eye ? a.w : J.P.eps, __int_as_float(0x7f800000), st);
            if (STACK) stack_init(J.S, sw);
        }
        if (__ballot_sync(0xffffffffu, i >= 0) == 0) break;
        const PathJob& J = jobs[jb];
        if (STACK)
            stack_steps(J.S, st, sw, i >= 0, cap);
        else
            trav_steps(J.S, st, pend, i >= 0, cap);
        const bool walked = STACK ? sw.node == kWalkDone : (st.node < 0 && pend < 0);
        if (i >= 0 && walked) {
            const Hit h = walk_hit(J.S, st);
            float3 o = st.o, d = st.d;
            bool more = false;
            if (eye) {
                more = h.id >= 0 && eye_interact<SHADE>(J.S, J.P, J.O, id, h, o, d, w, rng) && ++depth <= J.P.max_eye;
            } else {
                if (h.id >= 0) {
                    const uint32_t pid = (uint32_t)id * kSlotsPerPath + depth;
                    const uint32_t slot = (uint32_t)id * kSlotsPerPath + ndep;
                    more = photon_bounce<SHADE>(J.S, J.P, J.D, rng, h, o, d, w, pid, slot, ndep) && ++depth < J.P.max_photon;
                }
                if (!more) J.D.pcount[id] = ndep;
            }
            if (more) {
                trav_init(J.S, o, d, J.P.eps, __int_as_float(0x7f800000), st);
                if (STACK) stack_init(J.S, sw);
            } else {
                i = -1;
            }
        }
    }
}

struct RegenDev {
    float4* __restrict__ ro;    // {o.xyz, depth bits}
    float4* __restrict__ rd;    // {d.xyz, alive bits}
    float4* __restrict__ rphi;  // {flux.rgb, 0}
    unsigned long long* __restrict__ started;
};

// One bounce per thread and pass (Sec. 3.3): thread j continues its stored path, or starts a new
// one when the stored path has ended (N_e counts the starts), traces exactly one ray, deposits at
// a diffuse hit and stores the path state for the next pass. Persistent, with per-lane refill
// over the threads (counter *ctr) as the path kernel; STACK as in k_paths.
template <bool STACK, bool SHADE>
__global__ void __launch_bounds__(kTraceThreads, GSP_PATH_MIN_BLOCKS)
k_photon_regen(DevScene S, EmitDev E, PassDev P, DepositDev D, RegenDev R, uint32_t* __restrict__ ctr) {
    const int32_t cap = trav_cap(S);
    WarpQueue wq;
    wq.init((int32_t)P.np);
    Trav st;
    st.node = -1;
    st.slot = -1;
    StackWalk sw;
    sw.node = kWalkDone;
    sw.sp = 0;
    int32_t j = -1, pend = -1, depth = 0;
    uint32_t starts = 0;
    float3 phi = make_float3(0.0f, 0.0f, 0.0f);
    Rng rng;
    while (true) {
        const int32_t got = wq.take(j < 0, ctr);
        if (got >= 0) {
            j = got;
            rng = rng_seed(P.seed, P.scene_id, 1u, pass_index(P), (uint64_t)j);
            const float4 a = R.ro[j], b = R.rd[j], c = R.rphi[j];
            float3 o = f3(a), d = f3(b);
            phi = f3(c);
            depth = __float_as_int(a.w);
            if (__float_as_int(b.w) == 0) {  // the stored path has ended: start a new one
                emit_photon(E, rng, o, d, phi);
                depth = 0;
                ++starts;
            }
            trav_init(S, o, d, P.eps, __int_as_float(0x7f800000), st);
            if (STACK) stack_init(S, sw);
        }
        if (__ballot_sync(0xffffffffu, j >= 0) == 0) break;
        if (STACK)
            stack_steps(S, st, sw, j >= 0, cap);
        else
            trav_steps(S, st, pend, j >= 0, cap);
        const bool walked = STACK ? sw.node == kWalkDone : (st.node < 0 && pend < 0);
        if (j >= 0 && walked) {
            const Hit h = walk_hit(S, st);
            float3 o = st.o, d = st.d;
            uint32_t ndep = 0;
            bool alive = h.id >= 0 && photon_bounce<SHADE>(S, P, D, rng, h, o, d, phi, (uint32_t)j, (uint32_t)j, ndep) &&
                         ++depth < P.max_photon;
            D.pcount[j] = ndep;
            R.ro[j] = make_float4(o.x, o.y, o.z, __int_as_float(depth));
            R.rd[j] = make_float4(d.x, d.y, d.z, __int_as_float(alive ? 1 : 0));
            R.rphi[j] = make_float4(phi.x, phi.y, phi.z, 0.0f);
            j = -1;
        }
    }
    // paths started by this warp
    for (int off = 16; off > 0; off >>= 1) starts += __shfl_xor_sync(0xffffffffu, starts, off);
    if ((threadIdx.x & 31) == 0 && starts) atomicAdd(R.started, (unsigned long long)starts);
}

// ------------------------------------------------------------------------------------------
// exact hash-grid deposit: compaction in id order, bucket keys, bucket counts
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_compact(const float4* __restrict__ slots, const uint32_t* __restrict__ pcount,
          const uint32_t* __restrict__ poff, int64_t np, int32_t slots_per_path, float inv_h,
          uint32_t tmask, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
          uint32_t* __restrict__ bcount) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np) return;
    const uint32_t c = pcount[k], off = poff[k];
    for (uint32_t i = 0; i < c; ++i) {
        const uint32_t slot = (uint32_t)k * slots_per_path + i;
        const float4 a = slots[2 * (size_t)slot];
        const uint32_t b = bucket_of(f3(a), inv_h, tmask);
        keys[off + i] = b;
        vals[off + i] = slot;
        atomicAdd(bcount + b, 1u);
    }
}

__global__ void __launch_bounds__(256)
k_permute(const float4* __restrict__ slots, const uint32_t* __restrict__ order,
          const uint32_t* __restrict__ d_n, float4* __restrict__ spos, float4* __restrict__ spay) {
    const int64_t n = *d_n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = order[i];
        spos[i] = slots[2 * (size_t)s];
        spay[i] = slots[2 * (size_t)s + 1];
    }
}

// ------------------------------------------------------------------------------------------
// range query + progressive density estimation (fused)
// ------------------------------------------------------------------------------------------
struct GatherDev {
    const float4* __restrict__ hx;
    const float4* __restrict__ hn;
    const float4* __restrict__ hf;
    const float4* __restrict__ hd;  // direct emission of this pass, folded into st1.xyz
    float4* __restrict__ st0;
    float4* __restrict__ st1;
    // exact
    const float4* __restrict__ spos;
    const float4* __restrict__ spay;
    const uint32_t* __restrict__ bstart;
    // stochastic
    const float4* __restrict__ slots;
    const unsigned long long* __restrict__ entry;
    const uint32_t* __restrict__ ecount;
    int64_t npix;
    float* __restrict__ rhist;  // optional: [pass][npix] radius each pixel gathered with (gradient)
    float4* __restrict__ shist; // optional: [pass][npix] sum of the gathered photons' flux (gradient)
};

// Distinct buckets of the cells that overlap the ball of radius R about x. A photon within R
// lies in one of these cells, so visiting each distinct bucket once finds every such photon
// exactly once (photons of colliding cells fail the distance test).
__device__ __forceinline__ int query_buckets(float3 x, float R, float inv_h, uint32_t mask, uint32_t* out) {
    const float Rq = R * 1.00001f;
    int32_t lo[3], hi[3];
    const float xs[3] = {x.x, x.y, x.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = cell_of(xs[a] - Rq, inv_h);
        hi[a] = cell_of(xs[a] + Rq, inv_h);
        hi[a] = min(hi[a], lo[a] + 2);
    }
    int nb = 0;
    for (int32_t ix = lo[0]; ix <= hi[0]; ++ix)
        for (int32_t iy = lo[1]; iy <= hi[1]; ++iy)
            for (int32_t iz = lo[2]; iz <= hi[2]; ++iz) {
                const uint32_t b = cell_hash(ix, iy, iz, mask);
                bool dup = false;
                for (int q = 0; q < nb; ++q) dup |= out[q] == b;
                if (!dup) out[nb++] = b;
            }
    return nb;
}

// The photon acceptance test of the range query, with explicit rounding so that the adjoint
// replay decides exactly as the forward gather did: |x_k - x_p|^2 < R^2 and w_in . n_p < 0.
__device__ __forceinline__ bool photon_accept(float3 xk, float3 xp, float R, uint32_t dir, float3 n) {
    const float dx = __fsub_rn(xk.x, xp.x), dy = __fsub_rn(xk.y, xp.y), dz = __fsub_rn(xk.z, xp.z);
    const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    if (!(d2 < __fmul_rn(R, R))) return false;
    const float3 w = oct_decode(dir);
    return __fmaf_rn(w.z, n.z, __fmaf_rn(w.y, n.y, __fmul_rn(w.x, n.x))) < 0.0f;
}

__device__ __forceinline__ void add_direct(float4& s1, float4 d) {
    s1.x += d.x;
    s1.y += d.y;
    s1.z += d.z;
}

__device__ __forceinline__ void progressive_update(float4& s0, float4& s1, float M, float3 Phi, float alpha) {
    if (!(M > 0.0f)) return;
    const float N = s0.w;
    const float Nn = N + alpha * M;
    const float ratio = Nn / (N + M);
    s1.w = s1.w * sqrtf(ratio);
    s0.x = (s0.x + Phi.x) * ratio;
    s0.y = (s0.y + Phi.y) * ratio;
    s0.z = (s0.z + Phi.z) * ratio;
    s0.w = Nn;
}

// Cells overlapping the box x +- R along one axis. The box is widened by a few ulps of |x| so
// that a photon which the rounded distance test accepts always lies in one of its cells.
__device__ __forceinline__ void cell_range(float x, float R, float inv_h, int32_t& lo, int32_t& hi) {
    const float Rq = fmaf(R, 1.0001f, (fabsf(x) + R) * 4.8e-7f);
    lo = cell_of(x - Rq, inv_h);
    hi = cell_of(x + Rq, inv_h);
}

// Stochastic range query + progressive update, one hit point per thread: each distinct bucket
// of the at most 3 x 3 x 3 query cells once, its survivor weighted by the bucket's count (the
// cell edge is >= 2 r0 in this mode).
__global__ void __launch_bounds__(128) k_gather_stoch(GatherDev G, PassDev P) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= G.npix) return;
    const float4 hxp = G.hx[p];
    float4 s1 = G.st1[p];
    add_direct(s1, G.hd[p]);
    if (__float_as_int(hxp.w) < 0) {
        G.st1[p] = s1;
        return;
    }
    const float3 x = f3(hxp);
    const float3 n = f3(G.hn[p]);
    const float3 f = f3(G.hf[p]);
    float4 s0 = G.st0[p];
    const float R = s1.w;
    if (G.rhist) G.rhist[(size_t)pass_index(P) * G.npix + p] = R;
    float M = 0.0f;
    float3 acc = make_float3(0.0f, 0.0f, 0.0f);
    uint32_t buckets[27];
    const int nb = query_buckets(x, R, P.inv_h, P.tmask, buckets);
    for (int q = 0; q < nb; ++q) {
        const uint32_t b = buckets[q];
        const uint32_t cnt = G.ecount[b];
        if (cnt == 0) continue;
        const uint32_t slot = (uint32_t)(G.entry[b] & 0xffffffffull);
        const float4 a = __ldg(G.slots + 2 * (size_t)slot);
        const float4 c = __ldg(G.slots + 2 * (size_t)slot + 1);
        if (!photon_accept(f3(a), x, R, __float_as_uint(c.w), n)) continue;
        const float w = (float)cnt;
        M += w;
        acc = acc + f3(c) * w;
    }
    if (G.shist) G.shist[(size_t)pass_index(P) * G.npix + p] = make_float4(acc.x, acc.y, acc.z, 0.0f);
    progressive_update(s0, s1, M, mul3(f, acc), P.alpha);
    G.st0[p] = s0;
    G.st1[p] = s1;
}

// Exact range query + progressive update, a group of L lanes per hit point. The group visits
// every cell overlapping the box x +- R (any number per axis, so the cell may be smaller than the
// radius); its lanes split each bucket's photons (consecutive, coalesced), and a photon that passes
// the distance test counts only while its own cell is the one being visited, so a photon whose
// bucket several visited cells share (hash collisions) counts once. Lane sums are combined by a
// fixed butterfly, so the result does not depend on scheduling.
template <int L>
__global__ void __launch_bounds__(128) k_gather_exact(GatherDev G, PassDev P) {
    static_assert(L >= 1 && L <= 32 && (L & (L - 1)) == 0, "group size");
    const int gl = threadIdx.x & (L - 1);
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / L;
    if (p >= G.npix) return;
    const float4 hxp = G.hx[p];
    if (__float_as_int(hxp.w) < 0) {  // the whole group leaves together
        if (gl == 0) {
            float4 s1 = G.st1[p];
            add_direct(s1, G.hd[p]);
            G.st1[p] = s1;
        }
        return;
    }
    const float3 x = f3(hxp);
    const float3 n = f3(G.hn[p]);
    const float R = G.st1[p].w, R2p = R * R * 1.0001f;  // cheap pre-test, then the exact one
    int32_t lx, hx, ly, hy, lz, hz;
    cell_range(x.x, R, P.inv_h, lx, hx);
    cell_range(x.y, R, P.inv_h, ly, hy);
    cell_range(x.z, R, P.inv_h, lz, hz);
    float M = 0.0f;
    float3 acc = make_float3(0.0f, 0.0f, 0.0f);
    for (int32_t ix = lx; ix <= hx; ++ix)
        for (int32_t iy = ly; iy <= hy; ++iy)
            for (int32_t iz = lz; iz <= hz; ++iz) {
                const uint32_t b = cell_hash(ix, iy, iz, P.tmask);
                const uint32_t e = __ldg(G.bstart + b + 1);
                for (uint32_t i = __ldg(G.bstart + b) + gl; i < e; i += L) {
                    const float4 a = __ldg(G.spos + i);
                    const float3 dx = f3(a) - x;
                    if (!(dot3(dx, dx) < R2p)) continue;
                    if (cell_of(a.x, P.inv_h) != ix || cell_of(a.y, P.inv_h) != iy || cell_of(a.z, P.inv_h) != iz)
                        continue;  // a colliding cell's photon, counted when its own cell is visited
                    const float4 c = __ldg(G.spay + i);
                    if (!photon_accept(f3(a), x, R, __float_as_uint(c.w), n)) continue;
                    M += 1.0f;
                    acc = acc + f3(c);
                }
            }
    if (L > 1) {
        const int lane = threadIdx.x & 31;
        const uint32_t gmask = (L == 32 ? 0xffffffffu : ((1u << L) - 1u)) << (lane & ~(L - 1));
#pragma unroll
        for (int off = L / 2; off > 0; off >>= 1) {
            M += __shfl_xor_sync(gmask, M, off, L);
            acc.x += __shfl_xor_sync(gmask, acc.x, off, L);
            acc.y += __shfl_xor_sync(gmask, acc.y, off, L);
            acc.z += __shfl_xor_sync(gmask, acc.z, off, L);
        }
    }
    if (gl != 0) return;
    if (G.rhist) G.rhist[(size_t)pass_index(P) * G.npix + p] = R;
    if (G.shist) G.shist[(size_t)pass_index(P) * G.npix + p] = make_float4(acc.x, acc.y, acc.z, 0.0f);
    float4 s0 = G.st0[p], s1 = G.st1[p];
    add_direct(s1, G.hd[p]);
    progressive_update(s0, s1, M, mul3(f3(G.hf[p]), acc), P.alpha);
    G.st0[p] = s0;
    G.st1[p] = s1;
}

// ------------------------------------------------------------------------------------------
// adjoint (gradient of an image loss w.r.t. diffuse albedos and emission) by pass replay
// ------------------------------------------------------------------------------------------
constexpr int kMaxGradMats = 64;

struct AdjDev {
    const float4* __restrict__ hx;      // replayed hit points: x, material bits (< 0: none)
    const float4* __restrict__ hn;
    const float4* __restrict__ hf;      // w * albedo / pi
    const float4* __restrict__ hw;      // w (eye throughput)
    const float* __restrict__ rhist;    // radius each pixel gathered with in this pass
    const float* __restrict__ g;        // dLoss/dL [npix][3]
    const uint32_t* __restrict__ hp_order;   // hit-point grid: pixel at each sorted position
    const uint32_t* __restrict__ hp_bstart;
    uint32_t hp_mask;
    float inv_hp;                       // 1 / hit-point cell size
    float rmax;                         // largest gather radius (r0)
    const float4* __restrict__ spos;    // deposits of the pass, bucket-sorted
    const float4* __restrict__ spay;
    const uint32_t* __restrict__ order; // sorted deposit -> photon slot
    const uint32_t* __restrict__ d_total;
    float4* __restrict__ badj;          // per slot: B_k, the weight of Phi_k in the loss
};

// Photon-centric adjoint gather. For deposit k the hit points that gathered it in the forward
// pass (same acceptance test, same radii) give B_k = sum_p g_p (w rho / pi)_p / R_p^2, the weight
// of Phi_k in the loss. A group of L lanes serves one deposit: it visits the hit-point grid's cells
// overlapping xk +- r0 (no radius exceeds r0), its lanes split each bucket's hit points, and a hit
// point counts only in its own cell. Group sums combine by a fixed butterfly; nothing is atomic.
template <int L>
__global__ void __launch_bounds__(128) k_adj_photons(AdjDev A) {
    const int nd = (int)*A.d_total;
    const int gl = threadIdx.x & (L - 1);
    const int lane = threadIdx.x & 31;
    const uint32_t gmask = (L == 32 ? 0xffffffffu : ((1u << L) - 1u)) << (lane & ~(L - 1));
    const int groups = (int)(((int64_t)gridDim.x * blockDim.x) / L);
    for (int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / L); i < nd; i += groups) {
        const float4 a = A.spos[i], c = A.spay[i];
        const float3 xk = f3(a);
        const uint32_t dir = __float_as_uint(c.w);
        int32_t lx, hx, ly, hy, lz, hz;
        cell_range(xk.x, A.rmax, A.inv_hp, lx, hx);
        cell_range(xk.y, A.rmax, A.inv_hp, ly, hy);
        cell_range(xk.z, A.rmax, A.inv_hp, lz, hz);
        float3 B = make_float3(0.0f, 0.0f, 0.0f);
        for (int32_t ix = lx; ix <= hx; ++ix)
            for (int32_t iy = ly; iy <= hy; ++iy)
                for (int32_t iz = lz; iz <= hz; ++iz) {
                    const uint32_t b = cell_hash(ix, iy, iz, A.hp_mask);
                    const uint32_t e = __ldg(A.hp_bstart + b + 1);
                    for (uint32_t j = __ldg(A.hp_bstart + b) + gl; j < e; j += L) {
                        const uint32_t p = __ldg(A.hp_order + j);
                        const float4 hxp = __ldg(A.hx + p);
                        if (__float_as_int(hxp.w) < 0) continue;
                        if (cell_of(hxp.x, A.inv_hp) != ix || cell_of(hxp.y, A.inv_hp) != iy ||
                            cell_of(hxp.z, A.inv_hp) != iz)
                            continue;
                        const float R = __ldg(A.rhist + p);
                        if (!photon_accept(xk, f3(hxp), R, dir, f3(__ldg(A.hn + p)))) continue;
                        const float3 gp =
                            make_float3(__ldg(A.g + 3 * p), __ldg(A.g + 3 * p + 1), __ldg(A.g + 3 * p + 2));
                        B = B + mul3(gp, f3(__ldg(A.hf + p))) * (1.0f / (R * R));
                    }
                }
#pragma unroll
        for (int off = L / 2; off > 0; off >>= 1) {
            B.x += __shfl_xor_sync(gmask, B.x, off, L);
            B.y += __shfl_xor_sync(gmask, B.y, off, L);
            B.z += __shfl_xor_sync(gmask, B.z, off, L);
        }
        if (gl == 0) A.badj[A.order[i]] = make_float4(B.x, B.y, B.z, 0.0f);
    }
}

// Hit-point albedo terms: through the factor rho_{m_p} of its weight, pixel p gives
// dLoss/drho_{m_p} += g_p (w_p / pi) S_p / R_p^2, with S_p the flux sum its forward gather saw.
__global__ void __launch_bounds__(256)
k_adj_pixels(const float4* __restrict__ hx, const float4* __restrict__ hw, const float* __restrict__ rhist,
             const float4* __restrict__ shist, const float* __restrict__ g, int64_t npix, double* __restrict__ acc,
             int32_t nmat) {
    __shared__ float s_acc[kMaxGradMats * 3];
    for (int i = threadIdx.x; i < nmat * 3; i += blockDim.x) s_acc[i] = 0.0f;
    __syncthreads();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t m = __float_as_int(hx[p].w);
        if (m < 0) continue;
        const float R = rhist[p];
        const float3 t = mul3(mul3(make_float3(g[3 * p], g[3 * p + 1], g[3 * p + 2]), f3(hw[p])), f3(shist[p])) *
                         (1.0f / (kPi * R * R));
        atomicAdd(&s_acc[3 * m], t.x);
        atomicAdd(&s_acc[3 * m + 1], t.y);
        atomicAdd(&s_acc[3 * m + 2], t.z);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nmat * 3; i += blockDim.x)
        if (s_acc[i] != 0.0f) atomicAdd(&acc[i], (double)s_acc[i]);
}

// Path terms: Phi_j of deposit j carries rho_m / p_c for every diffuse bounce on material m before
// it, so dLoss/drho_m gains sum over those bounces b of (sum_{j > b} B_j Phi_j) / rho_m (per
// channel; channels with rho = 0 are skipped). A reverse walk over each path's deposits keeps
// that suffix sum.
__global__ void __launch_bounds__(128)
k_adj_paths(const float4* __restrict__ slots, const uint32_t* __restrict__ pcount, const int32_t* __restrict__ smat,
            const float4* __restrict__ badj, const float4* __restrict__ mats, int64_t np, double* __restrict__ acc,
            int32_t nmat) {
    __shared__ float s_acc[kMaxGradMats * 3];
    for (int i = threadIdx.x; i < nmat * 3; i += blockDim.x) s_acc[i] = 0.0f;
    __syncthreads();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t n = (int32_t)pcount[k];
        float3 suffix = make_float3(0.0f, 0.0f, 0.0f);
        for (int32_t j = n - 1; j >= 0; --j) {
            const size_t slot = (size_t)k * kSlotsPerPath + j;
            const int32_t m = smat[slot];
            if (j < n - 1) {
                const float3 al = f3(__ldg(mats + 2 * m));
                if (al.x > 0.0f) atomicAdd(&s_acc[3 * m], suffix.x / al.x);
                if (al.y > 0.0f) atomicAdd(&s_acc[3 * m + 1], suffix.y / al.y);
                if (al.z > 0.0f) atomicAdd(&s_acc[3 * m + 2], suffix.z / al.z);
            }
            suffix = suffix + mul3(f3(badj[slot]), f3(slots[2 * slot + 1]));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nmat * 3; i += blockDim.x)
        if (s_acc[i] != 0.0f) atomicAdd(&acc[i], (double)s_acc[i]);
}

// Emission: with one emitting material the image is linear in its Le, so dLoss/dLe_c is
// sum_p g_pc L_pc / Le_c; this kernel sums g * L.
__global__ void __launch_bounds__(256)
k_adj_emission(const float4* __restrict__ st0, const float4* __restrict__ st1, const float* __restrict__ g,
               int64_t npix, float inv_passes, double ne, double* __restrict__ acc_le) {
    __shared__ double s[3];
    if (threadIdx.x < 3) s[threadIdx.x] = 0.0;
    __syncthreads();
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const float4 t = st0[p], d = st1[p];
        const double k = 1.0 / ((double)kPi * (double)d.w * (double)d.w * ne);
        a0 += (double)g[3 * p] * ((double)d.x * inv_passes + (double)t.x * k);
        a1 += (double)g[3 * p + 1] * ((double)d.y * inv_passes + (double)t.y * k);
        a2 += (double)g[3 * p + 2] * ((double)d.z * inv_passes + (double)t.z * k);
    }
    atomicAdd(&s[0], a0);
    atomicAdd(&s[1], a1);
    atomicAdd(&s[2], a2);
    __syncthreads();
    if (threadIdx.x < 3) atomicAdd(&acc_le[threadIdx.x], s[threadIdx.x]);
}

__global__ void k_adj_finalize(const double* __restrict__ acc, int32_t nmat, double scale, float4 le,
                               float* __restrict__ out_albedo, float* __restrict__ out_le) {
    for (int i = threadIdx.x; i < nmat * 3; i += blockDim.x) out_albedo[i] = (float)(acc[i] * scale);
    if (threadIdx.x < 3) {
        const double l = threadIdx.x == 0 ? le.x : (threadIdx.x == 1 ? le.y : le.z);
        out_le[threadIdx.x] = l > 0.0 ? (float)(acc[nmat * 3 + threadIdx.x] / l) : 0.0f;
    }
}

__global__ void k_image(const float4* __restrict__ st0, const float4* __restrict__ st1, int64_t npix,
                        float inv_passes, double ne_host, const unsigned long long* __restrict__ ne_dev,
                        float* __restrict__ rgb) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const double ne = ne_dev ? (double)*ne_dev : ne_host;
    const float4 a = st0[p], b = st1[p];
    const float k = ne > 0.0 ? (float)(1.0 / ((double)kPi * (double)b.w * (double)b.w * ne)) : 0.0f;
    rgb[3 * p] = b.x * inv_passes + a.x * k;
    rgb[3 * p + 1] = b.y * inv_passes + a.y * k;
    rgb[3 * p + 2] = b.z * inv_passes + a.z * k;
}

__global__ void k_state(const float4* __restrict__ st0, const float4* __restrict__ st1, int64_t npix,
                        float* N, float* R, float* tau, float* direct) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const float4 a = st0[p], b = st1[p];
    if (N) N[p] = a.w;
    if (R) R[p] = b.w;
    if (tau) { tau[3 * p] = a.x; tau[3 * p + 1] = a.y; tau[3 * p + 2] = a.z; }
    if (direct) { direct[3 * p] = b.x; direct[3 * p + 1] = b.y; direct[3 * p + 2] = b.z; }
}

__global__ void k_init_state(float4* st0, float4* st1, int64_t npix, float r0) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    st0[p] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    st1[p] = make_float4(0.0f, 0.0f, 0.0f, r0);
}

// Bucket key of each point of a hash-grid build; counts per bucket. With skip_invalid, points
// whose w holds a negative integer (hit points of pixels that saw no diffuse surface) get the key
// T = mask + 1: they sort after every bucket and are in none.
__global__ void k_grid_keys(const float4* __restrict__ pos, int64_t n, float inv_h, uint32_t mask,
                            uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, uint32_t* __restrict__ bcount,
                            int32_t skip_invalid) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 q = pos[i];
        vals[i] = (uint32_t)i;
        if (skip_invalid && __float_as_int(q.w) < 0) {
            keys[i] = mask + 1u;
            continue;
        }
        const uint32_t b = bucket_of(f3(q), inv_h, mask);
        keys[i] = b;
        atomicAdd(bcount + b, 1u);
    }
}

__global__ void k_store_u32(uint32_t* p, uint32_t v) { *p = v; }

__global__ void k_add_u32(uint32_t* p, uint32_t v) { *p += v; }

__global__ void k_fill_u64(unsigned long long* p, int64_t n, unsigned long long v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

}  // namespace gspd

// ============================================================================================
// host side
// ============================================================================================
using namespace gspd;

int64_t gsp_grid_scratch_words(int64_t n, int64_t T);
gsp_status gsp_grid_build_with(const float4* pos, int64_t n, float cell_h, int64_t T, uint32_t* order,
                               uint32_t* bstart, uint32_t* scratch, cudaStream_t st, bool skip_invalid);

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
    // tuning
    int32_t gather_lanes = 8;  // lanes per hit point in the exact gather
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
    (void)cudaGetLastError();  // drop a stale error left by an unrelated earlier runtime call
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
    {  // camera basis in FP64, rounded once
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
        r->cam.fwd = make_double3(f[0], f[1], f[2]);
        r->cam.right = make_double3(rt[0], rt[1], rt[2]);
        r->cam.up = make_double3(up[0], up[1], up[2]);
        r->cam.th = std::tan((double)c.vfov_deg * M_PI / 180.0 / 2.0);
        r->cam.aspect = (double)c.width / (double)c.height;
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
    } else {
        A(&r->entry, r->T);
        A(&r->ecount, r->T);
    }
    r->qcap = std::max(r->npix, P.photon_mode == GSP_FULL_PATH ? r->np : (int64_t)0);
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
    // exact mode traces several passes into both trace sets: the second one is made now, so
    // that no pass allocates
    if (e == cudaSuccess && P.hash_mode == GSP_EXACT) {
        const gsp_status se = ensure_second_buffer(r);
        if (se != GSP_OK) {
            gsp_sppm_destroy(r);
            return se;
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        gsp_set_last_error(cudaGetErrorString(e));
        free_all(r);
        delete r;
        return e == cudaErrorMemoryAllocation ? GSP_ERR_OOM : GSP_ERR_CUDA;
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
    return P;
}

// Renderer counters (uint32): [0] deposits of the pass, [7] first pass index of a replayed graph.
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

// Grid of k_paths: resident blocks on every SM, but no more warps than items.
static int path_grid(int64_t items, int device, bool stack) {
    static int per_sm[2][64] = {{0}};
    static int sms[64] = {0};
    if (device < 0 || device >= 64) device = 0;
    if (!per_sm[stack][device]) {
        int b = 0;
        cudaDeviceGetAttribute(&sms[device], cudaDevAttrMultiProcessorCount, device);
        if (stack)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_paths<true, false>, kTraceThreads, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_paths<false, false>, kTraceThreads, 0);
        per_sm[stack][device] = std::max(1, b);
    }
    const int64_t full = (int64_t)std::max(1, sms[device]) * per_sm[stack][device];
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
        const unsigned grid = (unsigned)path_grid(r->np, r->scene->ctx->device, stack);
        if (stack)
            S.attr ? k_photon_regen<true, true><<<grid, kTraceThreads, 0, st>>>(S, E, P, D, R, r->qctr + 13)
                   : k_photon_regen<true, false><<<grid, kTraceThreads, 0, st>>>(S, E, P, D, R, r->qctr + 13);
        else
            S.attr ? k_photon_regen<false, true><<<grid, kTraceThreads, 0, st>>>(S, E, P, D, R, r->qctr + 13)
                   : k_photon_regen<false, false><<<grid, kTraceThreads, 0, st>>>(S, E, P, D, R, r->qctr + 13);
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
    J.nchunks = (int32_t)((items + kTraceChunk - 1) / kTraceChunk);
    return GSP_OK;
}

static gsp_status stage_paths(gsp_sppm* r, const PassDev& P, const EyeOut& O, const DepositDev& D, cudaStream_t st) {
    NvtxRange nvtx("gsp: eye + photon paths");
    PathJob J;
    gsp_status e = paths_front(r, P, O, D, st, J);
    if (e != GSP_OK) return e;
    if (J.nchunks > 0) {
        const bool stack = r->traversal == GSP_TRAVERSAL_STACK;
        const unsigned grid = (unsigned)path_grid((int64_t)J.nchunks * kTraceChunk, r->scene->ctx->device, stack);
        if (stack)
            J.S.attr ? k_paths<true, true><<<grid, kTraceThreads, 0, st>>>(J.S, P, J.qe, O, J.ne_ptr, J.qp, D, J.np_ptr, r->qctr + 12)
                     : k_paths<true, false><<<grid, kTraceThreads, 0, st>>>(J.S, P, J.qe, O, J.ne_ptr, J.qp, D, J.np_ptr, r->qctr + 12);
        else
            J.S.attr ? k_paths<false, true><<<grid, kTraceThreads, 0, st>>>(J.S, P, J.qe, O, J.ne_ptr, J.qp, D, J.np_ptr, r->qctr + 12)
                     : k_paths<false, false><<<grid, kTraceThreads, 0, st>>>(J.S, P, J.qe, O, J.ne_ptr, J.qp, D, J.np_ptr, r->qctr + 12);
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
        launch_gather_exact(r->gather_lanes, G, P, r->npix, st);
    }
    GSP_CUDA_TRY(cudaGetLastError());
    return GSP_OK;
}

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
    if (r->tb[1].hx && r->tb[1].qctr && (!r->grad || r->tb[1].hw)) return GSP_OK;
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
    if (!r->tb[1].qctr) alloc_trace_queues(r, 1, A);
    for (cudaStream_t& t : r->tstream)
        if (e == cudaSuccess && !t) e = cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&r->ev_start, &r->ev_traced[0], &r->ev_traced[1], &r->ev_free[0], &r->ev_free[1]})
        if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        gsp_set_last_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? GSP_ERR_OOM : GSP_ERR_CUDA;
    }
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
    r->eye_steps = eye_steps;
    r->photon_steps = photon_steps;
    r->refine_factor = refine_factor;
    if (gather_lanes) r->gather_lanes = gather_lanes;
    if (traversal) r->traversal = traversal;
    return GSP_OK;
}

gsp_status gsp_sppm_pass(gsp_sppm* r, int32_t npasses, void* stream) {
    if (!r || npasses < 0) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(r->scene->ctx->device));
    (void)cudaGetLastError();  // drop a stale error left by an unrelated earlier runtime call
    gsp_status s = check_grad_room(r, npasses);
    if (s != GSP_OK) return s;
    if (npasses >= 2 && r->P.hash_mode == GSP_EXACT) return passes_overlapped(r, npasses, (cudaStream_t)stream);
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
    if (e != cudaSuccess) {
        gsp_set_last_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? GSP_ERR_OOM : GSP_ERR_CUDA;
    }
    r->grad = true;
    r->grad_max_passes = max_passes;
    r->emit_mat = em;
    use_buf(r, r->cur);
    return GSP_OK;
}

gsp_status gsp_render_grad(gsp_sppm* r, const float* d_dloss_dimg, float* d_grad_albedo, float* d_grad_emission,
                           void* stream) {
    if (!r || !d_dloss_dimg || !d_grad_albedo || !d_grad_emission) return GSP_ERR_INVALID_ARG;
    (void)cudaGetLastError();
    if (!r->grad || r->passes < 1) return GSP_ERR_BAD_STATE;
    GSP_CUDA_TRY(cudaSetDevice(r->scene->ctx->device));
    (void)cudaGetLastError();
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
        e = stage_deposit(r, P, st);
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
        k_adj_photons<8><<<grid * 8, 128, 0, st>>>(A);
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
};

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
            const unsigned grid = (unsigned)path_grid((int64_t)total[k] * kTraceChunk, b->device, stack);
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
    if (ce != cudaSuccess) {
        gsp_set_last_error(cudaGetErrorString(ce));
        return GSP_ERR_CUDA;
    }
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
    if (ce != cudaSuccess) {
        gsp_set_last_error(cudaGetErrorString(ce));
        return GSP_ERR_CUDA;
    }
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
        gsp_set_last_error(cudaGetErrorString(e));
        batch_free(b);
        return GSP_ERR_CUDA;
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
    (void)cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    for (gsp_sppm* r : b->rs)
        if (r->grad && r->passes + npasses > r->grad_max_passes) return GSP_ERR_OVERFLOW;
    if (npasses == 0) return GSP_OK;
    // pairs of passes as two-pass graphs where they apply, the rest one pass per graph
    const int32_t pairs = batch_pairs(b) ? npasses / 2 : 0, singles = npasses - 2 * pairs;
    if (pairs > 0 && !b->exec2) {
        gsp_status e = batch_capture_fused(b, b->cap, 2, &b->exec2);  // capture runs nothing
        if (e != GSP_OK) return e;
    }
    if (singles > 0 && !b->exec) {
        gsp_status e = batch_capture(b, b->cap);  // capture runs nothing; the graph launches on st
        if (e != GSP_OK) return e;
    }
    for (gsp_sppm* r : b->rs) k_store_u32<<<1, 1, 0, st>>>(r->counters + 7, (uint32_t)r->passes);
    for (int32_t k = 0; k < pairs; ++k) GSP_CUDA_TRY(cudaGraphLaunch(b->exec2, st));
    for (int32_t k = 0; k < singles; ++k) GSP_CUDA_TRY(cudaGraphLaunch(b->exec, st));
    for (gsp_sppm* r : b->rs) r->passes += npasses;
    GSP_CUDA_TRY(cudaGetLastError());
    return GSP_OK;
}

gsp_status gsp_batch_autotune(gsp_batch* b, int32_t trial_passes, gsp_tune_result* out) {
    if (!b || trial_passes < 1) return GSP_ERR_INVALID_ARG;
    for (gsp_sppm* r : b->rs)
        if (r->passes != 0 || r->grad) return GSP_ERR_BAD_STATE;
    GSP_CUDA_TRY(cudaSetDevice(b->device));
    (void)cudaGetLastError();
    cudaStream_t st = b->cap;
    cudaEvent_t a = nullptr, z = nullptr;
    cudaError_t ce = cudaEventCreate(&a);
    if (ce == cudaSuccess) ce = cudaEventCreate(&z);
    gsp_status e = GSP_OK;
    struct Cand { int32_t es, ps, gl, tr; bool fused; };
    const Cand start{b->rs[0]->eye_steps, b->rs[0]->photon_steps, b->rs[0]->gather_lanes, b->rs[0]->traversal,
                     b->fused};
    bool stack_ok = true;
    for (gsp_sppm* r : b->rs) stack_ok = stack_ok && r->scene->bvh.depth < kStackDepth;
    Cand pick = start;
    float best = INFINITY, first = INFINITY;
    int32_t ncand = 0;
    auto apply = [&](const Cand& c) {
        for (gsp_sppm* r : b->rs) {
            r->eye_steps = c.es;
            r->photon_steps = c.ps;
            r->gather_lanes = c.gl;
            r->traversal = c.tr;
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
        if (ms < best) {
            best = ms;
            pick = c;
        }
    };
    trial(start);
    const bool full = b->rs[0]->P.photon_mode == GSP_FULL_PATH;
    for (int32_t es : {0, 1})
        for (int32_t ps : full ? std::vector<int32_t>{0, 1, 2} : std::vector<int32_t>{0})
            if (es != start.es || ps != start.ps) trial({es, ps, start.gl, start.tr, start.fused});
    const Cand steps = pick;
    for (int32_t gl : {4, 8, 16})
        if (gl != start.gl) trial({steps.es, steps.ps, gl, start.tr, start.fused});
    const Cand lanes = pick;
    for (int32_t tr : {GSP_TRAVERSAL_MTBVH, GSP_TRAVERSAL_STACK})
        if (tr != start.tr && (tr != GSP_TRAVERSAL_STACK || stack_ok))
            trial({lanes.es, lanes.ps, lanes.gl, tr, start.fused});
    // last: one fused path launch for all renderers, or a path launch per renderer; with the
    // steps searched again for the other form (the best split moves)
    const Cand form = pick;
    for (int32_t es : {0, 1})
        for (int32_t ps : full ? std::vector<int32_t>{0, 1, 2} : std::vector<int32_t>{0})
            trial({es, ps, form.gl, form.tr, !form.fused});
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (a) cudaEventDestroy(a);
    if (z) cudaEventDestroy(z);
    apply(pick);  // captured again at the next gsp_batch_pass
    if (e != GSP_OK) return e;
    if (ce != cudaSuccess) {
        gsp_set_last_error(cudaGetErrorString(ce));
        return GSP_ERR_CUDA;
    }
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
    GSP_CUDA_TRY(cudaSetDevice(r->scene->ctx->device));
    (void)cudaGetLastError();
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
    // way gsp_sppm_pass runs them (overlapped in exact mode), which changes which settings win:
    // the overlap hides the path kernel's tail.
    const bool overlap = trial_passes >= 2 && r->P.hash_mode == GSP_EXACT;
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
        if (ms < best) {
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
    if (ce != cudaSuccess) {
        gsp_set_last_error(cudaGetErrorString(ce));
        return GSP_ERR_CUDA;
    }
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
    if (bytes && cudaMemcpy(buf.data(), d_src, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    return fwrite(buf.data(), 1, bytes, f) == bytes;
}

static bool ck_read(FILE* f, void* d_dst, size_t bytes, std::vector<char>& buf) {
    buf.resize(bytes);
    if (fread(buf.data(), 1, bytes, f) != bytes) return false;
    return !bytes || cudaMemcpy(d_dst, buf.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
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
    std::vector<char> buf;
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
        bool ok = ck_read(f, r->st0, r->npix * sizeof(float4), buf) && ck_read(f, r->st1, r->npix * sizeof(float4), buf);
        if (ok && r->P.photon_mode == GSP_REGEN)
            ok = ck_read(f, r->ro, r->np * sizeof(float4), buf) && ck_read(f, r->rd, r->np * sizeof(float4), buf) &&
                 ck_read(f, r->rphi, r->np * sizeof(float4), buf) &&
                 ck_read(f, r->started, sizeof(unsigned long long), buf);
        if (ok && hdr[6] > 0)
            ok = ck_read(f, r->rhist, (size_t)hdr[6] * r->npix * sizeof(float), buf) &&
                 ck_read(f, r->shist, (size_t)hdr[6] * r->npix * sizeof(float4), buf);
        if (ok) r->passes = hdr[3];
        st = ok ? GSP_OK : GSP_ERR_IO;
    }
    fclose(f);
    return st;
}

gsp_status gsp_sppm_image(gsp_sppm* r, float* d_rgb, void* stream) {
    if (!r || !d_rgb) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(r->scene->ctx->device));
    (void)cudaGetLastError();
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
    (void)cudaGetLastError();
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

int64_t gsp_sppm_last_deposits(gsp_sppm* r, uint32_t* h_ids, int64_t capacity) {
    if (!r) return GSP_ERR_INVALID_ARG;
    if (cudaSetDevice(r->scene->ctx->device) != cudaSuccess) return GSP_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return GSP_ERR_CUDA;
    uint32_t total = 0;
    if (cudaMemcpy(&total, r->counters, sizeof total, cudaMemcpyDeviceToHost) != cudaSuccess) return GSP_ERR_CUDA;
    if (!h_ids) return (int64_t)total;
    if (capacity < (int64_t)total) return GSP_ERR_INVALID_ARG;
    // ids of every deposit: walk the per-path counts on the host
    std::vector<uint32_t> cnt(r->np);
    std::vector<float4> rec(2 * (size_t)r->slot_cap);
    if (cudaMemcpy(cnt.data(), r->pcount, r->np * sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(rec.data(), r->slots, rec.size() * sizeof(float4), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GSP_ERR_CUDA;
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
int64_t gsp_grid_scratch_words(int64_t n, int64_t T) {
    return 4 * n + gsp_sort_hist_elems() +
           std::max(gsp_scan_temp_elems(T), gsp_scan_temp_elems(gsp_sort_hist_elems())) + 64;
}

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
    (void)cudaGetLastError();
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
