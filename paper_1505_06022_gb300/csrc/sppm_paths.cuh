// sppm_paths.cuh -- device side of an SPPM pass up to its deposits: pass parameters, hash-grid
// cells, wavefront queues, per-vertex shading data, the eye pass (Sec. 2), the photon pass
// (Sec. 2 whole paths; Sec. 3.3 one bounce per pass with regeneration) and the persistent path
// kernels (one renderer, or many in one launch). Included by sppm.cu only.
#pragma once

#include "devcommon.cuh"
#include "gsp_internal.h"
#include "launch.h"
#include "persist.cuh"

// resident blocks per SM of the path kernels beside GSP_PATH_MIN_BLOCKS (launch.h)
#ifndef GSP_PATH_SHADE_MIN_BLOCKS  // path kernels of scenes with shading data (72 registers)
#define GSP_PATH_SHADE_MIN_BLOCKS 7
#endif
#ifndef GSP_PATH_MULTI_MIN_BLOCKS  // the multi-scene path kernel: 70 registers without spills
#define GSP_PATH_MULTI_MIN_BLOCKS 7
#endif
#ifndef GSP_MULTI_CHUNK  // items (eye or photon paths) of one job that a warp takes at once
#define GSP_MULTI_CHUNK 64
#endif

namespace gspd {

constexpr float kPi = 3.14159265358979323846f;
constexpr int kMultiChunk = GSP_MULTI_CHUNK;  // a job's chunk in the multi-scene path kernel
constexpr int kSlotsPerPath = 32;

// The camera with its FP64 basis, tan(vfov / 2) and aspect ratio each split into double-float
// hi + lo parts (about 48 of their 53 bits).
struct CamDev {
    float3 eye;
    float3 fwd_hi, fwd_lo, right_hi, right_lo, up_hi, up_lo;
    float th_hi, th_lo, aspect_hi, aspect_lo;
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
    unsigned long long* work;  // work counters (kWork*), null unless the renderer counts its work
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
    // primary ray d = fwd + right sx + up sy, sx = ((px + u0) / w 2 - 1) tan(vfov/2) aspect,
    // sy = (1 - (py + u1) / h 2) tan(vfov/2), normalised: in double-float arithmetic (FP64 runs
    // at a small fraction of the FP32 rate here) and rounded once, the FP32 rounding of the exact
    // direction up to near-ties
    const DF th{C.th_hi, C.th_lo};
    DF sx = df_div_f(two_sum_df((float)px, u0), (float)C.w);
    sx = df_mul(df_add(DF{2.0f * sx.hi, 2.0f * sx.lo}, DF{-1.0f, 0.0f}), th);
    sx = df_mul(sx, DF{C.aspect_hi, C.aspect_lo});
    DF sy = df_div_f(two_sum_df((float)py, u1), (float)C.h);
    sy = df_mul(df_add(DF{1.0f, 0.0f}, DF{-2.0f * sy.hi, -2.0f * sy.lo}), th);
    const auto comp = [&](float fh, float fl, float rh, float rl, float uh, float ul) {
        return df_add(df_add(DF{fh, fl}, df_mul(DF{rh, rl}, sx)), df_mul(DF{uh, ul}, sy));
    };
    const DF dx = comp(C.fwd_hi.x, C.fwd_lo.x, C.right_hi.x, C.right_lo.x, C.up_hi.x, C.up_lo.x);
    const DF dy = comp(C.fwd_hi.y, C.fwd_lo.y, C.right_hi.y, C.right_lo.y, C.up_hi.y, C.up_lo.y);
    const DF dz = comp(C.fwd_hi.z, C.fwd_lo.z, C.right_hi.z, C.right_lo.z, C.up_hi.z, C.up_lo.z);
    const DF il = df_rsqrt(df_add(df_add(df_mul(dx, dx), df_mul(dy, dy)), df_mul(dz, dz)));
    const auto out = [&](DF v) {
        const DF c = df_mul(v, il);
        return __fadd_rn(c.hi, c.lo);
    };
    Q.ray[2 * p] = make_float4(C.eye.x, C.eye.y, C.eye.z, 0.0f);
    Q.ray[2 * p + 1] = make_float4(out(dx), out(dy), out(dz), __int_as_float(0x7f800000));
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
    // point on the triangle v0 + e1 b1 + e2 b2, b1 = sqrt(u1) (1 - u2), b2 = sqrt(u1) u2, in
    // double-float arithmetic (FP64 runs at a small fraction of the FP32 rate here) and rounded
    // once: the FP32 rounding of the exact point up to near-ties
    float th, tl;
    two_sum(1.0f, -u2, th, tl);  // 1 - u2 exactly
    const DF su = df_sqrt(u1), b1 = df_mul(su, DF{th, tl}), b2 = df_mul_f(su, u2);
    const auto coord = [&](float v, float a, float b) {
        const DF c = df_add(df_add(DF{v, 0.0f}, df_mul_f(b1, a)), df_mul_f(b2, b));
        return __fadd_rn(c.hi, c.lo);
    };
    o = make_float3(coord(v0.x, e1.x, e2.x), coord(v0.y, e1.y, e2.y), coord(v0.z, e1.z, e2.z));
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
// Once nothing is left to take, a path left alone in its warp has its walks done by all lanes
// (coop_walk).
// STACK: walk the child-pair layout with a stack (StackWalk) instead of the hit/miss links.
// COUNT: add the work of the launch to P.work (the instantiation used only while counting, so
// that the counters take no registers in the others).
template <bool STACK, bool SHADE, bool COUNT>
__global__ void __launch_bounds__(kTraceThreads, SHADE ? GSP_PATH_SHADE_MIN_BLOCKS : GSP_PATH_MIN_BLOCKS)
k_paths(DevScene S, PassDev P, PathQ qe, EyeOut O, const uint32_t* __restrict__ ne_ptr, PathQ qp, DepositDev D,
        const uint32_t* __restrict__ np_ptr, uint32_t* __restrict__ ctr) {
    const int32_t cap = trav_cap(S);
    const int32_t ne = ne_ptr ? (int32_t)*ne_ptr : 0;
    const int32_t nph = np_ptr ? (int32_t)*np_ptr : 0;
    WarpQueue<kPathChunk> wq;
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
    uint32_t c_eye = 0, c_ph = 0, c_nodes = 0, c_tris = 0;  // work of this lane
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
            trav_steps(S, st, pend, i >= 0, cap, c_tris);
        const bool walked = STACK ? sw.node == kWalkDone : (st.node < 0 && pend < 0);
        if (i >= 0 && walked) {
            const Hit h = walk_hit(S, st);
            float3 o = st.o, d = st.d;
            bool more = false;
            if (COUNT) {
                c_nodes += (uint32_t)st.steps;
                c_eye += eye ? 1u : 0u;
                c_ph += eye ? 0u : 1u;
            }
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
        if (!STACK && wq.done) {  // nothing left to take: a path left alone in the warp walks with all lanes
            const uint32_t act = __ballot_sync(0xffffffffu, i >= 0);
            if (act && !(act & (act - 1)) && __shfl_sync(0xffffffffu, max(st.node, pend), __ffs(act) - 1) >= 0) {
                const int owner = __ffs(act) - 1;
                const CoopWalk r = coop_walk(S.tris, S.nnodes, S.status, st, pend, owner, cap);
                st = r.st;
                pend = -1;
                if (COUNT && (threadIdx.x & 31) == owner) c_tris += r.ntri;
            }
        }
    }
    if (COUNT) {  // the whole warp leaves the loop together
        work_add_warp(P.work, kWorkEyeRays, c_eye);
        work_add_warp(P.work, kWorkPhotonRays, c_ph);
        work_add_warp(P.work, kWorkNodes, c_nodes);
        work_add_warp(P.work, kWorkTris, c_tris);
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
        pos = (c - J.first_chunk) * kMultiChunk;
        pend = min(pos + kMultiChunk, items);
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
__global__ void __launch_bounds__(kTraceThreads, SHADE ? GSP_PATH_SHADE_MIN_BLOCKS : GSP_PATH_MULTI_MIN_BLOCKS)
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
        uint32_t ntri = 0;  // work is not counted in batched passes
        if (STACK)
            stack_steps(J.S, st, sw, i >= 0, cap);
        else
            trav_steps(J.S, st, pend, i >= 0, cap, ntri);
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
// over the threads (counter *ctr) as the path kernel; STACK and COUNT as in k_paths.
template <bool STACK, bool SHADE, bool COUNT>
__global__ void __launch_bounds__(kTraceThreads, GSP_PATH_MIN_BLOCKS)
k_photon_regen(DevScene S, EmitDev E, PassDev P, DepositDev D, RegenDev R, uint32_t* __restrict__ ctr) {
    const int32_t cap = trav_cap(S);
    WarpQueue<kPathChunk> wq;
    wq.init((int32_t)P.np);
    Trav st;
    st.node = -1;
    st.slot = -1;
    StackWalk sw;
    sw.node = kWalkDone;
    sw.sp = 0;
    int32_t j = -1, pend = -1, depth = 0;
    uint32_t starts = 0;
    uint32_t c_ph = 0, c_nodes = 0, c_tris = 0;  // work of this lane
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
            trav_steps(S, st, pend, j >= 0, cap, c_tris);
        const bool walked = STACK ? sw.node == kWalkDone : (st.node < 0 && pend < 0);
        if (j >= 0 && walked) {
            if (COUNT) {
                c_ph += 1;
                c_nodes += (uint32_t)st.steps;
            }
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
    if (COUNT) {
        work_add_warp(P.work, kWorkPhotonRays, c_ph);
        work_add_warp(P.work, kWorkNodes, c_nodes);
        work_add_warp(P.work, kWorkTris, c_tris);
    }
}

}  // namespace gspd
