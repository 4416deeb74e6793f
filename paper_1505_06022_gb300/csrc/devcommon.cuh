// devcommon.cuh -- device-side building blocks: PRNG, ray/box and ray/triangle tests, and the
// stackless multiple-threaded BVH traversal (Sec. 3.1-3.2, Fig. 3, Fig. 5).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gspd {

// ----------------------------------------------------------------------------------------------
// device status word: the first error a kernel detects (0 = none). Never traps.
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ void report(int32_t* status, int32_t code) {
    if (status) atomicCAS(status, 0, code);
}

// ----------------------------------------------------------------------------------------------
// PRNG (Sec. 3.2, Fig. 5): four MLCGs s' = a s mod m, advanced with Schrage's decomposition in
// int32 (q = m div a, r = m mod a), combined as fract(s0/m0 - s1/m1 + s2/m2 - s3/m3) in FP32
// with a fixed evaluation order and round-to-nearest operations (no contraction).
// ----------------------------------------------------------------------------------------------
struct Rng {
    int32_t s[4];
};

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    // SplitMix64 (Steele, Lea & Flood 2014) output function at x + golden gamma.
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Counter-based stream: (seed, scene, domain, pass, id) -> four states in [1, m_i - 1].
__device__ __forceinline__ Rng rng_seed(uint64_t seed, uint32_t scene, uint32_t domain,
                                        uint32_t pass, uint64_t id) {
    uint64_t h = splitmix64(seed);
    h = splitmix64(h ^ (uint64_t)scene);
    h = splitmix64(h ^ (((uint64_t)domain << 32) | (uint64_t)pass));
    uint64_t h3 = splitmix64(h ^ id);
    uint64_t h4 = splitmix64(h3);
    Rng r;
    r.s[0] = 1 + (int32_t)((uint32_t)h3 % 4194286u);
    r.s[1] = 1 + (int32_t)((uint32_t)(h3 >> 32) % 4194276u);
    r.s[2] = 1 + (int32_t)((uint32_t)h4 % 4194190u);
    r.s[3] = 1 + (int32_t)((uint32_t)(h4 >> 32) % 4194166u);
    return r;
}

template <int A, int M, int Q, int R>
__device__ __forceinline__ int32_t mlcg(int32_t s) {
    int32_t hi = s / Q;
    int32_t lo = s - hi * Q;
    int32_t p = A * lo - R * hi;  // |p| < m, never 0 for 0 < s < m (m prime)
    return p < 0 ? p + M : p;
}

__device__ __forceinline__ float rng_next(Rng& r) {
    r.s[0] = mlcg<3423, 4194287, 1225, 1112>(r.s[0]);
    r.s[1] = mlcg<2646, 4194277, 1585, 367>(r.s[1]);
    r.s[2] = mlcg<1707, 4194191, 2457, 92>(r.s[2]);
    r.s[3] = mlcg<1999, 4194167, 2098, 265>(r.s[3]);
    float f0 = __fdiv_rn((float)r.s[0], 4194287.0f);
    float f1 = __fdiv_rn((float)r.s[1], 4194277.0f);
    float f2 = __fdiv_rn((float)r.s[2], 4194191.0f);
    float f3 = __fdiv_rn((float)r.s[3], 4194167.0f);
    float acc = __fsub_rn(f0, f1);
    acc = __fadd_rn(acc, f2);
    acc = __fsub_rn(acc, f3);
    float u = __fsub_rn(acc, floorf(acc));
    return u >= 1.0f ? 0x1.fffffep-1f : u;
}

// ----------------------------------------------------------------------------------------------
// small float3 algebra
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 mul3(float3 a, float3 b) { return make_float3(a.x * b.x, a.y * b.y, a.z * b.z); }
// The library is compiled without automatic multiply-add contraction (-fmad=false): every
// expression rounds as written, so an inlined function gives the same bits in every kernel that
// uses it (the batched path kernel agrees with the single-renderer one). Fused multiply-adds are
// spelled out where they belong: dot and cross products and b + a s.
__device__ __forceinline__ float dot3(float3 a, float3 b) {
    return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x)));
}
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(__fmaf_rn(a.y, b.z, -__fmul_rn(a.z, b.y)), __fmaf_rn(a.z, b.x, -__fmul_rn(a.x, b.z)),
                       __fmaf_rn(a.x, b.y, -__fmul_rn(a.y, b.x)));
}
// b + a s, one rounding per component
__device__ __forceinline__ float3 madd3(float3 a, float s, float3 b) {
    return make_float3(__fmaf_rn(a.x, s, b.x), __fmaf_rn(a.y, s, b.y), __fmaf_rn(a.z, s, b.z));
}
__device__ __forceinline__ float3 normalize3(float3 a) { return a * rsqrtf(dot3(a, a)); }

// ----------------------------------------------------------------------------------------------
// scene as the kernels see it
// ----------------------------------------------------------------------------------------------
struct DevScene {
    const float4* __restrict__ nodes;  // link_sets * nnodes * 2
    const float4* __restrict__ tris;   // 3 per triangle, leaf order
    const float4* __restrict__ shade;  // per triangle (upload order): normal xyz, material bits
    const float4* __restrict__ nlo;    // per triangle (upload order): FP32 remainder of the normal
    const float4* __restrict__ mats;   // 2 per material
    const float4* __restrict__ bin;    // child-pair layout of the same tree (stack traversal)
    const float4* __restrict__ attr;   // per triangle (upload order): vertex normals + texture coordinates, or null
    const float4* __restrict__ texels; // albedo textures
    const int4* __restrict__ mtex;     // per material: {first texel, width, height, 0}, or null
    int64_t nnodes;
    int64_t stride;  // nodes per link set in memory (nnodes + 1 padding node)
    int32_t link_sets;
    int32_t bin_root;
    int32_t step_limit;  // > 0: box tests one walk may make before it ends with an error
    int32_t* status;
};

struct Hit {
    int32_t id;  // triangle index in upload order, -1 = none
    float t, u, v;
    int32_t slot;  // SPPM hits: the triangle's leaf-ordered slot (its vertices), -1 = not known
};

// Ray direction class for the multiple-threaded BVH (replaces Fig. 3's cubemap lookup):
// principal axis = largest |d| component (ties x, y, z), sign = d_axis >= 0.
__device__ __forceinline__ int ray_class(float3 d) {
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int a = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    float da = a == 0 ? d.x : (a == 1 ? d.y : d.z);
    return 2 * a + (da >= 0.0f ? 0 : 1);
}

__device__ __forceinline__ float safe_inv(float d) {
    return __frcp_rn(fabsf(d) < 1e-30f ? copysignf(1e-30f, d) : d);
}

// 1 + 2 gamma_3 with gamma_n = n u / (1 - n u), u = 2^-24: the far-plane scale that makes the
// FP32 slab test conservative against relative rounding errors (Ize 2013).
#define GSP_ROBUST_FAR 1.0000003576278687f

// Three-input minimum and maximum (one instruction each on sm_100 and later).
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// The triangle is chosen in FP32. Its t can lose relative accuracy when the ray origin is far
// from the triangle compared with t, or the ray is grazing (cancellation in o - v0 and in det);
// hit_error_factor() estimates that amplification and refine_hit() re-evaluates t, u, v in FP64
// from the exact vertices for the hits that need it.
__device__ __forceinline__ bool refine_hit(const float4* __restrict__ tri, float3 of, float3 df, Hit& h) {
    const float4 A = __ldg(tri), B = __ldg(tri + 1), C = __ldg(tri + 2);
    const double ax = A.x, ay = A.y, az = A.z;
    const double e1x = (double)B.x - ax, e1y = (double)B.y - ay, e1z = (double)B.z - az;
    const double e2x = (double)C.x - ax, e2y = (double)C.y - ay, e2z = (double)C.z - az;
    const double dx = df.x, dy = df.y, dz = df.z;
    const double px = dy * e2z - dz * e2y, py = dz * e2x - dx * e2z, pz = dx * e2y - dy * e2x;
    const double det = e1x * px + e1y * py + e1z * pz;
    if (det == 0.0) return false;
    const double f = __drcp_rn(det);
    const double sx = (double)of.x - ax, sy = (double)of.y - ay, sz = (double)of.z - az;
    const double qx = sy * e1z - sz * e1y, qy = sz * e1x - sx * e1z, qz = sx * e1y - sy * e1x;
    h.u = (float)(f * (sx * px + sy * py + sz * pz));
    h.v = (float)(f * (dx * qx + dy * qy + dz * qz));
    h.t = (float)(f * (e2x * qx + e2y * qy + e2z * qz));
    return true;
}

// Relative-error amplification of the FP32 t of a hit, (|s| / (t |d|) + 1) |e1| |e2| |d| / |det|
// in L1 norms; FP32 Moller-Trumbore errs by about 1e-7 times this. Also returns FP32 (u, v).
__device__ __forceinline__ float hit_error_factor(const float4* __restrict__ tri, float3 o, float3 d, float t,
                                                  float& u, float& v) {
    const float4 A = __ldg(tri), B = __ldg(tri + 1), C = __ldg(tri + 2);
    const float3 v0 = f3(A);
    const float3 e1 = f3(B) - v0, e2 = f3(C) - v0;
    const float3 p = cross3(d, e2);
    const float det = dot3(e1, p);
    const float3 s = o - v0;
    const float f = 1.0f / det;
    u = f * dot3(s, p);
    v = f * dot3(d, cross3(s, e1));
    const float l1d = fabsf(d.x) + fabsf(d.y) + fabsf(d.z);
    const float l1s = fabsf(s.x) + fabsf(s.y) + fabsf(s.z);
    const float l1e = (fabsf(e1.x) + fabsf(e1.y) + fabsf(e1.z)) * (fabsf(e2.x) + fabsf(e2.y) + fabsf(e2.z));
    return (l1s / (t * l1d) + 1.0f) * l1e * l1d / fabsf(det);
}

// hit_error_factor(...) > rf without its divisions: with L1 norms and t > 0 the test is
// (|s| + t |d|) |e1| |e2| > rf t |det|. FP32 (u, v) only when want_uv (else left as they are).
__device__ __forceinline__ bool hit_needs_refine(const float4* __restrict__ tri, float3 o, float3 d, float t,
                                                 float rf, bool want_uv, float& u, float& v) {
    const float4 A = __ldg(tri), B = __ldg(tri + 1), C = __ldg(tri + 2);
    const float3 v0 = f3(A);
    const float3 e1 = f3(B) - v0, e2 = f3(C) - v0;
    const float3 p = cross3(d, e2);
    const float det = dot3(e1, p);
    const float3 s = o - v0;
    if (want_uv) {
        const float f = 1.0f / det;
        u = f * dot3(s, p);
        v = f * dot3(d, cross3(s, e1));
    }
    const float l1d = fabsf(d.x) + fabsf(d.y) + fabsf(d.z);
    const float l1s = fabsf(s.x) + fabsf(s.y) + fabsf(s.z);
    const float l1e = (fabsf(e1.x) + fabsf(e1.y) + fabsf(e1.z)) * (fabsf(e2.x) + fabsf(e2.y) + fabsf(e2.z));
    return (l1s + t * l1d) * l1e > rf * t * fabsf(det);
}

// Hits whose estimated amplification exceeds this are re-evaluated in FP64 (expected FP32
// relative error below about 64 * 6e-8 ~ 4e-6 for the rest).
#define GSP_REFINE_FACTOR 64.0f

// Error-free transformations in FP32: a + b = s + e exactly (Knuth's two-sum) and a * b = p + e
// exactly (two-product with one FMA). Sums and dot products built from them carry about twice
// the working precision (Ogita, Rump & Oishi, SIAM J. Sci. Comput. 26(6), 2005).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Double-float numbers hi + lo (|lo| <= ulp(hi) / 2) and the few operations the emission kernels
// need, after Dekker (Numer. Math. 18, 1971), built on the error-free sum and product above: about
// 44 bits of precision at FP32 instruction cost. A result rounded to FP32 (its hi) is the FP32
// rounding of the exact value except within about 2^-20 of a tie.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ DF df_mul_f(DF a, float b) {
    float p, e;
    two_prod(a.hi, b, p, e);
    return fast_two_sum(p, __fmaf_rn(a.lo, b, e));
}

__device__ __forceinline__ DF two_sum_df(float a, float b) {
    DF r;
    two_sum(a, b, r.hi, r.lo);
    return r;
}

// a / b: the FP32 quotient plus its correction from the exact remainder a.hi - q b.
__device__ __forceinline__ DF df_div_f(DF a, float b) {
    const float q = __fdiv_rn(a.hi, b);
    const float r = __fadd_rn(__fmaf_rn(-q, b, a.hi), a.lo);
    return fast_two_sum(q, __fdiv_rn(r, b));
}

// 1 / sqrt(a) for a > 0: the FP32 value refined by one Newton step y + y (1 - a y^2) / 2 in
// double-float arithmetic.
__device__ __forceinline__ DF df_rsqrt(DF a) {
    const float y = __frsqrt_rn(a.hi);
    float yh, yl;
    two_prod(y, y, yh, yl);
    const DF t = df_mul(a, DF{yh, yl});
    const DF e = df_add(DF{1.0f, 0.0f}, DF{-t.hi, -t.lo});
    return df_add(DF{y, 0.0f}, df_mul_f(e, 0.5f * y));
}

// sqrt(a) for a >= 0: the FP32 root plus its correction from the exact residual a - s^2.
__device__ __forceinline__ DF df_sqrt(float a) {
    const float s = __fsqrt_rn(a);
    if (!(s > 0.0f)) return DF{s, 0.0f};
    return fast_two_sum(s, __fdiv_rn(__fmaf_rn(-s, s, a), __fadd_rn(s, s)));
}

// (nh + nl) . (vh + vl) as a normalised double-float hi + lo (|lo| <= ulp(hi) / 2): the
// products nh * vh exactly, the cross terms once rounded, nl * vl dropped. Normalising matters
// when the dot product cancels: the quotient below corrects only to first order in lo / hi.
__device__ __forceinline__ void dot2(float3 nh, float3 nl, float3 vh, float3 vl, float& hi, float& lo) {
    float p0, e0, p1, e1, p2, e2, c;
    two_prod(nh.x, vh.x, p0, e0);
    two_prod(nh.y, vh.y, p1, e1);
    two_prod(nh.z, vh.z, p2, e2);
    two_sum(p0, p1, hi, lo);
    two_sum(hi, p2, hi, c);
    lo = __fadd_rn(lo, c);
    lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(e0, e1), e2));
    lo = __fmaf_rn(nh.x, vl.x, __fmaf_rn(nh.y, vl.y, __fmaf_rn(nh.z, vl.z, lo)));
    lo = __fmaf_rn(nl.x, vh.x, __fmaf_rn(nl.y, vh.y, __fmaf_rn(nl.z, vh.z, lo)));
    two_sum(hi, lo, hi, lo);
}

// Distance along the ray to the plane through v0 with unit normal nh + nl (a double-float
// normal, exact to ~2^-48), t = n.(v0 - o) / n.d, with v0 - o formed exactly and both dot
// products and the quotient carried in double-float FP32 arithmetic: t comes out within about
// one FP32 rounding of the exact value, at FP32 instruction cost (GB300's FP64 rate is a small
// fraction of its FP32 rate). Returns false if the ray is parallel to the plane.
__device__ __forceinline__ bool plane_t(float3 v0, float3 nh, float3 nl, float3 o, float3 d, float& t) {
    float3 sh, sl;
    two_sum(v0.x, -o.x, sh.x, sl.x);
    two_sum(v0.y, -o.y, sh.y, sl.y);
    two_sum(v0.z, -o.z, sh.z, sl.z);
    float num_h, num_l, den_h, den_l;
    dot2(nh, nl, sh, sl, num_h, num_l);
    dot2(nh, nl, d, make_float3(0.0f, 0.0f, 0.0f), den_h, den_l);
    if (den_h == 0.0f) return false;
    const float q = __fdiv_rn(num_h, den_h);
    const float r = __fadd_rn(__fmaf_rn(-q, den_h, num_h), __fmaf_rn(-q, den_l, num_l));  // num - q den
    t = __fadd_rn(q, __fdiv_rn(r, den_h));
    return true;
}

// SPPM hits (eye hit points and photon positions, where t decides which side of a gather radius
// a photon falls): t from the plane of the winning triangle (slot in leaf order, upload-order
// index id) in double-float arithmetic.
__device__ __forceinline__ void refine_plane(const float4* __restrict__ tris, const float4* __restrict__ shade,
                                             const float4* __restrict__ nlo, int32_t slot, int32_t id, float3 o,
                                             float3 d, float& t) {
    const float3 v0 = f3(__ldg(tris + 3 * (int64_t)slot));
    const float3 nh = f3(__ldg(shade + id)), nl = f3(__ldg(nlo + id));
    float tt;
    if (plane_t(v0, nh, nl, o, d, tt)) t = tt;
}

// Traversal state of one ray (Fig. 3): current node in the ray's link set, best hit so far.
struct Trav {
    float3 o, d, inv;
    float tmin, tbest;
    int32_t best, slot, node, steps;
    const float4* __restrict__ nodes;
};

__device__ __forceinline__ void trav_init(const DevScene& S, float3 o, float3 d, float tmin, float tmax, Trav& st) {
    st.o = o;
    st.d = d;
    st.inv = make_float3(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
    st.tmin = tmin;
    st.tbest = tmax;
    st.best = -1;
    st.slot = -1;
    st.node = 0;
    st.steps = 0;
    const int c = S.link_sets == 6 ? ray_class(d) : 0;
    st.nodes = S.nodes + (size_t)c * (size_t)S.stride * 2;
}

// Moller-Trumbore test of one triangle (vertices P.xyz, V1.xyz, V2.xyz): true when the ray's
// line meets it (det != 0, u >= 0, v >= 0, u + v <= 1); t is the distance in units of |d|.
__device__ __forceinline__ bool tri_hit(float3 o, float3 d, const float4& P, const float4& V1, const float4& V2,
                                        float& t) {
    const float3 v0 = f3(P);
    const float3 e1 = f3(V1) - v0, e2 = f3(V2) - v0;
    const float3 p = cross3(d, e2);
    const float det = dot3(e1, p);
    if (det == 0.0f) return false;
    const float f = 1.0f / det;
    const float3 s = o - v0;
    const float u = f * dot3(s, p);
    const float3 q = cross3(s, e1);
    const float v = f * dot3(d, q);
    t = f * dot3(e2, q);
    return u >= 0.0f && v >= 0.0f && u + v <= 1.0f;
}

// Moller-Trumbore on the triangles [first, first + cnt) of the leaf-ordered triangle array,
// keeping the lexicographic (t, triangle index) minimum over tmin < t < best t.
__device__ __forceinline__ void trav_leaf(const DevScene& S, Trav& st, int32_t first, int32_t cnt) {
    for (int32_t k = 0; k < cnt; ++k) {
        const float4 P = __ldg(S.tris + 3 * (first + k));
        const float4 V1 = __ldg(S.tris + 3 * (first + k) + 1);
        const float4 V2 = __ldg(S.tris + 3 * (first + k) + 2);
        float t;
        const int32_t id = __float_as_int(P.w);
        if (tri_hit(st.o, st.d, P, V1, V2, t) && t > st.tmin &&
            (t < st.tbest || (t == st.tbest && st.best >= 0 && id < st.best))) {
            st.tbest = t;
            st.best = id;
            st.slot = first + k;
        }
    }
}

// 64 bytes at a 32-byte aligned address (two adjacent nodes, or a node's two child boxes) as two
// 256-bit read-only vector loads (sm_100 and later): half the load instructions of four 128-bit
// loads on the traversal's dependent fetch.
__device__ __forceinline__ void ldg64(const float4* p, float4& A, float4& B, float4& C, float4& D) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(A.x), "=f"(A.y), "=f"(A.z), "=f"(A.w), "=f"(B.x), "=f"(B.y), "=f"(B.z), "=f"(B.w)
        : "l"(p));
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8+32];"
        : "=f"(C.x), "=f"(C.y), "=f"(C.z), "=f"(C.w), "=f"(D.x), "=f"(D.y), "=f"(D.z), "=f"(D.w)
        : "l"(p));
}

// Slab test of the box [lo, hi] against [tmin, best t] (Fig. 3's intersect(node.aabb, ray)):
// t = (b - o) inv per plane, three-input min and max for the interval, the far end scaled by
// GSP_ROBUST_FAR; conservative. On a hit tn is the entry distance. (The fused form
// t = b inv + (-o inv) saves six instructions per box but errs in absolute terms by about
// u |o inv|, which needs a per-plane pad held in six more registers per ray; on GB300 the spills
// and lost residency that cost made the traversal slower: 5,132 against 5,217 Mrays/s.)
__device__ __forceinline__ bool slab(const Trav& st, float3 lo, float3 hi, float& tn) {
    const float3 o = st.o, inv = st.inv;
    const float t0x = __fmul_rn(lo.x - o.x, inv.x), t1x = __fmul_rn(hi.x - o.x, inv.x);
    const float t0y = __fmul_rn(lo.y - o.y, inv.y), t1y = __fmul_rn(hi.y - o.y, inv.y);
    const float t0z = __fmul_rn(lo.z - o.z, inv.z), t1z = __fmul_rn(hi.z - o.z, inv.z);
    tn = max3f(fminf(t0x, t1x), fminf(t0y, t1y), fmaxf(fminf(t0z, t1z), st.tmin));
    const float tf = min3f(fmaxf(t0x, t1x), fmaxf(t0y, t1y), fmaxf(t0z, t1z));
    return tn <= fminf(st.tbest, __fmul_rn(tf, GSP_ROBUST_FAR));
}

// Box test of a node {A, B} = {min.xyz, miss | max.xyz, leaf word} against [tmin, best t].
// Returns true on a hit; `word` and `miss` receive the links.
__device__ __forceinline__ bool box_hit(const Trav& st, const float4& A, const float4& B, int32_t& word, int32_t& miss) {
    float tn;
    miss = __float_as_int(A.w);
    word = __float_as_int(B.w);
    return slab(st, f3(A), f3(B), tn);
}

// Slab test of the box [lo, hi] as box_hit, with the entry distance (stack-based traversal
// orders children by it).
__device__ __forceinline__ bool box_entry(const Trav& st, float3 lo, float3 hi, float& tn) {
    return slab(st, lo, hi, tn);
}

// One step of the stackless traversal (Fig. 3): on a box hit follow the hit link (index + 1),
// running Moller-Trumbore on a leaf's triangles first (a leaf's hit link is its miss link);
// otherwise follow the miss link. The node after the current one in preorder (the first child
// of an internal node) comes with the same fetch, so a descent tests two boxes per step.
__device__ __forceinline__ void trav_step(const DevScene& S, Trav& st) {
    float4 A, B, C, D;
    ldg64(st.nodes + 2 * st.node, A, B, C, D);
    int32_t word, miss;
    if (!box_hit(st, A, B, word, miss)) {
        st.node = miss;
    } else if (word >= 0) {
        trav_leaf(S, st, word >> 3, word & 7);
        st.node = miss;
    } else {
        int32_t w2, m2;
        if (!box_hit(st, C, D, w2, m2)) {
            st.node = m2;
        } else if (w2 >= 0) {
            trav_leaf(S, st, w2 >> 3, w2 & 7);
            st.node = m2;
        } else {
            st.node = st.node + 2;
        }
    }
}

// Closest hit of one ray: traversal to the end, then the winner's t re-evaluated, either always
// from its plane in double-float arithmetic (SPPM hit points: photons near the gather radius then
// fall on the same side of it as in an exact evaluation far more often), or with t, u, v in FP64
// when the FP32 value may be inaccurate.
template <bool ALWAYS_REFINE>
__device__ __forceinline__ Hit traverse(const DevScene& S, float3 o, float3 d, float tmin, float tmax) {
    Trav st;
    trav_init(S, o, d, tmin, tmax, st);
    const int64_t cap = S.step_limit > 0 ? S.step_limit : 2 * S.nnodes + 8;
    while (st.node >= 0) {
        if (++st.steps > cap) {
            report(S.status, -4);
            break;
        }
        trav_step(S, st);
    }
    Hit h;
    h.id = st.best;
    h.t = st.tbest;
    h.u = h.v = 0.0f;
    if (st.slot >= 0) {
        const float4* tri = S.tris + 3 * st.slot;
        if (ALWAYS_REFINE)
            refine_plane(S.tris, S.shade, S.nlo, st.slot, h.id, o, d, h.t);
        else if (hit_error_factor(tri, o, d, h.t, h.u, h.v) > GSP_REFINE_FACTOR)
            refine_hit(tri, o, d, h);
    }
    return h;
}

}  // namespace gspd
