// gsp_oracle.cpp -- CPU oracle for the MTBVH ray caster and the SPPM renderer.
//
// TEST INFRASTRUCTURE ONLY. A plain, slow restatement of what the CUDA path computes, written
// from the paper (Hachisuka, "Implementing a Photorealistic Rendering System using GLSL",
// EGSR 2015) and the methods it cites. Only the tests, the smoke check and the CPU-baseline leg
// of the benchmark may load it; the product library never does, and the two share no code.
//
// Precision: geometry, sampling and density estimation run in FP64. The PRNG output is FP32,
// because the FP32 value is what the method defines (Sec. 3.2, Fig. 5) and both sides must draw
// bit-identical numbers; this file must be compiled with -ffp-contract=off and no fast-math.
//
// What each part follows:
//  * rng_*            Sec. 3.2 / Fig. 5: four multiplicative LCGs combined as
//                     fract(s0/m0 - s1/m1 + s2/m2 - s3/m3); the state update is written as the
//                     textbook MLCG s' = a*s mod m. Per-stream seeding is counter-based
//                     (splitmix64, Steele/Lea/Flood 2014) instead of host xorshift (Sec. 3.2).
//  * mt_intersect     Moller-Trumbore ray/triangle test (the leaf test of Fig. 3), FP64.
//  * sah split        the binned SAH split of Sec. 3.1's top-down build (Wald 2007), every
//                     candidate evaluated from scratch; the library's host build must pick it.
//  * closest hit      brute force over every triangle (definition of the closest hit) with
//                     the lexicographic (t, id) minimum; a simple median-split BVH with a stack
//                     is used only for speed and is checked against brute force by the tests.
//  * SPPM             Sec. 2 (photon tracing, eye tracing to the first non-specular hit, range
//                     query + progressive density estimation; Hachisuka & Jensen 2009),
//                     Sec. 3.3 (photon path regeneration), Sec. 3.4 (stochastic hashing with a
//                     random depth per photon).
//  * surface          Sec. 3.1's triangle record with a normal and texture coordinates per
//                     vertex: the shading normal is the barycentric blend of the vertex
//                     normals, normalised; the albedo of a diffuse material is multiplied by a
//                     bilinear, wrapping lookup of its texture at the blended coordinates.
//  Parity unpinned: none of the functions exported here; every one is pinned by a CPU test.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

// ------------------------------------------------------------------------------------------
// PRNG (Sec. 3.2, Fig. 5)
// ------------------------------------------------------------------------------------------
const int64_t kA[4] = {3423, 2646, 1707, 1999};
const int64_t kM[4] = {4194287, 4194277, 4194191, 4194167};

struct Rng {
    int64_t s[4];
};

uint64_t splitmix64(uint64_t x) {
    // Steele, Lea & Flood (2014), SplitMix64 output function applied to x + golden gamma.
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

Rng rng_seed(uint64_t seed, uint32_t scene, uint32_t domain, uint32_t pass, uint64_t id) {
    uint64_t h0 = splitmix64(seed);
    uint64_t h1 = splitmix64(h0 ^ (uint64_t)scene);
    uint64_t h2 = splitmix64(h1 ^ (((uint64_t)domain << 32) | (uint64_t)pass));
    uint64_t h3 = splitmix64(h2 ^ id);
    uint64_t h4 = splitmix64(h3);
    uint32_t w[4] = {(uint32_t)h3, (uint32_t)(h3 >> 32), (uint32_t)h4, (uint32_t)(h4 >> 32)};
    Rng r;
    for (int i = 0; i < 4; ++i) r.s[i] = 1 + (int64_t)(w[i] % (uint32_t)(kM[i] - 1));
    return r;
}

float rng_next(Rng& r) {
    for (int i = 0; i < 4; ++i) r.s[i] = (kA[i] * r.s[i]) % kM[i];  // MLCG definition
    float f[4];
    for (int i = 0; i < 4; ++i) f[i] = (float)r.s[i] / (float)kM[i];  // exact operands, RN
    float acc = f[0] - f[1];
    acc = acc + f[2];
    acc = acc - f[3];
    float u = acc - std::floor(acc);
    if (u >= 1.0f) u = 0x1.fffffep-1f;  // fract() of a tiny negative rounds up to 1
    return u;
}

// ------------------------------------------------------------------------------------------
// small FP64 vector algebra
// ------------------------------------------------------------------------------------------
struct V3 {
    double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline V3 mul(V3 a, V3 b) { return {a.x * b.x, a.y * b.y, a.z * b.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 normalize(V3 a) { return a * (1.0 / norm(a)); }
inline double comp(V3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

struct Tri {
    V3 v0, e1, e2, n;  // n = normalize(e1 x e2), the geometric (front) normal
    double area;
    int mat;
};

// ------------------------------------------------------------------------------------------
// Moller-Trumbore, FP64 (leaf test of Fig. 3)
// ------------------------------------------------------------------------------------------
struct MT {
    bool ok;  // det != 0
    double t, u, v, det;
};

MT mt_intersect(const V3& o, const V3& d, const Tri& T) {
    MT r{false, 0, 0, 0, 0};
    V3 p = cross(d, T.e2);
    double det = dot(T.e1, p);
    r.det = det;
    if (det == 0.0) return r;
    double f = 1.0 / det;
    V3 s = o - T.v0;
    V3 q = cross(s, T.e1);
    r.u = f * dot(s, p);
    r.v = f * dot(d, q);
    r.t = f * dot(T.e2, q);
    r.ok = true;
    return r;
}

inline bool mt_inside(const MT& m) { return m.ok && m.u >= 0 && m.v >= 0 && m.u + m.v <= 1.0; }

// ------------------------------------------------------------------------------------------
// closest hit: lexicographic (t, id) minimum over tmin < t < tmax
// ------------------------------------------------------------------------------------------
struct Hit {
    int id;
    double t, u, v;
};

inline bool better(double t, int id, const Hit& h) {
    return h.id < 0 || t < h.t || (t == h.t && id < h.id);
}

struct BVHNode {
    V3 lo, hi;
    int left, right;  // children (internal) or -1
    int first, count; // triangle range in `order` (leaf)
};

// Per-vertex shading data of one triangle (Sec. 3.1 stores a normal and texture coordinates
// with each vertex of a triangle).
struct Shading {
    bool normals;
    V3 n[3];
    double st[3][2];  // texture coordinates (s, t) of the three vertices
};

struct Mesh {
    std::vector<Tri> tris;
    std::vector<BVHNode> nodes;
    std::vector<int> order;
    std::vector<Shading> shade;  // empty: face normals, no texture coordinates
};

void bvh_build(Mesh& M) {
    // Object-median split along the widest centroid axis; only an accelerator for the oracle.
    int n = (int)M.tris.size();
    M.order.resize(n);
    for (int i = 0; i < n; ++i) M.order[i] = i;
    M.nodes.clear();
    std::vector<V3> cen(n), lo(n), hi(n);
    for (int i = 0; i < n; ++i) {
        const Tri& T = M.tris[i];
        V3 a = T.v0, b = T.v0 + T.e1, c = T.v0 + T.e2;
        lo[i] = {std::min({a.x, b.x, c.x}), std::min({a.y, b.y, c.y}), std::min({a.z, b.z, c.z})};
        hi[i] = {std::max({a.x, b.x, c.x}), std::max({a.y, b.y, c.y}), std::max({a.z, b.z, c.z})};
        cen[i] = (lo[i] + hi[i]) * 0.5;
    }
    if (n == 0) return;
    struct Job { int node, first, count; };
    M.nodes.push_back({});
    std::vector<Job> stack{{0, 0, n}};
    while (!stack.empty()) {
        Job j = stack.back();
        stack.pop_back();
        V3 blo = {1e300, 1e300, 1e300}, bhi = {-1e300, -1e300, -1e300};
        V3 clo = blo, chi = bhi;
        for (int k = j.first; k < j.first + j.count; ++k) {
            int t = M.order[k];
            blo = {std::min(blo.x, lo[t].x), std::min(blo.y, lo[t].y), std::min(blo.z, lo[t].z)};
            bhi = {std::max(bhi.x, hi[t].x), std::max(bhi.y, hi[t].y), std::max(bhi.z, hi[t].z)};
            clo = {std::min(clo.x, cen[t].x), std::min(clo.y, cen[t].y), std::min(clo.z, cen[t].z)};
            chi = {std::max(chi.x, cen[t].x), std::max(chi.y, cen[t].y), std::max(chi.z, cen[t].z)};
        }
        BVHNode& nd = M.nodes[j.node];
        nd.lo = blo;
        nd.hi = bhi;
        nd.left = nd.right = -1;
        nd.first = j.first;
        nd.count = j.count;
        if (j.count <= 4) continue;
        V3 ext = chi - clo;
        int axis = (ext.x >= ext.y && ext.x >= ext.z) ? 0 : (ext.y >= ext.z ? 1 : 2);
        int mid = j.first + j.count / 2;
        std::nth_element(M.order.begin() + j.first, M.order.begin() + mid,
                         M.order.begin() + j.first + j.count, [&](int a, int b) {
                             double ca = comp(cen[a], axis), cb = comp(cen[b], axis);
                             return ca < cb || (ca == cb && a < b);
                         });
        int l = (int)M.nodes.size();
        M.nodes.push_back({});
        M.nodes.push_back({});
        M.nodes[j.node].left = l;
        M.nodes[j.node].right = l + 1;
        stack.push_back({l, j.first, mid - j.first});
        stack.push_back({l + 1, mid, j.first + j.count - mid});
    }
}

// Slab test with a padded box so that no box is ever culled by rounding.
bool box_hit(const BVHNode& nd, const V3& o, const V3& d, double tmin, double tmax) {
    double t0 = tmin, t1 = tmax;
    for (int k = 0; k < 3; ++k) {
        double ok_ = comp(o, k), dk = comp(d, k);
        double lo = comp(nd.lo, k), hi = comp(nd.hi, k);
        double pad = 1e-9 * (std::fabs(lo) + std::fabs(hi) + 1.0);
        lo -= pad;
        hi += pad;
        if (dk == 0.0) {
            if (ok_ < lo || ok_ > hi) return false;
            continue;
        }
        double a = (lo - ok_) / dk, b = (hi - ok_) / dk;
        if (a > b) std::swap(a, b);
        t0 = std::max(t0, a);
        t1 = std::min(t1, b);
        if (t0 > t1 * (1 + 1e-12) + 1e-300) return false;
    }
    return true;
}

// Visits every triangle whose (padded) leaf box the ray segment touches.
template <class F>
void bvh_visit(const Mesh& M, const V3& o, const V3& d, double tmin, const double& tmax, F&& f) {
    if (M.nodes.empty()) return;
    int stack[128];
    int sp = 0;
    stack[sp++] = 0;
    while (sp) {
        const BVHNode& nd = M.nodes[stack[--sp]];
        if (!box_hit(nd, o, d, tmin, tmax)) continue;
        if (nd.left < 0) {
            for (int k = nd.first; k < nd.first + nd.count; ++k) f(M.order[k]);
        } else {
            stack[sp++] = nd.left;
            stack[sp++] = nd.right;
        }
    }
}

Hit closest_brute(const Mesh& M, const V3& o, const V3& d, double tmin, double tmax) {
    Hit h{-1, tmax, 0, 0};
    for (int i = 0; i < (int)M.tris.size(); ++i) {
        MT m = mt_intersect(o, d, M.tris[i]);
        if (!mt_inside(m) || !(m.t > tmin) || !(m.t < tmax)) continue;
        if (better(m.t, i, h)) h = {i, m.t, m.u, m.v};
    }
    return h;
}

Hit closest_bvh(const Mesh& M, const V3& o, const V3& d, double tmin, double tmax) {
    Hit h{-1, tmax, 0, 0};
    double tcull = tmax;
    bvh_visit(M, o, d, tmin, tcull, [&](int i) {
        MT m = mt_intersect(o, d, M.tris[i]);
        if (!mt_inside(m) || !(m.t > tmin) || !(m.t < tmax)) return;
        if (better(m.t, i, h)) {
            h = {i, m.t, m.u, m.v};
            tcull = m.t;
        }
    });
    return h;
}

// Non-degenerate ray: the FP32 and FP64 answers must agree on it (see the header of
// oracle/__init__.py for the rule).
bool classify(const Mesh& M, bool brute, const V3& o, const V3& d, double tmin, double tmax,
              const Hit& w) {
    const double kBary = 1e-6, kTRel = 1e-5, kDet = 1e-7;
    bool ok = true;
    double dn = norm(d);
    if (w.id >= 0) {
        const Tri& T = M.tris[w.id];
        MT m = mt_intersect(o, d, T);
        double margin = std::min({m.u, m.v, 1.0 - m.u - m.v});
        if (!(margin > kBary)) ok = false;
        if (!(std::fabs(m.det) > kDet * norm(T.e1) * norm(T.e2) * dn)) ok = false;
        if (!(std::fabs(w.t - tmin) > kTRel * std::fabs(w.t))) ok = false;
        if (std::isfinite(tmax) && !(std::fabs(tmax - w.t) > kTRel * std::fabs(w.t))) ok = false;
    }
    if (!ok) return false;
    double tref = w.id >= 0 ? w.t : 0.0;
    double hi = std::isfinite(tmax) ? tmax * (1 + kTRel) + 1e-30 : tmax;
    auto check = [&](int i) {
        if (!ok || i == w.id) return;
        MT m = mt_intersect(o, d, M.tris[i]);
        if (!m.ok) return;
        double margin = std::min({m.u, m.v, 1.0 - m.u - m.v});
        if (margin < -kBary) return;
        if (!(m.t > tmin - kTRel * std::max(std::fabs(m.t), std::fabs(tmin)))) return;
        if (!(m.t < hi)) return;
        if (w.id < 0) { ok = false; return; }
        if (!(std::fabs(m.t - tref) > kTRel * std::fabs(tref))) ok = false;
        if (m.t < tref && margin >= -kBary) ok = false;  // a near-miss in front of the winner
    };
    if (brute) {
        for (int i = 0; i < (int)M.tris.size(); ++i) check(i);
    } else {
        double big = hi;
        bvh_visit(M, o, d, tmin - 1e-5 * (std::fabs(tmin) + 1.0), big, check);
    }
    return ok;
}

// ------------------------------------------------------------------------------------------
// threading helper: static contiguous chunks, results merged in chunk order
// ------------------------------------------------------------------------------------------
template <class F>
void parallel_for(int64_t n, int nthreads, F&& f) {
    if (nthreads <= 1 || n < 2) {
        f(0, n, 0);
        return;
    }
    nthreads = (int)std::min<int64_t>(nthreads, n);
    std::vector<std::thread> th;
    for (int t = 0; t < nthreads; ++t) {
        int64_t a = n * t / nthreads, b = n * (t + 1) / nthreads;
        th.emplace_back([&f, a, b, t] { f(a, b, t); });
    }
    for (auto& x : th) x.join();
}

}  // namespace

// ==========================================================================================
// exported C interface (ctypes)
// ==========================================================================================
extern "C" {

typedef struct {
    int32_t type;  // 0 diffuse, 1 mirror, 2 dielectric, 3 emitter
    float albedo[3];
    float emission[3];
    float ior;
} orc_material;

typedef struct {
    float eye[3], look[3], up[3];
    float vfov_deg;
    int32_t width, height;
} orc_camera;

typedef struct {
    int64_t photons_per_pass;
    int64_t table_size;      // hash table entries (power of two)
    uint64_t seed;
    float alpha, r0, rr_continue, cell_h, eps;
    int32_t photon_mode;     // 0 full path per pass, 1 one bounce per pass (Sec. 3.3)
    int32_t hash_mode;       // 0 exact (all photons in range), 1 stochastic (Sec. 3.4)
    int32_t max_eye_depth, max_photon_depth;
    uint32_t scene_id;
} orc_sppm_params;

// ---- RNG ----
int64_t orc_mlcg_step(int32_t i, int64_t s) { return (kA[i] * s) % kM[i]; }

void orc_mlcg_step_many(int32_t i, const int64_t* s, int64_t n, int64_t* out) {
    for (int64_t k = 0; k < n; ++k) out[k] = (kA[i] * s[k]) % kM[i];
}

void orc_rng_seed(uint64_t seed, uint32_t scene, uint32_t domain, uint32_t pass, uint64_t id,
                  int64_t* state4) {
    Rng r = rng_seed(seed, scene, domain, pass, id);
    for (int i = 0; i < 4; ++i) state4[i] = r.s[i];
}

float orc_rng_next(int64_t* state4) {
    Rng r;
    for (int i = 0; i < 4; ++i) r.s[i] = state4[i];
    float u = rng_next(r);
    for (int i = 0; i < 4; ++i) state4[i] = r.s[i];
    return u;
}

// out[k * ndraw + j] = draw j of stream (seed, scene, domain, pass, ids[k])
void orc_rng_draws(uint64_t seed, uint32_t scene, uint32_t domain, uint32_t pass,
                   const uint64_t* ids, int64_t nid, int32_t ndraw, float* out) {
    for (int64_t k = 0; k < nid; ++k) {
        Rng r = rng_seed(seed, scene, domain, pass, ids[k]);
        for (int j = 0; j < ndraw; ++j) out[k * ndraw + j] = rng_next(r);
    }
}

uint64_t orc_splitmix64(uint64_t x) { return splitmix64(x); }

// ---- geometry ----
void* orc_mesh_create(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                      const int32_t* tri_mat) {
    Mesh* M = new Mesh;
    M->tris.resize(nt);
    for (int64_t i = 0; i < nt; ++i) {
        V3 p[3];
        for (int k = 0; k < 3; ++k) {
            const float* q = verts + 3 * (int64_t)tris[3 * i + k];
            p[k] = {(double)q[0], (double)q[1], (double)q[2]};
        }
        Tri& T = M->tris[i];
        T.v0 = p[0];
        T.e1 = p[1] - p[0];
        T.e2 = p[2] - p[0];
        V3 c = cross(T.e1, T.e2);
        double cn = norm(c);
        T.area = 0.5 * cn;
        T.n = cn > 0 ? c * (1.0 / cn) : V3{0, 0, 0};
        T.mat = tri_mat ? tri_mat[i] : 0;
    }
    (void)nv;
    bvh_build(*M);
    return M;
}

void orc_mesh_destroy(void* m) { delete (Mesh*)m; }

// Per-vertex normals [nv][3] (NULL: face normals) and texture coordinates [nv][2] (NULL: none),
// gathered per triangle through the index buffer. Returns -1 on a zero normal.
int32_t orc_mesh_set_attributes(void* mesh, const float* normals, const float* st, const int32_t* tris,
                                int64_t nt) {
    Mesh& M = *(Mesh*)mesh;
    if ((int64_t)M.tris.size() != nt) return -1;
    M.shade.assign(nt, Shading{});
    for (int64_t i = 0; i < nt; ++i) {
        Shading& A = M.shade[i];
        A.normals = normals != nullptr;
        for (int k = 0; k < 3; ++k) {
            const int64_t v = tris[3 * i + k];
            if (normals) {
                A.n[k] = {normals[3 * v], normals[3 * v + 1], normals[3 * v + 2]};
                if (!(norm(A.n[k]) > 0)) return -1;
            }
            A.st[k][0] = st ? st[2 * v] : 0.0;
            A.st[k][1] = st ? st[2 * v + 1] : 0.0;
        }
    }
    return 0;
}

// rays: [n][8] = ox oy oz tmin dx dy dz tmax. mode 0 = brute force, 1 = oracle BVH.
// nondeg may be null.
void orc_closest_hit(void* mesh, const float* rays, int64_t n, int32_t mode, int32_t* out_id,
                     double* out_t, double* out_u, double* out_v, int32_t* nondeg, int nthreads) {
    const Mesh& M = *(const Mesh*)mesh;
    parallel_for(n, nthreads, [&](int64_t a, int64_t b, int) {
        for (int64_t i = a; i < b; ++i) {
            const float* r = rays + 8 * i;
            V3 o{r[0], r[1], r[2]}, d{r[4], r[5], r[6]};
            double tmin = r[3], tmax = r[7];
            Hit h = mode == 0 ? closest_brute(M, o, d, tmin, tmax) : closest_bvh(M, o, d, tmin, tmax);
            out_id[i] = h.id;
            if (out_t) out_t[i] = h.id >= 0 ? h.t : INFINITY;
            if (out_u) out_u[i] = h.u;
            if (out_v) out_v[i] = h.v;
            if (nondeg) nondeg[i] = classify(M, mode == 0, o, d, tmin, tmax, h) ? 1 : 0;
        }
    });
}

// Binned SAH split of a set of triangles (Sec. 3.1 builds the tree top-down with the surface
// area heuristic on the CPU, after Wald 2007), written out plainly: the centroid of a triangle
// is the centre of its bounding box; along each axis whose centroid extent is positive the
// centroid range is cut into `bins` equal bins (a centroid at the top end belongs to the last
// bin); each boundary b = 1 .. bins-1 splits the set into the triangles of bins < b (left) and
// of bins >= b (right); its cost is 1 + (A_L N_L + A_R N_R) / A_P with A the surface area of the
// bounding box of the triangles on each side and of the whole set. Every (axis, boundary) with
// two non-empty sides is evaluated from scratch; the cheapest wins, the first in (axis,
// boundary) order on ties. Returns 1 and (axis, boundary, cost) if such a split exists, else 0;
// left[i] = 1 if subset[i] goes to the left side of the split. *near_bin receives the smallest distance, in bin widths, of any centroid from an interior bin
// boundary on any axis (a build that bins in FP32 may put such a centroid in the other bin).
int32_t orc_sah_split(const float* verts, const int32_t* tris, const int32_t* subset, int64_t n,
                      int32_t bins, int32_t* out_axis, int32_t* out_boundary, double* out_cost,
                      double* near_bin, int32_t* left) {
    std::vector<V3> lo(n), hi(n), cen(n);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t t = subset[i];
        V3 p[3];
        for (int k = 0; k < 3; ++k) {
            const float* q = verts + 3 * (int64_t)tris[3 * t + k];
            p[k] = {(double)q[0], (double)q[1], (double)q[2]};
        }
        lo[i] = {std::min({p[0].x, p[1].x, p[2].x}), std::min({p[0].y, p[1].y, p[2].y}),
                 std::min({p[0].z, p[1].z, p[2].z})};
        hi[i] = {std::max({p[0].x, p[1].x, p[2].x}), std::max({p[0].y, p[1].y, p[2].y}),
                 std::max({p[0].z, p[1].z, p[2].z})};
        cen[i] = (lo[i] + hi[i]) * 0.5;
    }
    auto area = [](const V3& a, const V3& b) {
        const double dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    };
    V3 plo{INFINITY, INFINITY, INFINITY}, phi{-INFINITY, -INFINITY, -INFINITY};
    V3 clo = plo, chi = phi;
    for (int64_t i = 0; i < n; ++i) {
        plo = {std::min(plo.x, lo[i].x), std::min(plo.y, lo[i].y), std::min(plo.z, lo[i].z)};
        phi = {std::max(phi.x, hi[i].x), std::max(phi.y, hi[i].y), std::max(phi.z, hi[i].z)};
        clo = {std::min(clo.x, cen[i].x), std::min(clo.y, cen[i].y), std::min(clo.z, cen[i].z)};
        chi = {std::max(chi.x, cen[i].x), std::max(chi.y, cen[i].y), std::max(chi.z, cen[i].z)};
    }
    const double ap = area(plo, phi);
    double best = INFINITY, nearest = INFINITY;
    int best_axis = -1, best_b = -1;
    std::vector<int> bin(n), best_bin;
    for (int a = 0; a < 3; ++a) {
        const double ext = comp(chi, a) - comp(clo, a);
        if (!(ext > 0)) continue;
        for (int64_t i = 0; i < n; ++i) {
            const double q = bins * (comp(cen[i], a) - comp(clo, a)) / ext;
            bin[i] = std::min(bins - 1, (int)std::floor(q));
            const double dist = std::fabs(q - std::round(q));
            if (q > 0.5 && q < bins - 0.5) nearest = std::min(nearest, dist);
        }
        for (int b = 1; b < bins; ++b) {
            V3 llo{INFINITY, INFINITY, INFINITY}, lhi{-INFINITY, -INFINITY, -INFINITY};
            V3 rlo = llo, rhi = lhi;
            int64_t nl = 0, nr = 0;
            for (int64_t i = 0; i < n; ++i) {
                V3 &L = bin[i] < b ? llo : rlo, &H = bin[i] < b ? lhi : rhi;
                L = {std::min(L.x, lo[i].x), std::min(L.y, lo[i].y), std::min(L.z, lo[i].z)};
                H = {std::max(H.x, hi[i].x), std::max(H.y, hi[i].y), std::max(H.z, hi[i].z)};
                (bin[i] < b ? nl : nr) += 1;
            }
            if (nl == 0 || nr == 0) continue;
            const double c = 1.0 + (area(llo, lhi) * (double)nl + area(rlo, rhi) * (double)nr) / ap;
            if (c < best) {
                best = c;
                best_axis = a;
                best_b = b;
                best_bin = bin;
            }
        }
    }
    *near_bin = nearest;
    if (best_axis < 0) return 0;
    *out_axis = best_axis;
    *out_boundary = best_b;
    *out_cost = best;
    for (int64_t i = 0; i < n; ++i) left[i] = best_bin[i] < best_b ? 1 : 0;
    return 1;
}

// Moller-Trumbore on one triangle (for closed-form tests).
int32_t orc_mt(const float* v0, const float* v1, const float* v2, const float* ray, double* tuv) {
    Tri T;
    T.v0 = {v0[0], v0[1], v0[2]};
    T.e1 = V3{v1[0], v1[1], v1[2]} - T.v0;
    T.e2 = V3{v2[0], v2[1], v2[2]} - T.v0;
    MT m = mt_intersect({ray[0], ray[1], ray[2]}, {ray[4], ray[5], ray[6]}, T);
    tuv[0] = m.t;
    tuv[1] = m.u;
    tuv[2] = m.v;
    return mt_inside(m) ? 1 : 0;
}

}  // extern "C"

// ==========================================================================================
// SPPM (Sec. 2, 3.3, 3.4)
// ==========================================================================================
namespace {

const double kPi = 3.14159265358979323846;
enum { DIFFUSE = 0, MIRROR = 1, DIELECTRIC = 2, EMITTER = 3 };

// Derivative vectors (forward mode, for the gradient check): entry [c * NG + j] is the
// derivative of channel c with respect to parameter j; parameters 0..nmat-1 are the materials'
// albedos (same channel), parameter nmat is the emission of the single emitting material.
typedef std::vector<double> Deriv;

struct Photon {
    V3 x, din, phi;
    uint32_t id;
    float z;  // random depth (stochastic hashing)
    Deriv dphi;
};

struct HitPoint {
    bool valid;
    V3 x, n, w;
    int mat;
    Deriv dw;
    V3 tex;  // texture factor of the albedo at the hit point (1 without a texture)
};

// Albedo texture of a material: rgb factors, row-major [h][w][3]; w = 0 means none.
struct Texture {
    int w = 0, h = 0;
    std::vector<double> rgb;
};

struct Sppm {
    const Mesh* mesh;
    std::vector<orc_material> mats;
    std::vector<Texture> tex;  // per material
    orc_camera cam;
    orc_sppm_params P;
    V3 eye, fwd, right, up;
    double th, aspect;
    std::vector<int> emitters;
    std::vector<double> cdf;
    double emit_total = 0;
    // per-pixel progressive state
    std::vector<double> N, R, tau, direct;
    int64_t passes = 0;
    double Ne = 0;
    // one-bounce-per-pass photon state (Sec. 3.3)
    std::vector<V3> ro, rd, rphi;
    std::vector<int> rdepth;
    std::vector<char> ralive;
    // forward-mode derivatives (grad mode only)
    bool grad = false;
    int NG = 0, emit_mat = -1;
    std::vector<double> dtau, ddirect;  // [npix][3 * NG]
    // last pass diagnostics
    std::vector<Photon> last_photons;
    std::vector<HitPoint> last_hits;
    std::vector<double> last_M, last_Phi;
};

V3 albedo(const orc_material& m) { return {m.albedo[0], m.albedo[1], m.albedo[2]}; }
V3 emission(const orc_material& m) { return {m.emission[0], m.emission[1], m.emission[2]}; }
bool emits(const orc_material& m) {
    return (m.type == DIFFUSE || m.type == EMITTER) &&
           std::max({m.emission[0], m.emission[1], m.emission[2]}) > 0.0f;
}

// Orthonormal basis around a unit vector: Duff et al., "Building an Orthonormal Basis,
// Revisited" (JCGT 2017).
void onb(const V3& n, V3& t1, V3& t2) {
    double sign = std::copysign(1.0, n.z);
    double a = -1.0 / (sign + n.z);
    double b = n.x * n.y * a;
    t1 = {1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x};
    t2 = {b, sign + n.y * n.y * a, -n.y};
}

V3 cosine_dir(const V3& n, float ua, float ub) {
    double r = std::sqrt((double)ua), phi = 2.0 * kPi * (double)ub;
    double z = std::sqrt(std::max(0.0, 1.0 - (double)ua));
    V3 t1, t2;
    onb(n, t1, t2);
    return t1 * (r * std::cos(phi)) + t2 * (r * std::sin(phi)) + n * z;
}

V3 reflect(const V3& d, const V3& n) { return d - n * (2.0 * dot(d, n)); }

// Dielectric interface: returns the new direction; u picks reflection with Fresnel
// probability F (exact unpolarised Fresnel), refraction otherwise.
V3 dielectric(const V3& d, const V3& n, double ior, float u) {
    bool front = dot(d, n) < 0;
    V3 nf = front ? n : n * -1.0;
    double n1 = front ? 1.0 : ior, n2 = front ? ior : 1.0;
    double eta = n1 / n2;
    double cosi = -dot(d, nf);
    double k = 1.0 - eta * eta * (1.0 - cosi * cosi);
    if (k < 0.0) return reflect(d, nf);
    double cost = std::sqrt(k);
    double rs = (n1 * cosi - n2 * cost) / (n1 * cosi + n2 * cost);
    double rp = (n2 * cosi - n1 * cost) / (n2 * cosi + n1 * cost);
    double F = 0.5 * (rs * rs + rp * rp);
    if ((double)u < F) return reflect(d, nf);
    return d * eta + nf * (eta * cosi - cost);
}

// Bilinear lookup with wrapping at texture coordinates (s, t): texel (i, j) covers
// [i/w, (i+1)/w) x [j/h, (j+1)/h) and holds its value at the centre; between centres the four
// nearest texels are blended with the usual bilinear weights, across the border with the texels
// of the opposite side.
V3 bilinear(const Texture& X, double s, double t) {
    s -= std::floor(s);
    t -= std::floor(t);
    const double x = s * X.w - 0.5, y = t * X.h - 0.5;
    const double x0 = std::floor(x), y0 = std::floor(y);
    const double fx = x - x0, fy = y - y0;
    auto wrap = [](int64_t i, int n) { return (int)(((i % n) + n) % n); };
    const int i0 = wrap((int64_t)x0, X.w), i1 = wrap((int64_t)x0 + 1, X.w);
    const int j0 = wrap((int64_t)y0, X.h), j1 = wrap((int64_t)y0 + 1, X.h);
    auto T = [&](int i, int j) {
        const double* q = &X.rgb[3 * ((size_t)j * X.w + i)];
        return V3{q[0], q[1], q[2]};
    };
    return T(i0, j0) * ((1 - fx) * (1 - fy)) + T(i1, j0) * (fx * (1 - fy)) + T(i0, j1) * ((1 - fx) * fy) +
           T(i1, j1) * (fx * fy);
}

// Shading at a hit: the shading normal (the blend of the vertex normals at the hit's
// barycentrics, normalised and turned into the geometric normal's hemisphere; the face normal
// without vertex normals) and the texture factor of a diffuse material's albedo.
struct Surface {
    V3 ns, tex;
    bool smooth;  // ns comes from vertex normals
};

Surface surface(const Sppm& S, const Hit& h) {
    const Tri& T = S.mesh->tris[h.id];
    Surface sf{T.n, {1, 1, 1}, false};
    if (S.mesh->shade.empty()) return sf;
    const Shading& A = S.mesh->shade[h.id];
    const double b0 = 1.0 - h.u - h.v, b1 = h.u, b2 = h.v;
    if (A.normals) {
        V3 n = A.n[0] * b0 + A.n[1] * b1 + A.n[2] * b2;
        const double l = norm(n);
        if (l > 0) {
            n = n * (1.0 / l);
            sf.ns = dot(n, T.n) < 0 ? n * -1.0 : n;
            sf.smooth = true;
        }
    }
    const Texture& X = S.tex[T.mat];
    if (X.w > 0 && S.mats[T.mat].type == 0) {  // diffuse
        const double s = A.st[0][0] * b0 + A.st[1][0] * b1 + A.st[2][0] * b2;
        const double t = A.st[0][1] * b0 + A.st[1][1] * b1 + A.st[2][1] * b2;
        sf.tex = bilinear(X, s, t);
    }
    return sf;
}

Hit trace(const Sppm& S, const V3& o, const V3& d, double tmin) {
    if (S.mesh->tris.size() <= 64) return closest_brute(*S.mesh, o, d, tmin, INFINITY);
    return closest_bvh(*S.mesh, o, d, tmin, INFINITY);
}

// Eye pass for one pixel: jittered pinhole ray, specular chain, first non-specular hit.
HitPoint eye_path(const Sppm& S, int64_t pix, V3& direct_add, double* ddirect_add) {
    HitPoint hp{false, {}, {}, {}, 0, {}};
    const int NG = S.NG;
    Deriv dw(S.grad ? 3 * NG : 0, 0.0);
    int W = S.cam.width, H = S.cam.height;
    int px = (int)(pix % W), py = (int)(pix / W);
    Rng rng = rng_seed(S.P.seed, S.P.scene_id, 0, (uint32_t)S.passes, (uint64_t)pix);
    float u0 = rng_next(rng), u1 = rng_next(rng);
    double sx = (((double)px + u0) / W * 2.0 - 1.0) * S.th * S.aspect;
    double sy = (1.0 - ((double)py + u1) / H * 2.0) * S.th;
    V3 d = normalize(S.fwd + S.right * sx + S.up * sy);
    V3 o = S.eye;
    V3 w{1, 1, 1};
    double tmin = 0.0;
    for (int depth = 0; depth <= S.P.max_eye_depth; ++depth) {
        Hit h = trace(S, o, d, tmin);
        if (h.id < 0) break;
        const Tri& T = S.mesh->tris[h.id];
        const orc_material& m = S.mats[T.mat];
        bool front = dot(d, T.n) < 0;
        if (emits(m) && front) {
            direct_add = direct_add + mul(w, emission(m));
            if (S.grad) {
                const double le[3] = {m.emission[0], m.emission[1], m.emission[2]}, wc[3] = {w.x, w.y, w.z};
                for (int c = 0; c < 3; ++c) {
                    for (int j = 0; j < NG; ++j) ddirect_add[c * NG + j] += dw[c * NG + j] * le[c];
                    if (T.mat == S.emit_mat) ddirect_add[c * NG + NG - 1] += wc[c];
                }
            }
        }
        if (m.type == EMITTER) break;
        V3 x = o + d * h.t;
        const Surface sf = surface(S, h);
        if (m.type == DIFFUSE) {
            hp = {true, x, front ? T.n : T.n * -1.0, w, T.mat, dw, sf.tex};
            break;
        }
        if (m.type == MIRROR) {
            if (S.grad) {  // w' = w * a_m
                const double a[3] = {m.albedo[0], m.albedo[1], m.albedo[2]}, wc[3] = {w.x, w.y, w.z};
                for (int c = 0; c < 3; ++c) {
                    for (int j = 0; j < NG; ++j) dw[c * NG + j] *= a[c];
                    dw[c * NG + T.mat] += wc[c];
                }
            }
            w = mul(w, albedo(m));
            d = reflect(d, sf.ns);
        } else {  // dielectric
            float uf = rng_next(rng);
            d = dielectric(d, sf.ns, m.ior, uf);
        }
        o = x;
        tmin = S.P.eps;
    }
    return hp;
}

// Photon emission: pick an emitting triangle with probability proportional to
// area * mean(Le), a uniform point on it, a cosine-distributed direction about its normal.
void emit(const Sppm& S, Rng& rng, V3& o, V3& d, V3& phi, Deriv* dphi) {
    float u0 = rng_next(rng);
    size_t j = std::upper_bound(S.cdf.begin(), S.cdf.end(), (double)u0) - S.cdf.begin();
    if (j >= S.emitters.size()) j = S.emitters.size() - 1;
    const Tri& T = S.mesh->tris[S.emitters[j]];
    const orc_material& m = S.mats[T.mat];
    float u1 = rng_next(rng), u2 = rng_next(rng);
    double su = std::sqrt((double)u1);
    o = T.v0 + T.e1 * (su * (1.0 - (double)u2)) + T.e2 * (su * (double)u2);
    float u3 = rng_next(rng), u4 = rng_next(rng);
    d = cosine_dir(T.n, u3, u4);
    V3 le = emission(m);
    double mean = (le.x + le.y + le.z) / 3.0;
    phi = le * (kPi * S.emit_total / mean);
    if (dphi) {  // one emitting material: phi_c = pi * A * Le_c, linear in Le_c
        dphi->assign(3 * S.NG, 0.0);
        const double pc[3] = {phi.x, phi.y, phi.z}, lc[3] = {le.x, le.y, le.z};
        for (int c = 0; c < 3; ++c) (*dphi)[c * S.NG + S.NG - 1] = lc[c] > 0 ? pc[c] / lc[c] : kPi * S.emit_total / mean;
    }
}

enum Step { CONTINUE, STOP };

// One photon bounce at a hit (shared by both photon modes). Appends a deposit at diffuse hits.
Step photon_bounce(const Sppm& S, Rng& rng, const Hit& h, V3& o, V3& d, V3& phi, uint32_t id,
                   std::vector<Photon>& out, Deriv* dphi) {
    const Tri& T = S.mesh->tris[h.id];
    const orc_material& m = S.mats[T.mat];
    if (m.type == EMITTER) return STOP;
    V3 x = o + d * h.t;
    const Surface sf = surface(S, h);
    if (m.type == DIFFUSE) {
        Photon p{x, d, phi, id, 0.0f, dphi ? *dphi : Deriv()};
        if (S.P.hash_mode == 1) p.z = rng_next(rng);
        out.push_back(p);
        float urr = rng_next(rng);
        if (!((double)urr < (double)S.P.rr_continue)) return STOP;
        if (dphi) {  // phi' = phi * rho_m * tex / p_c
            const double rr = (double)S.P.rr_continue, a[3] = {m.albedo[0], m.albedo[1], m.albedo[2]},
                         pc[3] = {phi.x, phi.y, phi.z}, tx[3] = {sf.tex.x, sf.tex.y, sf.tex.z};
            for (int c = 0; c < 3; ++c) {
                for (int j = 0; j < S.NG; ++j) (*dphi)[c * S.NG + j] *= a[c] * tx[c] / rr;
                (*dphi)[c * S.NG + T.mat] += pc[c] * tx[c] / rr;
            }
        }
        phi = mul(mul(phi, albedo(m)), sf.tex) * (1.0 / (double)S.P.rr_continue);
        const bool fr = dot(d, T.n) < 0;
        V3 ns = fr ? sf.ns : sf.ns * -1.0;
        float ua = rng_next(rng), ub = rng_next(rng);
        d = cosine_dir(ns, ua, ub);
        // a direction sampled about a shading normal can point into the surface: the path ends
        if (sf.smooth && !(dot(d, fr ? T.n : T.n * -1.0) > 0)) return STOP;
    } else if (m.type == MIRROR) {
        if (dphi) {  // phi' = phi * a_m
            const double a[3] = {m.albedo[0], m.albedo[1], m.albedo[2]}, pc[3] = {phi.x, phi.y, phi.z};
            for (int c = 0; c < 3; ++c) {
                for (int j = 0; j < S.NG; ++j) (*dphi)[c * S.NG + j] *= a[c];
                (*dphi)[c * S.NG + T.mat] += pc[c];
            }
        }
        phi = mul(phi, albedo(m));
        d = reflect(d, sf.ns);
    } else {
        float uf = rng_next(rng);
        d = dielectric(d, sf.ns, m.ior, uf);
    }
    o = x;
    return CONTINUE;
}

// Photon tracing stage, whole paths per pass.
void photons_full(Sppm& S, int64_t k, std::vector<Photon>& out) {
    Rng rng = rng_seed(S.P.seed, S.P.scene_id, 1, (uint32_t)S.passes, (uint64_t)k);
    V3 o, d, phi;
    Deriv dphi;
    emit(S, rng, o, d, phi, S.grad ? &dphi : nullptr);
    for (int depth = 0; depth < S.P.max_photon_depth; ++depth) {
        Hit h = trace(S, o, d, S.P.eps);
        if (h.id < 0) return;
        if (photon_bounce(S, rng, h, o, d, phi, (uint32_t)(k * 32 + depth), out, S.grad ? &dphi : nullptr) == STOP)
            return;
    }
}

// Photon tracing stage, one bounce per pass with path regeneration (Sec. 3.3).
// Returns 1 if a new path was started.
int photons_regen(Sppm& S, int64_t j, std::vector<Photon>& out) {
    Rng rng = rng_seed(S.P.seed, S.P.scene_id, 1, (uint32_t)S.passes, (uint64_t)j);
    int started = 0;
    if (!S.ralive[j]) {
        emit(S, rng, S.ro[j], S.rd[j], S.rphi[j], nullptr);
        S.rdepth[j] = 0;
        S.ralive[j] = 1;
        started = 1;
    }
    Hit h = trace(S, S.ro[j], S.rd[j], S.P.eps);
    if (h.id < 0) {
        S.ralive[j] = 0;
        return started;
    }
    if (photon_bounce(S, rng, h, S.ro[j], S.rd[j], S.rphi[j], (uint32_t)j, out, nullptr) == STOP) {
        S.ralive[j] = 0;
        return started;
    }
    if (++S.rdepth[j] >= S.P.max_photon_depth) S.ralive[j] = 0;
    return started;
}

struct CellKey {
    int64_t x, y, z;
    bool operator==(const CellKey& o) const { return x == o.x && y == o.y && z == o.z; }
};
struct CellHash {
    size_t operator()(const CellKey& k) const {
        return (size_t)(k.x * 1000003 + k.y * 10007 + k.z * 101);
    }
};

// Hash-grid cell of a coordinate. Sec. 3.4 does not fix the lattice; it is shifted by 0.381966
// of a cell so that axis-aligned walls at multiples of h (a scene's bounding planes are often at
// 0) do not lie on cell boundaries, where rounding alone would pick the cell.
const double kCellOffset = 0.381966;
inline int64_t cell_of(double x, double h) { return (int64_t)std::floor(x / h + kCellOffset); }

// Teschner et al. 2003 spatial hash, 32-bit wraparound, table size a power of two.
inline uint32_t teschner(int64_t ix, int64_t iy, int64_t iz, uint64_t T) {
    uint32_t h = ((uint32_t)(int32_t)ix * 73856093u) ^ ((uint32_t)(int32_t)iy * 19349663u) ^
                 ((uint32_t)(int32_t)iz * 83492791u);
    return h & (uint32_t)(T - 1);
}

void sppm_pass(Sppm& S, int nthreads) {
    const int64_t npix = (int64_t)S.cam.width * S.cam.height;
    // ---- eye tracing stage ----
    std::vector<HitPoint> hits(npix);
    std::vector<V3> dadd(npix, V3{0, 0, 0});
    const int NG = S.NG, G3 = 3 * S.NG;
    parallel_for(npix, nthreads, [&](int64_t a, int64_t b, int) {
        for (int64_t p = a; p < b; ++p)
            hits[p] = eye_path(S, p, dadd[p], S.grad ? &S.ddirect[(size_t)p * G3] : nullptr);
    });
    for (int64_t p = 0; p < npix; ++p) {
        S.direct[3 * p] += dadd[p].x;
        S.direct[3 * p + 1] += dadd[p].y;
        S.direct[3 * p + 2] += dadd[p].z;
    }
    // ---- photon tracing stage ----
    const int64_t np = S.P.photons_per_pass;
    std::vector<std::vector<Photon>> chunks(std::max(1, nthreads));
    std::vector<int64_t> started(std::max(1, nthreads), 0);
    parallel_for(np, nthreads, [&](int64_t a, int64_t b, int t) {
        for (int64_t k = a; k < b; ++k) {
            if (S.P.photon_mode == 0)
                photons_full(S, k, chunks[t]);
            else
                started[t] += photons_regen(S, k, chunks[t]);
        }
    });
    std::vector<Photon> ph;
    for (auto& c : chunks) ph.insert(ph.end(), c.begin(), c.end());
    if (S.P.photon_mode == 0)
        S.Ne += (double)np;
    else
        for (auto s : started) S.Ne += (double)s;
    // ---- range query + progressive density estimation ----
    std::vector<double> Mv(npix, 0.0), Phiv(3 * npix, 0.0);
    std::vector<double> dPhiv(S.grad ? (size_t)npix * G3 : 0, 0.0);
    // d(f * phi_k) for f = w * rho_{m_p} / pi (the hit point's weight), scaled by `scale`
    auto add_dflux = [&](const HitPoint& hp, const Photon& q, double scale, double* out) {
        const orc_material& m = S.mats[hp.mat];
        // f = w * rho_m * tex / pi: tex is a constant factor of the albedo
        const double tx[3] = {hp.tex.x, hp.tex.y, hp.tex.z},
                     a[3] = {m.albedo[0] * tx[0], m.albedo[1] * tx[1], m.albedo[2] * tx[2]},
                     wc[3] = {hp.w.x, hp.w.y, hp.w.z}, pc[3] = {q.phi.x, q.phi.y, q.phi.z};
        for (int c = 0; c < 3; ++c) {
            const double f = wc[c] * a[c] / kPi;
            for (int j = 0; j < NG; ++j)
                out[c * NG + j] += scale * (hp.dw[c * NG + j] * a[c] / kPi * pc[c] + f * q.dphi[c * NG + j]);
            out[c * NG + hp.mat] += scale * wc[c] * tx[c] / kPi * pc[c];
        }
    };
    const double h = S.P.cell_h;
    if (S.P.hash_mode == 0) {
        // exact: every photon within R (cells are only an index, keyed exactly, no hashing)
        std::unordered_map<CellKey, std::vector<int>, CellHash> grid;
        for (int i = 0; i < (int)ph.size(); ++i)
            grid[{cell_of(ph[i].x.x, h), cell_of(ph[i].x.y, h), cell_of(ph[i].x.z, h)}].push_back(i);
        parallel_for(npix, nthreads, [&](int64_t a, int64_t b, int) {
            std::vector<int> acc;
            for (int64_t p = a; p < b; ++p) {
                if (!hits[p].valid) continue;
                const HitPoint& hp = hits[p];
                double R = S.R[p];
                acc.clear();
                int64_t lo[3], hi[3];
                for (int k = 0; k < 3; ++k) {
                    lo[k] = cell_of(comp(hp.x, k) - R, h) - 1;
                    hi[k] = cell_of(comp(hp.x, k) + R, h) + 1;
                }
                for (int64_t cx = lo[0]; cx <= hi[0]; ++cx)
                    for (int64_t cy = lo[1]; cy <= hi[1]; ++cy)
                        for (int64_t cz = lo[2]; cz <= hi[2]; ++cz) {
                            auto it = grid.find({cx, cy, cz});
                            if (it == grid.end()) continue;
                            for (int i : it->second) {
                                V3 dx = ph[i].x - hp.x;
                                if (dot(dx, dx) < R * R && dot(ph[i].din, hp.n) < 0) acc.push_back(i);
                            }
                        }
                std::sort(acc.begin(), acc.end(), [&](int a2, int b2) { return ph[a2].id < ph[b2].id; });
                V3 f = mul(mul(hp.w, albedo(S.mats[hp.mat])), hp.tex) * (1.0 / kPi);
                V3 sum{0, 0, 0};
                for (int i : acc) sum = sum + mul(f, ph[i].phi);
                if (S.grad)
                    for (int i : acc) add_dflux(hp, ph[i], 1.0, &dPhiv[(size_t)p * G3]);
                Mv[p] = (double)acc.size();
                Phiv[3 * p] = sum.x;
                Phiv[3 * p + 1] = sum.y;
                Phiv[3 * p + 2] = sum.z;
            }
        });
    } else {
        // stochastic hashing (Sec. 3.4): one survivor per entry = minimum (random depth, id)
        const uint64_t T = (uint64_t)S.P.table_size;
        std::vector<uint64_t> key(T, ~0ull);
        std::vector<int64_t> cnt(T, 0);
        std::vector<int> surv(T, -1);
        for (int i = 0; i < (int)ph.size(); ++i) {
            uint32_t b = teschner(cell_of(ph[i].x.x, h), cell_of(ph[i].x.y, h), cell_of(ph[i].x.z, h), T);
            uint32_t zb;
            std::memcpy(&zb, &ph[i].z, 4);
            uint64_t k = ((uint64_t)zb << 32) | ph[i].id;
            cnt[b] += 1;
            if (k < key[b]) {
                key[b] = k;
                surv[b] = i;
            }
        }
        parallel_for(npix, nthreads, [&](int64_t a, int64_t b, int) {
            for (int64_t p = a; p < b; ++p) {
                if (!hits[p].valid) continue;
                const HitPoint& hp = hits[p];
                double R = S.R[p];
                int64_t lo[3], hi[3];
                for (int k = 0; k < 3; ++k) {
                    lo[k] = cell_of(comp(hp.x, k) - R, h);
                    hi[k] = cell_of(comp(hp.x, k) + R, h);
                }
                V3 f = mul(mul(hp.w, albedo(S.mats[hp.mat])), hp.tex) * (1.0 / kPi);
                V3 sum{0, 0, 0};
                double M = 0;
                for (int64_t cx = lo[0]; cx <= hi[0]; ++cx)
                    for (int64_t cy = lo[1]; cy <= hi[1]; ++cy)
                        for (int64_t cz = lo[2]; cz <= hi[2]; ++cz) {
                            uint32_t bb = teschner(cx, cy, cz, T);
                            if (cnt[bb] == 0) continue;
                            const Photon& q = ph[surv[bb]];
                            if (cell_of(q.x.x, h) != cx || cell_of(q.x.y, h) != cy ||
                                cell_of(q.x.z, h) != cz)
                                continue;
                            V3 dx = q.x - hp.x;
                            if (!(dot(dx, dx) < R * R && dot(q.din, hp.n) < 0)) continue;
                            M += (double)cnt[bb];
                            sum = sum + mul(f, q.phi) * (double)cnt[bb];
                            if (S.grad) add_dflux(hp, q, (double)cnt[bb], &dPhiv[(size_t)p * G3]);
                        }
                Mv[p] = M;
                Phiv[3 * p] = sum.x;
                Phiv[3 * p + 1] = sum.y;
                Phiv[3 * p + 2] = sum.z;
            }
        });
    }
    // progressive radius / flux / count update (Hachisuka & Jensen 2009)
    const double alpha = S.P.alpha;
    for (int64_t p = 0; p < npix; ++p) {
        double M = Mv[p];
        if (!(M > 0)) continue;
        double Nn = S.N[p] + alpha * M;
        double ratio = Nn / (S.N[p] + M);
        S.R[p] = S.R[p] * std::sqrt(ratio);
        for (int c = 0; c < 3; ++c) S.tau[3 * p + c] = (S.tau[3 * p + c] + Phiv[3 * p + c]) * ratio;
        if (S.grad)
            for (int g = 0; g < G3; ++g)
                S.dtau[(size_t)p * G3 + g] = (S.dtau[(size_t)p * G3 + g] + dPhiv[(size_t)p * G3 + g]) * ratio;
        S.N[p] = Nn;
    }
    S.passes += 1;
    S.last_photons.swap(ph);
    S.last_hits.swap(hits);
    S.last_M.swap(Mv);
    S.last_Phi.swap(Phiv);
}

}  // namespace

extern "C" {

void* orc_sppm_create(void* mesh, const orc_material* mats, int32_t nmat, const orc_camera* cam,
                      const orc_sppm_params* params) {
    Sppm* S = new Sppm;
    S->mesh = (const Mesh*)mesh;
    S->mats.assign(mats, mats + nmat);
    S->cam = *cam;
    S->P = *params;
    S->eye = {cam->eye[0], cam->eye[1], cam->eye[2]};
    V3 look{cam->look[0], cam->look[1], cam->look[2]}, up{cam->up[0], cam->up[1], cam->up[2]};
    S->fwd = normalize(look - S->eye);
    S->right = normalize(cross(S->fwd, up));
    S->up = cross(S->right, S->fwd);
    S->th = std::tan((double)cam->vfov_deg * kPi / 180.0 / 2.0);
    S->aspect = (double)cam->width / (double)cam->height;
    // emitter distribution (area * mean emission), in triangle order
    double acc = 0;
    for (int i = 0; i < (int)S->mesh->tris.size(); ++i) {
        const Tri& T = S->mesh->tris[i];
        const orc_material& m = S->mats[T.mat];
        if (!emits(m) || !(T.area > 0)) continue;
        V3 le = emission(m);
        S->emitters.push_back(i);
        acc += T.area * (le.x + le.y + le.z) / 3.0;
        S->cdf.push_back(acc);
    }
    for (auto& c : S->cdf) c /= acc;
    S->emit_total = acc;
    int64_t npix = (int64_t)cam->width * cam->height;
    S->N.assign(npix, 0.0);
    S->R.assign(npix, (double)params->r0);
    S->tau.assign(3 * npix, 0.0);
    S->direct.assign(3 * npix, 0.0);
    S->tex.assign(nmat, Texture{});
    int64_t np = params->photons_per_pass;
    S->ro.assign(np, V3{0, 0, 0});
    S->rd.assign(np, V3{0, 0, 0});
    S->rphi.assign(np, V3{0, 0, 0});
    S->rdepth.assign(np, 0);
    S->ralive.assign(np, 0);
    return S;
}

void orc_sppm_destroy(void* s) { delete (Sppm*)s; }

// Albedo texture of material `mat`: rgb [h][w][3] (applies to diffuse materials).
int32_t orc_sppm_set_texture(void* s, int32_t mat, const float* rgb, int32_t w, int32_t h) {
    Sppm* S = (Sppm*)s;
    if (mat < 0 || mat >= (int32_t)S->mats.size() || w < 1 || h < 1 || !rgb) return -1;
    Texture& X = S->tex[mat];
    X.w = w;
    X.h = h;
    X.rgb.assign(rgb, rgb + 3 * (size_t)w * h);
    return 0;
}

// Shading at the closest hit of each ray [n][8]: out[n][10] = id, u, v, shading normal (3),
// texture factor (3), 1 if the normal comes from vertex normals (id -1: no hit).
void orc_sppm_surface(void* s, const float* rays, int64_t n, double* out) {
    const Sppm& S = *(const Sppm*)s;
    for (int64_t i = 0; i < n; ++i) {
        const float* r = rays + 8 * i;
        V3 o{r[0], r[1], r[2]}, d{r[4], r[5], r[6]};
        const Mesh& M = *S.mesh;
        Hit h = M.tris.size() <= 64 ? closest_brute(M, o, d, r[3], r[7]) : closest_bvh(M, o, d, r[3], r[7]);
        double* q = out + 10 * i;
        std::fill(q, q + 10, 0.0);
        q[0] = h.id;
        if (h.id < 0) continue;
        const Surface sf = surface(S, h);
        q[1] = h.u;
        q[2] = h.v;
        q[3] = sf.ns.x; q[4] = sf.ns.y; q[5] = sf.ns.z;
        q[6] = sf.tex.x; q[7] = sf.tex.y; q[8] = sf.tex.z;
        q[9] = sf.smooth ? 1.0 : 0.0;
    }
}

int32_t orc_sppm_run(void* s, int32_t npasses, int32_t nthreads) {
    Sppm* S = (Sppm*)s;
    if (S->emitters.empty()) return -1;
    for (int i = 0; i < npasses; ++i) sppm_pass(*S, nthreads);
    return 0;
}

// Per-pixel state and the final estimate L = direct/P + tau / (pi R^2 N_e).
void orc_sppm_state(void* s, double* N, double* R, double* tau, double* direct, double* image,
                    double* ne_passes) {
    Sppm* S = (Sppm*)s;
    int64_t npix = (int64_t)S->cam.width * S->cam.height;
    for (int64_t p = 0; p < npix; ++p) {
        if (N) N[p] = S->N[p];
        if (R) R[p] = S->R[p];
        for (int c = 0; c < 3; ++c) {
            if (tau) tau[3 * p + c] = S->tau[3 * p + c];
            if (direct) direct[3 * p + c] = S->direct[3 * p + c];
            if (image) {
                double L = S->passes > 0 ? S->direct[3 * p + c] / (double)S->passes : 0.0;
                if (S->Ne > 0) L += S->tau[3 * p + c] / (kPi * S->R[p] * S->R[p] * S->Ne);
                image[3 * p + c] = L;
            }
        }
    }
    if (ne_passes) {
        ne_passes[0] = S->Ne;
        ne_passes[1] = (double)S->passes;
    }
}

// Diagnostics of the last pass: number of deposits, then (if arrays given) their ids and
// positions, and the per-pixel photon count M and flux sum.
int64_t orc_sppm_last_photons(void* s, uint32_t* ids, double* x, double* phi, double* din) {
    Sppm* S = (Sppm*)s;
    int64_t n = (int64_t)S->last_photons.size();
    for (int64_t i = 0; i < n; ++i) {
        const Photon& p = S->last_photons[i];
        if (ids) ids[i] = p.id;
        if (x) { x[3 * i] = p.x.x; x[3 * i + 1] = p.x.y; x[3 * i + 2] = p.x.z; }
        if (phi) { phi[3 * i] = p.phi.x; phi[3 * i + 1] = p.phi.y; phi[3 * i + 2] = p.phi.z; }
        if (din) { din[3 * i] = p.din.x; din[3 * i + 1] = p.din.y; din[3 * i + 2] = p.din.z; }
    }
    return n;
}

void orc_sppm_last_gather(void* s, double* M, double* Phi, int32_t* valid, double* hitx,
                          double* hitn, double* hitw, int32_t* hitmat) {
    Sppm* S = (Sppm*)s;
    int64_t npix = (int64_t)S->cam.width * S->cam.height;
    for (int64_t p = 0; p < npix; ++p) {
        if (M) M[p] = S->last_M.empty() ? 0 : S->last_M[p];
        for (int c = 0; c < 3; ++c)
            if (Phi) Phi[3 * p + c] = S->last_Phi.empty() ? 0 : S->last_Phi[3 * p + c];
        const HitPoint& h = S->last_hits[p];
        if (valid) valid[p] = h.valid ? 1 : 0;
        if (hitx) { hitx[3 * p] = h.x.x; hitx[3 * p + 1] = h.x.y; hitx[3 * p + 2] = h.x.z; }
        if (hitn) { hitn[3 * p] = h.n.x; hitn[3 * p + 1] = h.n.y; hitn[3 * p + 2] = h.n.z; }
        if (hitw) { hitw[3 * p] = h.w.x; hitw[3 * p + 1] = h.w.y; hitw[3 * p + 2] = h.w.z; }
        if (hitmat) hitmat[p] = h.mat;
    }
}

// Sampling primitives, exported for distribution tests.
void orc_cosine_dir(const double* n, float ua, float ub, double* out) {
    V3 d = cosine_dir({n[0], n[1], n[2]}, ua, ub);
    out[0] = d.x; out[1] = d.y; out[2] = d.z;
}

void orc_dielectric(const double* d, const double* n, double ior, float u, double* out) {
    V3 r = dielectric({d[0], d[1], d[2]}, {n[0], n[1], n[2]}, ior, u);
    out[0] = r.x; out[1] = r.y; out[2] = r.z;
}

// Exact hash grid of a point set (the index the deposit builds, Sec. 3.4's regular hashing):
// bucket of each point, points ordered by (bucket, input index), and bucket starts [T + 1].
// near[i] = 1 when a coordinate lies within 1e-5 + 1e-6 |x/h| cells of a cell boundary: an FP32
// evaluation of x/h + offset errs by up to about 1.2e-7 |x/h|, so FP32 and FP64 may then pick
// different cells.
void orc_hash_grid(const float* xyz, int64_t n, double h, int64_t T, uint32_t* bucket,
                   uint32_t* order, uint32_t* bstart, int32_t* near) {
    std::vector<std::pair<uint32_t, int64_t>> key(n);
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        bool nb = false;
        for (int k = 0; k < 3; ++k) {
            double q = (double)xyz[3 * i + k] / h + kCellOffset;
            c[k] = (int64_t)std::floor(q);
            double fr = q - std::floor(q);
            const double tol = 1e-5 + 1e-6 * std::fabs(q);
            nb = nb || fr < tol || fr > 1.0 - tol;
        }
        uint32_t b = teschner(c[0], c[1], c[2], (uint64_t)T);
        key[i] = {b, i};
        if (bucket) bucket[i] = b;
        if (near) near[i] = nb ? 1 : 0;
    }
    std::stable_sort(key.begin(), key.end(),
                     [](const std::pair<uint32_t, int64_t>& a, const std::pair<uint32_t, int64_t>& b) {
                         return a.first < b.first;
                     });
    for (int64_t i = 0; i < n; ++i) order[i] = (uint32_t)key[i].second;
    int64_t j = 0;
    for (int64_t b = 0; b <= T; ++b) {
        while (j < n && key[j].first < b) ++j;
        bstart[b] = (uint32_t)j;
    }
}

// Forward-mode derivatives for the gradient check (whole paths per pass only). Must be called
// before the first pass. Returns -1 unless exactly one material emits.
int32_t orc_sppm_enable_grad(void* s) {
    Sppm* S = (Sppm*)s;
    if (S->passes != 0 || S->P.photon_mode != 0) return -1;
    int em = -1;
    for (int m = 0; m < (int)S->mats.size(); ++m)
        if (emits(S->mats[m])) {
            if (em >= 0) return -1;
            em = m;
        }
    if (em < 0) return -1;
    S->grad = true;
    S->emit_mat = em;
    S->NG = (int)S->mats.size() + 1;
    int64_t npix = (int64_t)S->cam.width * S->cam.height;
    S->dtau.assign((size_t)npix * 3 * S->NG, 0.0);
    S->ddirect.assign((size_t)npix * 3 * S->NG, 0.0);
    return 0;
}

// Gradient of sum_p sum_c g[p][c] * L[p][c] (for L2 loss, g = L - target) with respect to every
// material's albedo (grad_albedo [nmat][3]) and the emitting material's emission (grad_le [3]):
// dL/dtheta = d(direct)/dtheta / P + d(tau)/dtheta / (pi R^2 N_e).
int32_t orc_sppm_grad(void* s, const double* g, double* grad_albedo, double* grad_le) {
    Sppm* S = (Sppm*)s;
    if (!S->grad || S->passes == 0) return -1;
    const int NG = S->NG, nm = NG - 1;
    const int64_t npix = (int64_t)S->cam.width * S->cam.height;
    std::vector<double> acc(3 * NG, 0.0);
    for (int64_t p = 0; p < npix; ++p) {
        const double kd = 1.0 / (double)S->passes, kt = 1.0 / (kPi * S->R[p] * S->R[p] * S->Ne);
        for (int c = 0; c < 3; ++c)
            for (int j = 0; j < NG; ++j) {
                const size_t i = (size_t)p * 3 * NG + c * NG + j;
                acc[c * NG + j] += g[3 * p + c] * (S->ddirect[i] * kd + S->dtau[i] * kt);
            }
    }
    for (int m = 0; m < nm; ++m)
        for (int c = 0; c < 3; ++c) grad_albedo[3 * m + c] = acc[c * NG + m];
    for (int c = 0; c < 3; ++c) grad_le[c] = acc[c * NG + nm];
    return 0;
}

// The progressive update alone, for recurrence tests: applies one pass with counts M and
// fluxes Phi to (N, R, tau) arrays in place.
void orc_sppm_update(int64_t n, double alpha, const double* M, const double* Phi, double* N,
                     double* R, double* tau) {
    for (int64_t p = 0; p < n; ++p) {
        if (!(M[p] > 0)) continue;
        double Nn = N[p] + alpha * M[p];
        double ratio = Nn / (N[p] + M[p]);
        R[p] *= std::sqrt(ratio);
        for (int c = 0; c < 3; ++c) tau[3 * p + c] = (tau[3 * p + c] + Phi[3 * p + c]) * ratio;
        N[p] = Nn;
    }
}

}  // extern "C"
