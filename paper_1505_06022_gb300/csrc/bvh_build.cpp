// bvh_build.cpp -- host BVH construction and threading (Sec. 3.1).
//
// The paper builds the BVH top-down with the SAH (Wald 2007) on the CPU, writes hit/miss links
// ("threading", Simonsen & Fahraeus) and uploads the result. The multiple-threaded BVH keeps
// six link sets, one per principal ray direction class, each in a preorder whose children are
// sorted front-to-back along that direction (Fig. 3).
//
// Here every link set gets its own node array laid out in its own preorder, so the hit link
// of an internal node is always index + 1 and only the miss link is stored. A node is two
// float4 (32 bytes): {min.xyz, miss} and {max.xyz, leaf word}. A triangle is three float4:
// {v0.xyz, triangle index}, {v1.xyz, 0}, {v2.xyz, 0}.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <numeric>
#include <thread>

#include "gsp_internal.h"

namespace {

struct BNode {
    float lo[3], hi[3];
    int32_t left = -1, right = -1;  // right == left + 1 for internal nodes
    int32_t first = 0, count = 0;
};

inline double half_area(const float lo[3], const float hi[3]) {
    double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1], dz = (double)hi[2] - lo[2];
    if (dx < 0 || dy < 0 || dz < 0) return 0.0;
    return dx * dy + dy * dz + dz * dx;
}

struct Bin {
    float lo[3], hi[3];
    int32_t n;
    void reset() {
        for (int k = 0; k < 3; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
        n = 0;
    }
    void grow(const float* a, const float* b) {
        for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], a[k]); hi[k] = std::max(hi[k], b[k]); }
    }
};

inline float as_float(int32_t i) { float f; std::memcpy(&f, &i, 4); return f; }
inline int32_t as_int(float f) { int32_t i; std::memcpy(&i, &f, 4); return i; }

}  // namespace

std::string bvh_build_host(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                           const gsp_bvh_params& p, HostBVH& out) {
    using clk = std::chrono::steady_clock;
    auto t0 = clk::now();
    if (nt <= 0) return "scene has no triangles";
    if (nt >= (int64_t(1) << 28)) return "more than 2^28 triangles";
    const int bins = p.bins, leaf_thr = p.leaf_threshold, max_leaf = p.max_leaf;

    // worker threads for the per-triangle pass, the subtrees and the link sets; the tree, and so
    // every output array, is the same for any number of threads
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nthreads = nt < 65536 ? 1 : (int)std::min(64u, hw);
    auto parallel_for = [&](int64_t n, auto&& fn) {  // fn(begin, end)
        if (nthreads == 1 || n < 4096) return fn((int64_t)0, n);
        std::vector<std::thread> th;
        const int64_t per = (n + nthreads - 1) / nthreads;
        for (int t = 0; t < nthreads; ++t) {
            const int64_t a = t * per, b = std::min(n, a + per);
            if (a < b) th.emplace_back([&fn, a, b] { fn(a, b); });
        }
        for (auto& x : th) x.join();
    };

    // per-triangle bounds and centroids
    std::vector<float> tlo(3 * nt), thi(3 * nt), cen(3 * nt);
    parallel_for(nt, [&](int64_t i0, int64_t i1) {
        for (int64_t i = i0; i < i1; ++i)
            for (int k = 0; k < 3; ++k) {
                float a = verts[3 * (int64_t)tris[3 * i] + k], b = verts[3 * (int64_t)tris[3 * i + 1] + k],
                      c = verts[3 * (int64_t)tris[3 * i + 2] + k];
                tlo[3 * i + k] = std::min({a, b, c});
                thi[3 * i + k] = std::max({a, b, c});
                cen[3 * i + k] = 0.5f * (tlo[3 * i + k] + thi[3 * i + k]);
            }
    });
    (void)nv;
    std::vector<int32_t> perm(nt);
    std::iota(perm.begin(), perm.end(), 0);
    // at most 2 nt - 1 nodes (every leaf holds a triangle); children are numbered after their
    // parent, in whatever order the workers split them
    std::vector<BNode> nodes((size_t)2 * nt);
    std::atomic<int32_t> next_node{1};
    std::atomic<int32_t> max_depth{1};
    std::atomic<int64_t> leaves{0};

    struct Job { int32_t node, first, count, depth; };
    // Splits node j: its bounds, then a leaf, or the binned SAH split (cost = 1 + (A_L N_L +
    // A_R N_R) / A_P) with the children's jobs handed to `push`.
    auto split = [&](const Job& j, std::vector<Bin>& binv, std::vector<Bin>& right, auto&& push) {
        int32_t d = max_depth.load(std::memory_order_relaxed);
        while (j.depth > d && !max_depth.compare_exchange_weak(d, j.depth)) {}
        float blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
        float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int32_t k = j.first; k < j.first + j.count; ++k) {
            int32_t t = perm[k];
            for (int a = 0; a < 3; ++a) {
                blo[a] = std::min(blo[a], tlo[3 * t + a]);
                bhi[a] = std::max(bhi[a], thi[3 * t + a]);
                clo[a] = std::min(clo[a], cen[3 * t + a]);
                chi[a] = std::max(chi[a], cen[3 * t + a]);
            }
        }
        BNode& nd = nodes[j.node];
        std::memcpy(nd.lo, blo, sizeof blo);
        std::memcpy(nd.hi, bhi, sizeof bhi);
        nd.first = j.first;
        nd.count = j.count;
        if (j.count <= leaf_thr) { ++leaves; return; }

        double best_cost = INFINITY;
        int best_axis = -1, best_split = -1;
        double ap = half_area(blo, bhi);
        float scale[3];
        for (int a = 0; a < 3; ++a) {
            float ext = chi[a] - clo[a];
            scale[a] = ext > 0 ? (float)bins * (1.0f - 1e-6f) / ext : 0.0f;
            for (int b = 0; b < bins; ++b) binv[a * bins + b].reset();
        }
        for (int32_t k = j.first; k < j.first + j.count; ++k) {
            int32_t t = perm[k];
            for (int a = 0; a < 3; ++a) {
                if (scale[a] == 0.0f) continue;
                int b = std::min(bins - 1, std::max(0, (int)((cen[3 * t + a] - clo[a]) * scale[a])));
                Bin& B = binv[a * bins + b];
                B.grow(&tlo[3 * t], &thi[3 * t]);
                B.n++;
            }
        }
        for (int a = 0; a < 3; ++a) {
            if (scale[a] == 0.0f) continue;
            Bin acc;
            acc.reset();
            for (int b = bins - 1; b > 0; --b) {
                acc.grow(binv[a * bins + b].lo, binv[a * bins + b].hi);
                acc.n += binv[a * bins + b].n;
                right[b] = acc;
            }
            acc.reset();
            for (int b = 0; b < bins - 1; ++b) {
                acc.grow(binv[a * bins + b].lo, binv[a * bins + b].hi);
                acc.n += binv[a * bins + b].n;
                const Bin& R = right[b + 1];
                if (acc.n == 0 || R.n == 0) continue;
                double c = 1.0 + (half_area(acc.lo, acc.hi) * acc.n + half_area(R.lo, R.hi) * R.n) /
                                     std::max(ap, 1e-300);
                if (c < best_cost) { best_cost = c; best_axis = a; best_split = b; }
            }
        }
        int32_t mid;
        if (best_axis < 0) {
            // every centroid coincides: split by position in the current order
            if (j.count <= max_leaf) { ++leaves; return; }
            mid = j.first + j.count / 2;
        } else {
            if (j.count <= max_leaf && (double)j.count <= best_cost) { ++leaves; return; }
            const int a = best_axis;
            const float lo_a = clo[a], sc = scale[a];
            auto it = std::stable_partition(perm.begin() + j.first, perm.begin() + j.first + j.count,
                                            [&](int32_t t) {
                                                int b = std::min(bins - 1, std::max(0, (int)((cen[3 * t + a] - lo_a) * sc)));
                                                return b <= best_split;
                                            });
            mid = (int32_t)(it - perm.begin());
            if (mid == j.first || mid == j.first + j.count) mid = j.first + j.count / 2;
        }
        const int32_t l = next_node.fetch_add(2);
        nd.left = l;
        nd.right = l + 1;
        nd.count = 0;
        push(Job{l + 1, mid, j.first + j.count - mid, j.depth + 1});
        push(Job{l, j.first, mid - j.first, j.depth + 1});
    };

    // Workers share a stack of large jobs; a job below kLocal triangles is finished by the worker
    // that takes it, depth first, without touching the shared stack.
    constexpr int32_t kLocal = 4096;
    std::mutex mu;
    std::condition_variable cv;
    std::vector<Job> shared{{0, 0, (int32_t)nt, 1}};
    int64_t busy = 0;  // jobs taken and not finished (under mu)
    auto worker = [&] {
        std::vector<Bin> binv(3 * bins), right(bins);
        std::vector<Job> local;
        while (true) {
            Job j;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return !shared.empty() || busy == 0; });
                if (shared.empty()) return;  // nothing queued and nobody working: done
                j = shared.back();
                shared.pop_back();
                ++busy;
            }
            local.clear();
            local.push_back(j);
            while (!local.empty()) {
                Job k = local.back();
                local.pop_back();
                split(k, binv, right, [&](const Job& c) {
                    if (c.count < kLocal || nthreads == 1) {
                        local.push_back(c);
                    } else {
                        std::lock_guard<std::mutex> lk(mu);
                        shared.push_back(c);
                        cv.notify_one();
                    }
                });
            }
            std::lock_guard<std::mutex> lk(mu);
            --busy;
            if (busy == 0 && shared.empty()) cv.notify_all();
        }
    };
    {
        std::vector<std::thread> th;
        for (int t = 1; t < nthreads; ++t) th.emplace_back(worker);
        worker();
        for (auto& x : th) x.join();
    }
    nodes.resize((size_t)next_node.load());
    auto t1 = clk::now();

    // ---- threading: one preorder (and miss links) per link set ----
    const int64_t nn = (int64_t)nodes.size();
    std::vector<int32_t> size(nn, 1);
    for (int64_t n = nn - 1; n >= 0; --n)
        if (nodes[n].left >= 0) size[n] = 1 + size[nodes[n].left] + size[nodes[n].right];
    const int sets = p.link_sets;
    // one padding node after each link set: a traversal step may read node + 1 past the last
    // node (a leaf) without using it; the padding box is empty and its links end the walk
    const int64_t stride = nn + 1;
    out.nodes.assign((size_t)sets * stride * 2, float4{0, 0, 0, 0});
    auto thread_set = [&](int c) {  // one link set, on its own worker
        std::vector<int32_t> pos(nn), st;
        st.reserve(256);
        const int axis = c / 2;
        const float sgn = (c % 2 == 0) ? 1.0f : -1.0f;
        int32_t counter = 0;
        st.push_back(0);
        while (!st.empty()) {
            int32_t n = st.back();
            st.pop_back();
            pos[n] = counter++;
            const BNode& nd = nodes[n];
            if (nd.left < 0) continue;
            int32_t first = nd.left, second = nd.right;
            if (sets == 6) {
                // front-to-back along the class direction; ties keep the build order
                const BNode &L = nodes[nd.left], &R = nodes[nd.right];
                float kl = sgn * (L.lo[axis] + L.hi[axis]), kr = sgn * (R.lo[axis] + R.hi[axis]);
                if (kr < kl) std::swap(first, second);
            }
            st.push_back(second);
            st.push_back(first);
        }
        float4* dst = out.nodes.data() + (size_t)c * stride * 2;
        dst[2 * nn] = float4{INFINITY, INFINITY, INFINITY, as_float(-1)};
        dst[2 * nn + 1] = float4{-INFINITY, -INFINITY, -INFINITY, as_float(0)};
        for (int64_t n = 0; n < nn; ++n) {
            const BNode& nd = nodes[n];
            int32_t q = pos[n];
            int32_t miss = q + size[n] < nn ? q + size[n] : -1;
            int32_t word = nd.left >= 0 ? (int32_t)0x80000000u : ((nd.first << 3) | nd.count);
            dst[2 * q] = float4{nd.lo[0], nd.lo[1], nd.lo[2], as_float(miss)};
            dst[2 * q + 1] = float4{nd.hi[0], nd.hi[1], nd.hi[2], as_float(word)};
        }
    };
    {
        std::vector<std::thread> th;
        for (int c = 1; c < sets; ++c) {
            if (nthreads > 1) th.emplace_back(thread_set, c);
            else thread_set(c);
        }
        thread_set(0);
        for (auto& x : th) x.join();
    }
    auto t2 = clk::now();

    // ---- the same tree as child pairs (stack-based traversal), internal nodes in preorder ----
    {
        std::vector<int32_t> ref(nn, 0), st;
        int32_t ni = 0;
        st.push_back(0);
        while (!st.empty()) {  // preorder numbering of the internal nodes
            int32_t n = st.back();
            st.pop_back();
            if (nodes[n].left < 0) {
                ref[n] = ~((nodes[n].first << 3) | nodes[n].count);
                continue;
            }
            ref[n] = ni++;
            st.push_back(nodes[n].right);
            st.push_back(nodes[n].left);
        }
        out.bin.assign((size_t)ni * 4, float4{0, 0, 0, 0});
        for (int64_t n = 0; n < nn; ++n) {
            const BNode& nd = nodes[n];
            if (nd.left < 0) continue;
            const BNode &L = nodes[nd.left], &R = nodes[nd.right];
            float4* q = out.bin.data() + (size_t)ref[n] * 4;
            q[0] = float4{L.lo[0], L.lo[1], L.lo[2], as_float(ref[nd.left])};
            q[1] = float4{L.hi[0], L.hi[1], L.hi[2], as_float(ref[nd.right])};
            q[2] = float4{R.lo[0], R.lo[1], R.lo[2], 0.0f};
            q[3] = float4{R.hi[0], R.hi[1], R.hi[2], 0.0f};
        }
        out.bin_root = ref[0];
    }

    // ---- triangles in leaf order: exact vertices v0, v1, v2 (edges are formed in the kernel) ----
    out.tris.resize((size_t)nt * 3);
    for (int64_t k = 0; k < nt; ++k) {
        int32_t t = perm[k];
        const float* a = verts + 3 * (int64_t)tris[3 * t];
        const float* b = verts + 3 * (int64_t)tris[3 * t + 1];
        const float* c = verts + 3 * (int64_t)tris[3 * t + 2];
        out.tris[3 * k] = float4{a[0], a[1], a[2], as_float(t)};
        out.tris[3 * k + 1] = float4{b[0], b[1], b[2], 0.0f};
        out.tris[3 * k + 2] = float4{c[0], c[1], c[2], 0.0f};
    }
    out.nnodes = nn;
    out.stride = stride;
    out.nleaves = leaves.load();
    out.depth = max_depth.load();
    out.link_sets = sets;
    out.build_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    out.thread_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
    return "";
}

// ---------------------------------------------------------------------------------------------
// instrumented host walk: the device traversal's control flow in FP32, counting the work
// ---------------------------------------------------------------------------------------------
namespace {

inline int ray_class(float dx, float dy, float dz) {
    float ax = std::fabs(dx), ay = std::fabs(dy), az = std::fabs(dz);
    int a = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    float da = a == 0 ? dx : (a == 1 ? dy : dz);
    return 2 * a + (da >= 0.0f ? 0 : 1);
}

}  // namespace

void bvh_host_walk(const HostBVH& bvh, const float* rays, int64_t n, int32_t* out_tri, float* out_t,
                   int32_t* visits, int32_t* tests) {
    const float kRobust = 1.0f + 2.0f * (3.0f * 5.9604645e-8f) / (1.0f - 3.0f * 5.9604645e-8f);
    for (int64_t i = 0; i < n; ++i) {
        const float* r = rays + 8 * i;
        float o[3] = {r[0], r[1], r[2]}, d[3] = {r[4], r[5], r[6]};
        float tmin = r[3], tbest = r[7];
        int32_t best = -1;
        float inv[3];
        for (int k = 0; k < 3; ++k) {
            float dk = d[k];
            if (std::fabs(dk) < 1e-30f) dk = std::copysign(1e-30f, dk);
            inv[k] = 1.0f / dk;
        }
        int c = bvh.link_sets == 6 ? ray_class(d[0], d[1], d[2]) : 0;
        const float4* nodes = bvh.nodes.data() + (size_t)c * bvh.stride * 2;
        int32_t node = 0, nv = 0, nt = 0;
        int64_t steps = 0, cap = 2 * bvh.nnodes + 8;
        while (node >= 0 && steps++ < cap) {
            ++nv;
            const float4 A = nodes[2 * node], B = nodes[2 * node + 1];
            float lo[3] = {A.x, A.y, A.z}, hi[3] = {B.x, B.y, B.z};
            float tn = tmin, tf = INFINITY;
            for (int k = 0; k < 3; ++k) {
                float t0 = (lo[k] - o[k]) * inv[k], t1 = (hi[k] - o[k]) * inv[k];
                tn = std::max(tn, std::min(t0, t1));
                tf = std::min(tf, std::max(t0, t1));
            }
            tf = std::min(tbest, tf * kRobust);
            int32_t miss = as_int(A.w), word = as_int(B.w);
            if (tn <= tf) {
                if (word >= 0) {
                    int32_t first = word >> 3, cnt = word & 7;
                    for (int32_t k = 0; k < cnt; ++k) {
                        ++nt;
                        const float4 P = bvh.tris[3 * (first + k)], V1 = bvh.tris[3 * (first + k) + 1],
                                     V2 = bvh.tris[3 * (first + k) + 2];
                        const float4 E1{V1.x - P.x, V1.y - P.y, V1.z - P.z, 0.0f};
                        const float4 E2{V2.x - P.x, V2.y - P.y, V2.z - P.z, 0.0f};
                        float px = d[1] * E2.z - d[2] * E2.y, py = d[2] * E2.x - d[0] * E2.z,
                              pz = d[0] * E2.y - d[1] * E2.x;
                        float det = E1.x * px + E1.y * py + E1.z * pz;
                        if (det == 0.0f) continue;
                        float f = 1.0f / det;
                        float sx = o[0] - P.x, sy = o[1] - P.y, sz = o[2] - P.z;
                        float u = f * (sx * px + sy * py + sz * pz);
                        float qx = sy * E1.z - sz * E1.y, qy = sz * E1.x - sx * E1.z, qz = sx * E1.y - sy * E1.x;
                        float v = f * (d[0] * qx + d[1] * qy + d[2] * qz);
                        float t = f * (E2.x * qx + E2.y * qy + E2.z * qz);
                        int32_t id = as_int(P.w);
                        if (u >= 0 && v >= 0 && u + v <= 1 && t > tmin &&
                            (t < tbest || (t == tbest && best >= 0 && id < best))) {
                            tbest = t;
                            best = id;
                        }
                    }
                    node = miss;
                } else {
                    node = node + 1;
                }
            } else {
                node = miss;
            }
        }
        if (out_tri) out_tri[i] = best;
        if (out_t) out_t[i] = best >= 0 ? tbest : INFINITY;
        if (visits) visits[i] = nv;
        if (tests) tests[i] = nt;
    }
}
