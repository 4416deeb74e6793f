// lbvh.cu -- BVH construction on the device, the paper's future work (Sec. 5: construction on
// the GPU). A linear BVH over Morton-ordered triangle centroids, with the internal nodes of the
// radix tree found independently per node (Karras, "Maximizing Parallelism in the Construction
// of BVHs, Octrees, and k-d Trees", HPG 2012), subtrees of at most max_leaf triangles collapsed
// into leaves, and the hit/miss links of every direction class (Sec. 3.1, Fig. 3) written into
// the same packed layout as the host SAH build, so every traversal kernel uses it unchanged.
//
// Radix-tree numbering: internal nodes 0 .. n-2 (root 0), leaves n-1 .. 2n-2 (leaf n-1+i holds
// the i-th triangle in Morton order). A node covers the sorted triangles [first, last].
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "devcommon.cuh"
#include "gsp_internal.h"
#include "launch.h"
#include "scan_sort.h"

namespace {

constexpr int kThreads = 256;
inline unsigned nblocks(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + kThreads - 1) / kThreads); }

// 30-bit Morton code of a point in the unit cube: 10 bits per axis, x in the highest position
// of each bit triple.
__device__ __forceinline__ uint32_t morton30(float x, float y, float z) {
    const uint32_t qx = (uint32_t)fminf(fmaxf(x * 1024.0f, 0.0f), 1023.0f);
    const uint32_t qy = (uint32_t)fminf(fmaxf(y * 1024.0f, 0.0f), 1023.0f);
    const uint32_t qz = (uint32_t)fminf(fmaxf(z * 1024.0f, 0.0f), 1023.0f);
    uint32_t code = 0;
#pragma unroll
    for (int b = 0; b < 10; ++b)
        code |= (((qx >> b) & 1u) << (3 * b + 2)) | (((qy >> b) & 1u) << (3 * b + 1)) | (((qz >> b) & 1u) << (3 * b));
    return code;
}

__global__ void k_codes(const float* __restrict__ verts, const int32_t* __restrict__ tris, int64_t nt, float3 lo,
                        float3 inv_ext, uint32_t* __restrict__ codes, uint32_t* __restrict__ ids) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    float c[3] = {0.0f, 0.0f, 0.0f};
    for (int k = 0; k < 3; ++k) {
        const float* v = verts + 3 * (int64_t)tris[3 * t + k];
        c[0] += v[0];
        c[1] += v[1];
        c[2] += v[2];
    }
    const float third = 1.0f / 3.0f;
    codes[t] = morton30((c[0] * third - lo.x) * inv_ext.x, (c[1] * third - lo.y) * inv_ext.y,
                        (c[2] * third - lo.z) * inv_ext.z);
    ids[t] = (uint32_t)t;
}

// Length of the common prefix of sorted keys i and j, each extended by its index so that equal
// codes still differ; -1 when j is outside [0, n).
__device__ __forceinline__ int prefix(const uint32_t* __restrict__ k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const uint32_t a = k[i], b = k[j];
    if (a == b) return 32 + __clz((uint32_t)i ^ (uint32_t)j);
    return __clz(a ^ b);
}

// Internal node i: the direction of its range from the neighbour prefixes, the range end by an
// exponential then binary search, the split where the prefix first grows, and the children.
__global__ void k_internal(const uint32_t* __restrict__ k, int n, int32_t* __restrict__ left,
                           int32_t* __restrict__ right, int32_t* __restrict__ parent, int32_t* __restrict__ first,
                           int32_t* __restrict__ last) {
    const int i = (int)((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n - 1) return;
    const int d = prefix(k, n, i, i + 1) - prefix(k, n, i, i - 1) >= 0 ? 1 : -1;
    const int pmin = prefix(k, n, i, i - d);
    int lmax = 2;
    while (prefix(k, n, i, i + lmax * d) > pmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (prefix(k, n, i, i + (l + t) * d) > pmin) l += t;
    const int j = i + l * d;
    const int pnode = prefix(k, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (prefix(k, n, i, i + (s + t) * d) > pnode) s += t;
    } while (t > 1);
    const int g = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    const int L = lo == g ? n - 1 + g : g;
    const int R = hi == g + 1 ? n - 1 + g + 1 : g + 1;
    left[i] = L;
    right[i] = R;
    parent[L] = i;
    parent[R] = i;
    first[i] = lo;
    last[i] = hi;
}

struct Box {
    float lo[3], hi[3];
};

// Boxes and final-tree sizes, bottom up: each leaf walks towards the root; at every internal
// node the first of the two children to arrive stops and the second (which then sees both
// children finished) computes the node. A node covering at most max_leaf triangles becomes a
// leaf of the final tree (size 1).
__global__ void k_bottom_up(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                            const uint32_t* __restrict__ ids, int n, const int32_t* __restrict__ left,
                            const int32_t* __restrict__ right, const int32_t* __restrict__ parent,
                            const int32_t* __restrict__ first, const int32_t* __restrict__ last, int max_leaf,
                            Box* __restrict__ box, int32_t* __restrict__ size, uint32_t* __restrict__ arrived) {
    const int i = (int)((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n) return;
    const int leaf = n - 1 + i;
    const int64_t t = ids[i];
    Box b;
    for (int a = 0; a < 3; ++a) {
        b.lo[a] = INFINITY;
        b.hi[a] = -INFINITY;
    }
    for (int k = 0; k < 3; ++k) {
        const float* v = verts + 3 * (int64_t)tris[3 * t + k];
        for (int a = 0; a < 3; ++a) {
            b.lo[a] = fminf(b.lo[a], v[a]);
            b.hi[a] = fmaxf(b.hi[a], v[a]);
        }
    }
    box[leaf] = b;
    size[leaf] = 1;
    int cur = parent[leaf];
    while (cur >= 0) {
        __threadfence();  // this child's box and size are visible before the arrival count
        if (atomicAdd(arrived + cur, 1u) == 0) return;
        __threadfence();
        const int L = left[cur], R = right[cur];
        const volatile float* bl = (const volatile float*)(box + L);
        const volatile float* br = (const volatile float*)(box + R);
        Box u;
        for (int a = 0; a < 3; ++a) {
            u.lo[a] = fminf(bl[a], br[a]);
            u.hi[a] = fmaxf(bl[3 + a], br[3 + a]);
        }
        box[cur] = u;
        const int sl = ((const volatile int32_t*)size)[L], sr = ((const volatile int32_t*)size)[R];
        size[cur] = last[cur] - first[cur] + 1 <= max_leaf ? 1 : 1 + sl + sr;
        cur = parent[cur];
    }
}

__device__ __forceinline__ bool final_leaf(int m, int n, const int32_t* first, const int32_t* last, int max_leaf) {
    return m >= n - 1 || last[m] - first[m] + 1 <= max_leaf;
}

// Whether node m is part of the final tree: the root, or a child of a node that was not
// collapsed (ranges are nested, so one check of the parent suffices).
__device__ __forceinline__ bool in_tree(int m, const int32_t* parent, const int32_t* first, const int32_t* last,
                                        int max_leaf) {
    const int p = parent[m];
    return p < 0 || last[p] - first[p] + 1 > max_leaf;
}

// Threading: for every node of the final tree and every link set, its preorder position (the
// sum over the path from the root of 1 + the size of the first-visited sibling when the path
// enters the second child), then its packed record {min, miss | max, leaf word} at that position.
__global__ void k_thread(int n, int sets, const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                         const int32_t* __restrict__ parent, const int32_t* __restrict__ first,
                         const int32_t* __restrict__ last, int max_leaf, const Box* __restrict__ box,
                         const int32_t* __restrict__ size, int32_t nfinal, int64_t stride, float4* __restrict__ nodes,
                         int32_t* __restrict__ depth) {
    const int m = (int)((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (m >= 2 * n - 1 || !in_tree(m, parent, first, last, max_leaf)) return;
    const bool leaf = final_leaf(m, n, first, last, max_leaf);
    int32_t word = (int32_t)0x80000000u;
    if (leaf) word = m >= n - 1 ? ((m - (n - 1)) << 3) | 1 : (first[m] << 3) | (last[m] - first[m] + 1);
    const Box b = box[m];
    int steps = 0;
    for (int c = 0; c < sets; ++c) {
        const int axis = c / 2;
        const float sgn = (c % 2 == 0) ? 1.0f : -1.0f;
        int32_t pos = 0;
        for (int cur = m; parent[cur] >= 0; cur = parent[cur]) {
            const int p = parent[cur];
            int fst = left[p], snd = right[p];
            if (sets == 6) {  // front-to-back along the class direction; ties keep the build order
                const float kl = sgn * (box[fst].lo[axis] + box[fst].hi[axis]);
                const float kr = sgn * (box[snd].lo[axis] + box[snd].hi[axis]);
                if (kr < kl) {
                    const int tmp = fst;
                    fst = snd;
                    snd = tmp;
                }
            }
            pos += 1 + (cur == fst ? 0 : size[fst]);
            if (c == 0) ++steps;
        }
        const int32_t miss = pos + size[m] < nfinal ? pos + size[m] : -1;
        float4* dst = nodes + (size_t)c * stride * 2 + 2 * (size_t)pos;
        dst[0] = make_float4(b.lo[0], b.lo[1], b.lo[2], __int_as_float(miss));
        dst[1] = make_float4(b.hi[0], b.hi[1], b.hi[2], __int_as_float(word));
    }
    atomicMax(depth, steps);
}

// The padding node after each link set (read as node + 1 of the last node, never used).
__global__ void k_padding(int sets, int32_t nfinal, int64_t stride, float4* __restrict__ nodes) {
    const int c = threadIdx.x;
    if (c >= sets) return;
    float4* dst = nodes + (size_t)c * stride * 2 + 2 * (size_t)nfinal;
    dst[0] = make_float4(INFINITY, INFINITY, INFINITY, __int_as_float(-1));
    dst[1] = make_float4(-INFINITY, -INFINITY, -INFINITY, __int_as_float(0));
}

// Triangles in leaf (Morton) order: {v0, index}, {v1, 0}, {v2, 0}.
__global__ void k_leaf_tris(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                            const uint32_t* __restrict__ ids, int64_t nt, float4* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const int64_t t = ids[i];
    for (int k = 0; k < 3; ++k) {
        const float* v = verts + 3 * (int64_t)tris[3 * t + k];
        out[3 * i + k] = make_float4(v[0], v[1], v[2], k == 0 ? __int_as_float((int32_t)t) : 0.0f);
    }
}

// Child-pair layout for the stack traversal, indexed by radix-tree internal node: children as
// internal indices, or ~(leaf word) for final leaves. Collapsed nodes' entries stay unused.
__global__ void k_child_pairs(int n, const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                              const int32_t* __restrict__ parent, const int32_t* __restrict__ first,
                              const int32_t* __restrict__ last, int max_leaf, const Box* __restrict__ box,
                              float4* __restrict__ bin) {
    const int i = (int)((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n - 1 || !in_tree(i, parent, first, last, max_leaf) || final_leaf(i, n, first, last, max_leaf)) return;
    auto ref = [&](int c) -> int32_t {
        if (!final_leaf(c, n, first, last, max_leaf)) return c;
        const int32_t w = c >= n - 1 ? ((c - (n - 1)) << 3) | 1 : (first[c] << 3) | (last[c] - first[c] + 1);
        return ~w;
    };
    const int L = left[i], R = right[i];
    const Box bl = box[L], br = box[R];
    float4* q = bin + 4 * (size_t)i;
    q[0] = make_float4(bl.lo[0], bl.lo[1], bl.lo[2], __int_as_float(ref(L)));
    q[1] = make_float4(bl.hi[0], bl.hi[1], bl.hi[2], __int_as_float(ref(R)));
    q[2] = make_float4(br.lo[0], br.lo[1], br.lo[2], 0.0f);
    q[3] = make_float4(br.hi[0], br.hi[1], br.hi[2], 0.0f);
}

}  // namespace

extern "C" gsp_status gsp_build_bvh_device(gsp_scene* s, int32_t link_sets, int32_t max_leaf, gsp_bvh_stats* stats) {
    if (!s || !s->ctx || (link_sets != 1 && link_sets != 6) || max_leaf < 1 || max_leaf > 7)
        return GSP_ERR_INVALID_ARG;
    const int64_t nt = s->nt;
    if (nt < 1 || nt > (int64_t(1) << 28)) return GSP_ERR_INVALID_ARG;
    GSP_CUDA_TRY(cudaSetDevice(s->ctx->device));
    GSP_NO_PENDING_ERROR("gsp_build_bvh_device");
    NvtxRange nvtx("gsp: device LBVH build + threading");
    const int n = (int)nt;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t v = 0; v < s->nv; ++v)  // bounds of all vertices (Morton quantisation range)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], s->verts[3 * v + a]);
            hi[a] = std::max(hi[a], s->verts[3 * v + a]);
        }
    float inv[3];
    for (int a = 0; a < 3; ++a) inv[a] = hi[a] > lo[a] ? 1.0f / (hi[a] - lo[a]) : 0.0f;

    // device scratch, freed before returning
    std::vector<void*> tmp;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, int64_t count) {
        *p = nullptr;
        if (e == cudaSuccess && count > 0) e = cudaMalloc((void**)p, (size_t)count * sizeof(**p));
        if (e == cudaSuccess && *p) tmp.push_back((void*)*p);
    };
    float* d_verts;
    int32_t *d_tris, *left, *right, *parent, *first, *last, *size, *d_depth;
    uint32_t *ka, *va, *kb, *vb, *hist, *stemp, *d_n, *arrived;
    Box* box;
    const int64_t nn = 2 * (int64_t)n - 1;
    A(&d_verts, 3 * s->nv);
    A(&d_tris, 3 * nt);
    A(&ka, nt);
    A(&va, nt);
    A(&kb, nt);
    A(&vb, nt);
    A(&hist, gsp_sort_hist_elems());
    A(&stemp, gsp_scan_temp_elems(gsp_sort_hist_elems()));
    A(&d_n, 1);
    A(&left, std::max<int64_t>(1, n - 1));
    A(&right, std::max<int64_t>(1, n - 1));
    A(&first, std::max<int64_t>(1, n - 1));
    A(&last, std::max<int64_t>(1, n - 1));
    A(&parent, nn);
    A(&size, nn);
    A(&box, nn);
    A(&arrived, std::max<int64_t>(1, n - 1));
    A(&d_depth, 1);
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // build and threading times
    auto drop_events = [&]() {
        for (cudaEvent_t& x : ev)
            if (x) {
                cudaEventDestroy(x);
                x = nullptr;
            }
    };
    auto fail = [&](cudaError_t ce) {
        drop_events();
        for (void* p : tmp) cudaFree(p);
        const gsp_status st = gsp_cuda_fail(ce);
        gsp_set_last_error(std::string("gsp_build_bvh_device: ") + cudaGetErrorString(ce));
        return st;
    };
    if (e != cudaSuccess) return fail(e);

    for (cudaEvent_t& x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    if (e != cudaSuccess) return fail(e);
    const uint32_t nn32 = (uint32_t)nt;
    e = cudaMemcpy(d_verts, s->verts.data(), 3 * s->nv * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_tris, s->tris.data(), 3 * nt * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_n, &nn32, sizeof nn32, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(parent, 0xff, nn * sizeof(int32_t));  // -1: the root has no parent
    if (e == cudaSuccess) e = cudaMemset(arrived, 0, std::max<int64_t>(1, n - 1) * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(d_depth, 0, sizeof(int32_t));
    if (e != cudaSuccess) return fail(e);
    cudaEventRecord(ev[0]);
    k_codes<<<nblocks(nt), kThreads>>>(d_verts, d_tris, nt, make_float3(lo[0], lo[1], lo[2]),
                                       make_float3(inv[0], inv[1], inv[2]), ka, va);
    uint32_t *keys = nullptr, *ids = nullptr;
    e = gsp_radix_sort_u32(ka, va, kb, vb, d_n, 30, hist, stemp, nullptr, &keys, &ids);
    if (e != cudaSuccess) return fail(e);
    if (n > 1) k_internal<<<nblocks(n - 1), kThreads>>>(keys, n, left, right, parent, first, last);
    k_bottom_up<<<nblocks(n), kThreads>>>(d_verts, d_tris, ids, n, left, right, parent, first, last, max_leaf, box,
                                          size, arrived);
    int32_t nfinal = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(&nfinal, size, sizeof nfinal, cudaMemcpyDeviceToHost);  // root: node 0
    if (e != cudaSuccess) return fail(e);
    cudaEventRecord(ev[1]);
    // final tree: nfinal nodes per link set (+ one padding node); triangles in Morton order
    const int64_t stride = (int64_t)nfinal + 1;
    float4 *d_nodes = nullptr, *d_tri4 = nullptr, *d_bin = nullptr;
    const int64_t nb = std::max<int64_t>(1, n - 1) * 4;
    e = cudaMalloc(&d_nodes, (size_t)link_sets * stride * 2 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&d_tri4, (size_t)nt * 3 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&d_bin, (size_t)nb * sizeof(float4));
    if (e != cudaSuccess) {
        cudaFree(d_nodes);
        cudaFree(d_tri4);
        cudaFree(d_bin);
        return fail(e);
    }
    // (n == 1: the single leaf is node 0 of the radix numbering, n - 1 + 0 = 0)
    k_thread<<<nblocks(nn), kThreads>>>(n, link_sets, left, right, parent, first, last, max_leaf, box, size, nfinal,
                                        stride, d_nodes, d_depth);
    k_padding<<<1, 32>>>(link_sets, nfinal, stride, d_nodes);
    k_leaf_tris<<<nblocks(nt), kThreads>>>(d_verts, d_tris, ids, nt, d_tri4);
    k_child_pairs<<<nblocks(n), kThreads>>>(n, left, right, parent, first, last, max_leaf, box, d_bin);
    cudaEventRecord(ev[2]);
    e = cudaEventSynchronize(ev[2]);
    if (e == cudaSuccess) e = cudaGetLastError();
    float build_ms = 0, thread_ms = 0;
    cudaEventElapsedTime(&build_ms, ev[0], ev[1]);
    cudaEventElapsedTime(&thread_ms, ev[1], ev[2]);
    drop_events();
    int32_t depth = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&depth, d_depth, sizeof depth, cudaMemcpyDeviceToHost);
    // host copies (host walk, export), as the host build keeps them
    HostBVH bvh;
    if (e == cudaSuccess) {
        bvh.nodes.resize((size_t)link_sets * stride * 2);
        bvh.tris.resize((size_t)nt * 3);
        bvh.bin.resize((size_t)nb);
        e = cudaMemcpy(bvh.nodes.data(), d_nodes, bvh.nodes.size() * sizeof(float4), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(bvh.tris.data(), d_tri4, bvh.tris.size() * sizeof(float4), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(bvh.bin.data(), d_bin, bvh.bin.size() * sizeof(float4), cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) {
        cudaFree(d_nodes);
        cudaFree(d_tri4);
        cudaFree(d_bin);
        return fail(e);
    }
    for (void* p : tmp) cudaFree(p);
    int64_t leaves = 0;
    for (int64_t q = 0; q < nfinal; ++q) {
        int32_t w;
        std::memcpy(&w, &bvh.nodes[2 * q + 1].w, 4);
        leaves += w >= 0;
    }
    // the root's reference in the child-pair layout: internal node 0, or the root leaf
    {
        int32_t w;
        std::memcpy(&w, &bvh.nodes[1].w, 4);
        bvh.bin_root = w >= 0 ? ~w : 0;
    }
    bvh.nnodes = nfinal;
    bvh.stride = stride;
    bvh.nleaves = leaves;
    bvh.depth = depth;
    bvh.link_sets = link_sets;
    bvh.build_ms = build_ms;
    bvh.thread_ms = thread_ms;
    gsp_scene_adopt_bvh(s, std::move(bvh), d_nodes, d_tri4, d_bin);
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
