// persist.cuh -- the machinery shared by the persistent traversal kernels (closest hit, eye
// paths, photon paths): warp-level work distribution with per-lane refill, and the stackless
// traversal steps of Fig. 3 with postponed leaf tests.
#pragma once

#include "launch.h"

namespace gspd {

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Work distribution of a persistent kernel over items [0, n). A warp takes CHUNK consecutive
// items at a time and hands them to its lanes as they become free, so a lane whose item has
// finished starts the next one without waiting for the rest of the warp. Each warp's first chunk
// is static (an empty or short launch costs no atomics); later chunks come from a counter that
// the caller has zeroed and that counts past the static chunks. All fields are warp-uniform.
template <int CHUNK = kTraceChunk>
struct WarpQueue {
    int32_t n, static_end, qbase, qend;
    bool done;

    __device__ __forceinline__ void init(int32_t n_) {
        n = n_;
        const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
        static_end = (int32_t)min(warps * CHUNK, (int64_t)n);
        qbase = (int32_t)min(((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * CHUNK, (int64_t)n);
        qend = min(qbase + CHUNK, n);
        done = false;
    }

    // Lanes with `need` set receive the next item (-1 once the queue is exhausted).
    template <typename CounterT>
    __device__ __forceinline__ int32_t take(bool need, CounterT* ctr) {
        int32_t item = -1;
        const uint32_t lt = lanemask_lt();
        need = need && !done;
        uint32_t m = __ballot_sync(0xffffffffu, need);
        while (m) {
            if (qbase >= qend) {
                CounterT b = 0;
                if (static_end < n && (threadIdx.x & 31) == 0) b = atomicAdd(ctr, (CounterT)CHUNK);
                b = __shfl_sync(0xffffffffu, b, 0);
                qbase = (int32_t)min((int64_t)static_end + (int64_t)b, (int64_t)n);
                qend = min(qbase + CHUNK, n);
                if (qbase >= n) {
                    done = true;
                    break;
                }
            }
            const int take = min(__popc(m), qend - qbase);
            const int rank = __popc(m & lt);
            if (need && rank < take) {
                item = qbase + rank;
                need = false;
            }
            qbase += take;
            m = __ballot_sync(0xffffffffu, need);
        }
        return item;
    }
};

// Up to kTraceInner traversal steps of the warp's active lanes. A lane that reaches a leaf keeps
// it pending and goes on along the miss link with its current best t (which can only make it
// visit more nodes, never skip the winner); when it meets a second leaf it waits. The warp tests
// all pending leaves together when kTraceLeafBatch lanes hold one, when a lane waits, or when a
// lane's walk has ended. A walk is over when st.node < 0 and pend < 0. `cap` bounds the box
// tests of one walk (corrupt links end the walk with GSP_ERR_TRAVERSAL_LIMIT). ntri counts the
// triangle tests (callers that do not read it lose the count to dead-code elimination).
__device__ __forceinline__ void trav_steps(const DevScene& S, Trav& st, int32_t& pend, bool active, int32_t cap,
                                           uint32_t& ntri) {
#pragma unroll 1
    for (int it = 0; it < kTraceInner; ++it) {
        bool waiting = false;
        if (active && st.node >= 0) {
            // one fetch brings the node and the next node in preorder (its first child when it
            // is internal, usually in the same cache line); both boxes can be tested
            float4 A, B, C, D;
            ldg64(st.nodes + 2 * st.node, A, B, C, D);
            st.steps += 1;
            int32_t word, miss;
            if (st.steps > cap) {
                report(S.status, -4);
                st.node = -1;
            } else if (!box_hit(st, A, B, word, miss)) {
                st.node = miss;
            } else if (word >= 0) {
                if (pend < 0) {
                    pend = word;
                    st.node = miss;
                } else {
                    waiting = true;
                }
            } else {
                st.steps += 1;
                int32_t w2, m2;
                if (!box_hit(st, C, D, w2, m2)) {
                    st.node = m2;
                } else if (w2 >= 0) {
                    if (pend < 0) {
                        pend = w2;
                        st.node = m2;
                    } else {
                        waiting = true;
                        st.node = st.node + 1;
                    }
                } else {
                    st.node = st.node + 2;
                }
            }
        }
        const uint32_t pm = __ballot_sync(0xffffffffu, pend >= 0);
        const uint32_t urgent = __ballot_sync(0xffffffffu, waiting || (pend >= 0 && st.node < 0));
        if (urgent || __popc(pm) >= kTraceLeafBatch) {
            if (pend >= 0) {
                trav_leaf(S, st, pend >> 3, pend & 7);
                ntri += (uint32_t)(pend & 7);
                pend = -1;
            }
        }
        if (__ballot_sync(0xffffffffu, active && (st.node >= 0 || pend >= 0)) == 0) break;
    }
}

// The tail of a warp's work: once its queue is exhausted and a single lane still has a ray, the
// whole warp walks that ray (coop_walk). A stackless walk only moves forward in preorder (a box
// hit leads to the next node, a miss to a later one), so the 32 lanes fetch and test the 32
// nodes from the current one on, one node each, and the walk then follows the hit and miss
// links through that window in registers, fetching again only when a link leaves it; a leaf's
// triangles are tested one per lane. The nodes visited and the hit found are those of the
// one-lane walk (a box in the window is retested against the best t found since it was
// fetched), but the chain of dependent fetches is several times shorter: the last ray of a
// launch no longer waits for one node fetch per box test.

// Makes every lane's walk state a copy of lane src's.
__device__ __forceinline__ void trav_bcast(Trav& st, int src) {
    const uint32_t F = 0xffffffffu;
    st.o = make_float3(__shfl_sync(F, st.o.x, src), __shfl_sync(F, st.o.y, src), __shfl_sync(F, st.o.z, src));
    st.d = make_float3(__shfl_sync(F, st.d.x, src), __shfl_sync(F, st.d.y, src), __shfl_sync(F, st.d.z, src));
    st.inv = make_float3(__shfl_sync(F, st.inv.x, src), __shfl_sync(F, st.inv.y, src), __shfl_sync(F, st.inv.z, src));
    st.tmin = __shfl_sync(F, st.tmin, src);
    st.tbest = __shfl_sync(F, st.tbest, src);
    st.best = __shfl_sync(F, st.best, src);
    st.slot = __shfl_sync(F, st.slot, src);
    st.node = __shfl_sync(F, st.node, src);
    st.steps = __shfl_sync(F, st.steps, src);
    st.nodes = (const float4*)__shfl_sync(F, (unsigned long long)st.nodes, src);
}

// Leaf test of a warp-uniform walk state, one triangle per lane: the same acceptance as
// trav_leaf (whose sequential updates keep the lexicographic (t, index) minimum, so the winner
// is that minimum over the accepted triangles); -0 and +0 compare equal, as there.
__device__ __forceinline__ void coop_leaf(const float4* __restrict__ tris, Trav& st, int32_t first, int32_t cnt) {
    const uint32_t F = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float t = 0.0f;
    int32_t id = 0;
    bool ok = false;
    if (lane < cnt) {
        const float4 P = __ldg(tris + 3 * (first + lane));
        const float4 V1 = __ldg(tris + 3 * (first + lane) + 1);
        const float4 V2 = __ldg(tris + 3 * (first + lane) + 2);
        id = __float_as_int(P.w);
        ok = tri_hit(st.o, st.d, P, V1, V2, t) && t > st.tmin &&
             (t < st.tbest || (t == st.tbest && st.best >= 0 && id < st.best));
    }
    if (__ballot_sync(F, ok) == 0) return;
    uint32_t key = 0xffffffffu;  // t as an unsigned key in float order
    if (ok) {
        const uint32_t b = __float_as_uint(t + 0.0f);
        key = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    }
    const uint32_t kmin = __reduce_min_sync(F, key);
    const bool tie = ok && key == kmin;
    const uint32_t imin = __reduce_min_sync(F, tie ? (uint32_t)id : 0xffffffffu);
    const int win = __ffs(__ballot_sync(F, tie && (uint32_t)id == imin)) - 1;
    st.tbest = __shfl_sync(F, t, win);
    st.best = (int32_t)imin;
    st.slot = first + win;
}

// Result of coop_walk: the walk's final state (node = -1) and the triangles it tested.
struct CoopWalk {
    Trav st;
    uint32_t ntri;
};

// Walks lane owner's ray to its end with the whole warp (every lane must call it; lanes other
// than owner hold no ray). Every lane receives the owner's final state. Not inlined: the
// callers' traversal loops keep their registers, the call costs only at the end of a launch.
// tris, nnodes and status are the scene's.
static __device__ __noinline__ CoopWalk coop_walk(const float4* __restrict__ tris, int64_t nnodes, int32_t* status,
                                                  Trav st, int32_t pend, int owner, int32_t cap) {
    const uint32_t F = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    trav_bcast(st, owner);
    const int32_t pw = __shfl_sync(F, pend, owner);
    uint32_t ntri = 0;
    if (pw >= 0) {
        coop_leaf(tris, st, pw >> 3, pw & 7);
        ntri += (uint32_t)(pw & 7);
    }
    int32_t cur = st.node;
    while (cur >= 0) {
        const int32_t ws = cur;
        bool hit = false;
        float tn = 0.0f;
        int32_t word = -1, miss = -1;
        if ((int64_t)ws + lane < nnodes) {
            const float4 A = __ldg(st.nodes + 2 * ((int64_t)ws + lane)), B = __ldg(st.nodes + 2 * ((int64_t)ws + lane) + 1);
            miss = __float_as_int(A.w);
            word = __float_as_int(B.w);
            hit = slab(st, f3(A), f3(B), tn);
        }
        const uint32_t hm = __ballot_sync(F, hit);
        do {
            const int k = cur - ws;
            const float tk = __shfl_sync(F, tn, k);
            const int32_t wk = __shfl_sync(F, word, k), mk = __shfl_sync(F, miss, k);
            if (++st.steps > cap) {
                if (lane == owner) report(status, -4);
                cur = -1;
            } else if (((hm >> k) & 1u) && tk <= st.tbest) {
                if (wk >= 0) {
                    coop_leaf(tris, st, wk >> 3, wk & 7);
                    ntri += (uint32_t)(wk & 7);
                    cur = mk;
                } else {
                    cur = cur + 1;
                }
            } else {
                cur = mk;
            }
        } while (cur >= 0 && (uint32_t)(cur - ws) < 32u);
    }
    st.node = -1;
    return CoopWalk{st, ntri};
}

// Stack-based near-first walk of the child-pair layout (the comparison traversal of Fig. 4):
// one 64-byte fetch brings both children's boxes, the nearer hit child is visited next and the
// other pushed with its entry distance, and popped entries farther than the best hit so far are
// skipped. node: internal index >= 0, ~(leaf word) < 0, or kWalkDone when the walk is over.
constexpr int kStackDepth = 64;           // callers require tree depth < kStackDepth
constexpr int32_t kWalkDone = INT32_MIN;  // never a node or leaf reference

struct StackWalk {
    int32_t node, sp;
    int32_t stk_node[kStackDepth];
    float stk_t[kStackDepth];
};

__device__ __forceinline__ void stack_init(const DevScene& S, StackWalk& w) {
    w.node = S.bin_root;
    w.sp = 0;
}

__device__ __forceinline__ int32_t stack_pop(const Trav& st, StackWalk& w) {
    while (w.sp > 0) {
        --w.sp;
        if (w.stk_t[w.sp] <= st.tbest) return w.stk_node[w.sp];  // ties may still hold a smaller index
    }
    return kWalkDone;
}

// Up to kTraceInner steps of the active lanes' stack walks (leaves are tested when reached).
__device__ __forceinline__ void stack_steps(const DevScene& S, Trav& st, StackWalk& w, bool active, int32_t cap) {
#pragma unroll 1
    for (int it = 0; it < kTraceInner; ++it) {
        if (active && w.node != kWalkDone && ++st.steps > cap) {  // corrupt data, or a test's limit
            report(S.status, -4);
            w.node = kWalkDone;
        } else if (active && w.node != kWalkDone) {
            if (w.node >= 0) {
                float4 a0, a1, a2, a3;
                ldg64(S.bin + 4 * (int64_t)w.node, a0, a1, a2, a3);
                float tl, tr;
                const bool hl = box_entry(st, f3(a0), f3(a1), tl);
                const bool hr = box_entry(st, f3(a2), f3(a3), tr);
                const int32_t rl = __float_as_int(a0.w), rr = __float_as_int(a1.w);
                if (hl && hr) {
                    const bool lnear = tl <= tr;
                    if (w.sp < kStackDepth) {
                        w.stk_node[w.sp] = lnear ? rr : rl;
                        w.stk_t[w.sp] = lnear ? tr : tl;
                        ++w.sp;
                        w.node = lnear ? rl : rr;
                    } else {  // deeper than callers allow: end the walk, report
                        report(S.status, -4);
                        w.node = kWalkDone;
                    }
                } else if (hl) {
                    w.node = rl;
                } else if (hr) {
                    w.node = rr;
                } else {
                    w.node = stack_pop(st, w);
                }
            } else {
                trav_leaf(S, st, (~w.node) >> 3, (~w.node) & 7);
                w.node = stack_pop(st, w);
            }
        }
        if (__ballot_sync(0xffffffffu, active && w.node != kWalkDone) == 0) break;
    }
}

// Work counters of an SPPM pass (uint64 each, in this order; the C header names them
// GSP_WORK_*): eye rays, photon rays, node box tests, triangle tests, deposits, hit points
// gathered, photons scanned by the gathers, hit points scanned by the adjoint gather.
enum { kWorkEyeRays, kWorkPhotonRays, kWorkNodes, kWorkTris, kWorkDeposits, kWorkHits, kWorkScanned,
       kWorkHitsScanned, kWorkCounts };

// Adds a per-lane count to work[k]: one atomic per warp. Every lane of the warp must call it.
__device__ __forceinline__ void work_add_warp(unsigned long long* work, int k, uint32_t v) {
    const uint32_t sum = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd(work + k, (unsigned long long)sum);
}

__device__ __forceinline__ int32_t trav_cap(const DevScene& S) {
    if (S.step_limit > 0) return S.step_limit;
    return (int32_t)min(4 * S.nnodes + 16, (int64_t)INT32_MAX);  // box tests incl. retests
}

}  // namespace gspd
