// sppm_gather.cuh -- device side of an SPPM pass from its deposits on: the exact hash-grid
// deposit (compaction, bucket keys), the fused range query + progressive update in both hashing
// modes (Sec. 2, Sec. 3.4), the adjoint kernels of the gradient replay, and small utility
// kernels. Included by sppm.cu only.
#pragma once

#include "sppm_paths.cuh"

namespace gspd {

// ------------------------------------------------------------------------------------------
// exact hash-grid deposit: compaction in id order, bucket keys, bucket counts
// ------------------------------------------------------------------------------------------
// keys == nullptr: the compaction alone (slot of each deposit in path order, no buckets).
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
        vals[off + i] = slot;
        if (!keys) continue;
        const float4 a = slots[2 * (size_t)slot];
        const uint32_t b = bucket_of(f3(a), inv_h, tmask);
        keys[off + i] = b;
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
    uint32_t* __restrict__ heavy;   // optional: hit points whose query goes to k_gather_heavy
    uint32_t* __restrict__ nheavy;  // their count (zeroed before k_gather_exact)
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
    uint32_t scanned = 0;
    for (int q = 0; q < nb; ++q) {
        const uint32_t b = buckets[q];
        const uint32_t cnt = G.ecount[b];
        if (cnt == 0) continue;
        ++scanned;
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
    if (P.work) {
        atomicAdd(P.work + kWorkHits, 1ull);
        atomicAdd(P.work + kWorkScanned, (unsigned long long)scanned);
    }
}

#ifndef GSP_GATHER_BATCH
#define GSP_GATHER_BATCH 4
#endif
constexpr int kGatherBatch = GSP_GATHER_BATCH;  // candidate positions a gather lane has in flight

// The cells of an exact range query: those overlapping the box x +- R.
struct QueryCells {
    int32_t lx, hx, ly, hy, lz, hz;
};

__device__ __forceinline__ QueryCells query_cells(float3 x, float R, float inv_h) {
    QueryCells q;
    cell_range(x.x, R, inv_h, q.lx, q.hx);
    cell_range(x.y, R, inv_h, q.ly, q.hy);
    cell_range(x.z, R, inv_h, q.lz, q.hz);
    return q;
}

// Photons in the buckets of the query's cells: the length of the range query.
__device__ __forceinline__ uint32_t query_cost(const GatherDev& G, const PassDev& P, const QueryCells& q) {
    uint32_t cost = 0;
    for (int32_t ix = q.lx; ix <= q.hx; ++ix)
        for (int32_t iy = q.ly; iy <= q.hy; ++iy)
            for (int32_t iz = q.lz; iz <= q.hz; ++iz) {
                const uint32_t b = cell_hash(ix, iy, iz, P.tmask);
                cost += __ldg(G.bstart + b + 1) - __ldg(G.bstart + b);
            }
    return cost;
}

// One lane's share of an exact range query split over S lanes: lane gl takes every S-th photon of
// each visited cell's bucket. A photon that passes the distance test counts only while its own
// cell is the one being visited, so a photon whose bucket several visited cells share (hash
// collisions) counts once. kGatherBatch of the lane's candidates are fetched before any is
// tested, so that a dense bucket costs kGatherBatch times fewer round trips to L2; they are then
// tested in the lane's order, as one at a time would.
__device__ __forceinline__ void gather_lane(const GatherDev& G, const PassDev& P, const QueryCells& q, float3 x,
                                            float3 n, float R, int gl, int S, float& M, float3& acc,
                                            uint32_t& scanned) {
    const float R2p = R * R * 1.0001f;  // cheap pre-test, then the exact one
    for (int32_t ix = q.lx; ix <= q.hx; ++ix)
        for (int32_t iy = q.ly; iy <= q.hy; ++iy)
            for (int32_t iz = q.lz; iz <= q.hz; ++iz) {
                const uint32_t b = cell_hash(ix, iy, iz, P.tmask);
                const uint32_t e = __ldg(G.bstart + b + 1);
                for (uint32_t i = __ldg(G.bstart + b) + gl; i < e; i += kGatherBatch * S) {
                    float4 a[kGatherBatch];
#pragma unroll
                    for (int u = 0; u < kGatherBatch; ++u)
                        if (i + u * S < e) a[u] = __ldg(G.spos + i + u * S);
#pragma unroll
                    for (int u = 0; u < kGatherBatch; ++u) {
                        if (i + u * S >= e) break;
                        ++scanned;
                        const float3 dx = f3(a[u]) - x;
                        if (!(dot3(dx, dx) < R2p)) continue;
                        if (cell_of(a[u].x, P.inv_h) != ix || cell_of(a[u].y, P.inv_h) != iy ||
                            cell_of(a[u].z, P.inv_h) != iz)
                            continue;  // a colliding cell's photon, counted when its own cell is visited
                        const float4 c = __ldg(G.spay + i + u * S);
                        if (!photon_accept(f3(a[u]), x, R, __float_as_uint(c.w), n)) continue;
                        M += 1.0f;
                        acc = acc + f3(c);
                    }
                }
            }
}

// The end of hit point p's gather: the pass's direct term, the gradient records, the progressive
// update with the gathered count M and flux sum acc.
__device__ __forceinline__ void gather_finish(const GatherDev& G, const PassDev& P, int64_t p, float R, float M,
                                              float3 acc, uint32_t scanned) {
    if (P.work) {
        atomicAdd(P.work + kWorkHits, 1ull);
        atomicAdd(P.work + kWorkScanned, (unsigned long long)scanned);
    }
    if (G.rhist) G.rhist[(size_t)pass_index(P) * G.npix + p] = R;
    if (G.shist) G.shist[(size_t)pass_index(P) * G.npix + p] = make_float4(acc.x, acc.y, acc.z, 0.0f);
    float4 s0 = G.st0[p], s1 = G.st1[p];
    add_direct(s1, G.hd[p]);
    progressive_update(s0, s1, M, mul3(f3(G.hf[p]), acc), P.alpha);
    G.st0[p] = s0;
    G.st1[p] = s1;
}

// A query longer than this many photons per lane of its group (of at least 8 lanes: with fewer,
// so many queries would qualify that the second launch would do most of the work) goes to
// k_gather_heavy.
#ifndef GSP_HEAVY_PER_LANE
#define GSP_HEAVY_PER_LANE 128
#endif
constexpr uint32_t kHeavyPerLane = GSP_HEAVY_PER_LANE;
// Images below this many pixels gather without the split: at 256^2 it only breaks even (the
// gather 67-71 us against 57 + 11 us), and in a batch of many smaller images its extra launches
// cost more than they save.
constexpr int64_t kHeavyMinPixels = 512 * 512;
// Images below this many pixels gather with 16 lanes per hit point by default, larger ones with 8.
constexpr int64_t kGatherWideBelow = 256 * 256;

// Exact range query + progressive update, a group of L lanes per hit point. The group visits
// every cell overlapping the box x +- R (any number per axis, so the cell may be smaller than the
// radius) and its lanes split each bucket's photons (gather_lane; consecutive, coalesced). Lane
// sums are combined by a fixed butterfly, so the result does not depend on scheduling. With a
// heavy list (G.heavy), a hit point whose query is longer than kHeavyPerLane photons per lane (the
// dense spots of a caustic, up to twenty times the median) is listed for k_gather_heavy instead:
// left to one group it would keep its SM busy long after the others are done.
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
    const float R = G.st1[p].w;
    const QueryCells q = query_cells(x, R, P.inv_h);
    if (G.heavy && query_cost(G, P, q) > kHeavyPerLane * (L < 8 ? 8 : L)) {  // the whole group leaves together
        if (gl == 0) G.heavy[atomicAdd(G.nheavy, 1u)] = (uint32_t)p;
        return;
    }
    float M = 0.0f;
    float3 acc = make_float3(0.0f, 0.0f, 0.0f);
    uint32_t scanned = 0;  // this lane's photons read (work counter)
    gather_lane(G, P, q, x, f3(G.hn[p]), R, gl, L, M, acc, scanned);
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
        if (P.work) {
#pragma unroll
            for (int off = L / 2; off > 0; off >>= 1) scanned += __shfl_xor_sync(gmask, scanned, off, L);
        }
    }
    if (gl == 0) gather_finish(G, P, p, R, M, acc, scanned);
}

// The listed heavy queries, a block of kHeavyThreads per hit point (persistent over the list):
// the same lane split as k_gather_exact with kHeavyThreads lanes, lane sums combined by a fixed
// butterfly in each warp and then warp by warp in order, so the result does not depend on
// scheduling either.
constexpr int kHeavyThreads = 256;

__global__ void __launch_bounds__(kHeavyThreads) k_gather_heavy(GatherDev G, PassDev P) {
    __shared__ float s_sum[kHeavyThreads / 32][4];
    __shared__ uint32_t s_scan[kHeavyThreads / 32];
    const uint32_t count = *G.nheavy;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t j = blockIdx.x; j < count; j += gridDim.x) {
        const int64_t p = G.heavy[j];
        const float3 x = f3(G.hx[p]);
        const float R = G.st1[p].w;
        const QueryCells q = query_cells(x, R, P.inv_h);
        float M = 0.0f;
        float3 acc = make_float3(0.0f, 0.0f, 0.0f);
        uint32_t scanned = 0;
        gather_lane(G, P, q, x, f3(G.hn[p]), R, threadIdx.x, kHeavyThreads, M, acc, scanned);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            M += __shfl_xor_sync(0xffffffffu, M, off);
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
            acc.z += __shfl_xor_sync(0xffffffffu, acc.z, off);
            scanned += __shfl_xor_sync(0xffffffffu, scanned, off);
        }
        if (lane == 0) {
            s_sum[warp][0] = M;
            s_sum[warp][1] = acc.x;
            s_sum[warp][2] = acc.y;
            s_sum[warp][3] = acc.z;
            s_scan[warp] = scanned;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            M = 0.0f;
            acc = make_float3(0.0f, 0.0f, 0.0f);
            scanned = 0;
            for (int w = 0; w < kHeavyThreads / 32; ++w) {
                M += s_sum[w][0];
                acc.x += s_sum[w][1];
                acc.y += s_sum[w][2];
                acc.z += s_sum[w][3];
                scanned += s_scan[w];
            }
            gather_finish(G, P, p, R, M, acc, scanned);
        }
        __syncthreads();
    }
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
    const float4* __restrict__ hp_rec;  // per sorted position (k_adj_hp_records): {x, bits}, {n, R}, {B term, 0}
    uint32_t hp_mask;
    float inv_hp;                       // 1 / hit-point cell size
    float rmax;                         // largest gather radius (r0)
    const float4* __restrict__ spos;    // deposits of the pass, bucket-sorted
    const float4* __restrict__ spay;
    const uint32_t* __restrict__ order; // sorted deposit -> photon slot
    const uint32_t* __restrict__ d_total;
    float4* __restrict__ badj;          // per slot: B_k, the weight of Phi_k in the loss
    unsigned long long* work;           // work counters, or null
};

// The hit points in the order of the hit-point grid, three float4 each: {x, material bits},
// {normal, R}, {g * f / R^2, 0} (g = dLoss/dL of the pixel, f = its w rho / pi, R its radius in
// this pass), so that the photon-centric gather reads a bucket's hit points one after another
// instead of through the order array, with the loss term already formed (the same operations as
// forming it per photon).
__global__ void __launch_bounds__(256) k_adj_hp_records(AdjDev A, int64_t npix, float4* __restrict__ rec) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= npix) return;
    const uint32_t p = A.hp_order[j];
    const float R = A.rhist[p];
    const float3 gp = make_float3(A.g[3 * p], A.g[3 * p + 1], A.g[3 * p + 2]);
    const float3 w = mul3(gp, f3(A.hf[p])) * (1.0f / (R * R));
    const float4 n = A.hn[p];
    rec[3 * j] = A.hx[p];
    rec[3 * j + 1] = make_float4(n.x, n.y, n.z, R);
    rec[3 * j + 2] = make_float4(w.x, w.y, w.z, 0.0f);
}

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
        uint32_t scanned = 0;
        for (int32_t ix = lx; ix <= hx; ++ix)
            for (int32_t iy = ly; iy <= hy; ++iy)
                for (int32_t iz = lz; iz <= hz; ++iz) {
                    const uint32_t b = cell_hash(ix, iy, iz, A.hp_mask);
                    const uint32_t e = __ldg(A.hp_bstart + b + 1);
                    for (uint32_t j = __ldg(A.hp_bstart + b) + gl; j < e; j += L) {
                        ++scanned;
                        const float4 hxp = __ldg(A.hp_rec + 3 * (size_t)j);
                        if (__float_as_int(hxp.w) < 0) continue;
                        if (cell_of(hxp.x, A.inv_hp) != ix || cell_of(hxp.y, A.inv_hp) != iy ||
                            cell_of(hxp.z, A.inv_hp) != iz)
                            continue;
                        const float4 nr = __ldg(A.hp_rec + 3 * (size_t)j + 1);
                        if (!photon_accept(xk, f3(hxp), nr.w, dir, f3(nr))) continue;
                        B = B + f3(__ldg(A.hp_rec + 3 * (size_t)j + 2));
                    }
                }
#pragma unroll
        for (int off = L / 2; off > 0; off >>= 1) {
            B.x += __shfl_xor_sync(gmask, B.x, off, L);
            B.y += __shfl_xor_sync(gmask, B.y, off, L);
            B.z += __shfl_xor_sync(gmask, B.z, off, L);
        }
        if (gl == 0) A.badj[A.order[i]] = make_float4(B.x, B.y, B.z, 0.0f);
        if (A.work) atomicAdd(A.work + kWorkHitsScanned, (unsigned long long)scanned);
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

// Counts in *bad the pixels of a progressive state outside the values a render can reach: N
// finite and >= 0, R finite in (0, r0], tau and the direct sums finite and >= 0.
__global__ void k_check_state(int64_t npix, const float* __restrict__ N, const float* __restrict__ R,
                              const float* __restrict__ tau, const float* __restrict__ direct, float r0,
                              uint32_t* __restrict__ bad) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    bool ok = isfinite(N[p]) && N[p] >= 0.0f && isfinite(R[p]) && R[p] > 0.0f && R[p] <= r0;
    for (int c = 0; c < 3; ++c)
        ok = ok && isfinite(tau[3 * p + c]) && tau[3 * p + c] >= 0.0f && isfinite(direct[3 * p + c]) &&
             direct[3 * p + c] >= 0.0f;
    if (!ok) atomicAdd(bad, 1u);
}

__global__ void k_set_state(float4* __restrict__ st0, float4* __restrict__ st1, int64_t npix,
                            const float* __restrict__ N, const float* __restrict__ R, const float* __restrict__ tau,
                            const float* __restrict__ direct) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    st0[p] = make_float4(tau[3 * p], tau[3 * p + 1], tau[3 * p + 2], N[p]);
    st1[p] = make_float4(direct[3 * p], direct[3 * p + 1], direct[3 * p + 2], R[p]);
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

__global__ void k_work_add(unsigned long long* p, const uint32_t* v) { *p += *v; }

__global__ void k_fill_u64(unsigned long long* p, int64_t n, unsigned long long v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

}  // namespace gspd
