// scan_sort.cu -- exclusive scan and stable LSD radix sort (8-bit digits) on the device.
//
// The exact hash-grid deposit needs the photon records of a pass ordered by (hash bucket,
// photon id): records arrive in id order after a deterministic compaction, so a stable sort on
// the bucket alone gives that order.
#include <algorithm>

#include "scan_sort.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;
constexpr int kSortBlocks = 512;
static_assert(kTile == kGspScanTile && kSortBlocks == kGspSortBlocks, "scratch sizes in scan_sort.h follow these");

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread over a 256-thread block; *total gets the block sum.
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t* s_warp, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kThreads / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kThreads / 32) s_warp[lane] = w;
    }
    __syncthreads();
    uint32_t before = warp > 0 ? s_warp[warp - 1] : 0u;
    *total = s_warp[kThreads / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const uint32_t* __restrict__ in, int64_t n,
                                                          uint32_t* __restrict__ bsum) {
    __shared__ uint32_t s_warp[kThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k)
        if (base + k < n) s += in[base + k];
    uint32_t total;
    block_exclusive(s, s_warp, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// One block scans the per-tile sums in chunks of 256, carrying the running total.
__global__ void __launch_bounds__(kThreads) k_scan_blocks(uint32_t* __restrict__ bsum, int64_t nb,
                                                          uint32_t* __restrict__ d_total) {
    __shared__ uint32_t s_warp[kThreads / 32];
    uint32_t carry = 0;
    for (int64_t c = 0; c < nb; c += kThreads) {
        const int64_t i = c + threadIdx.x;
        uint32_t v = i < nb ? bsum[i] : 0u, total;
        uint32_t ex = block_exclusive(v, s_warp, &total);
        if (i < nb) bsum[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0 && d_total) *d_total = carry;
}

__global__ void __launch_bounds__(kThreads) k_scan_down(const uint32_t* in, uint32_t* out, int64_t n,
                                                        const uint32_t* __restrict__ boff) {
    __shared__ uint32_t s_warp[kThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    uint32_t v[kItems], s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t run = boff[blockIdx.x] + block_exclusive(s, s_warp, &total);
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

__global__ void __launch_bounds__(kThreads) k_sort_hist(const uint32_t* __restrict__ keys,
                                                        const uint32_t* __restrict__ d_n, int shift,
                                                        uint32_t* __restrict__ hist) {
    __shared__ uint32_t s_h[256];
    const int64_t n = *d_n;
    const int64_t chunk = (n + kSortBlocks - 1) / kSortBlocks;
    const int64_t begin = blockIdx.x * chunk, end = min(n, begin + chunk);
    s_h[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = begin + threadIdx.x; i < end; i += kThreads) atomicAdd(&s_h[(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(int64_t)threadIdx.x * kSortBlocks + blockIdx.x] = s_h[threadIdx.x];
}

// Stable scatter: each block walks its contiguous range in rounds of 256 elements; ranks inside
// a round come from warp match masks and a per-digit prefix over the 8 warps, so equal digits
// keep their input order.
__global__ void __launch_bounds__(kThreads) k_sort_scatter(const uint32_t* __restrict__ kin,
                                                           const uint32_t* __restrict__ vin,
                                                           uint32_t* __restrict__ kout,
                                                           uint32_t* __restrict__ vout,
                                                           const uint32_t* __restrict__ d_n, int shift,
                                                           const uint32_t* __restrict__ offs) {
    __shared__ uint32_t s_cnt[kThreads / 32][257];
    __shared__ uint32_t s_base[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = *d_n;
    const int64_t chunk = (n + kSortBlocks - 1) / kSortBlocks;
    const int64_t begin = blockIdx.x * chunk, end = min(n, begin + chunk);
    s_base[threadIdx.x] = offs[(int64_t)threadIdx.x * kSortBlocks + blockIdx.x];
    for (int w = 0; w < kThreads / 32; ++w) s_cnt[w][threadIdx.x] = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) s_cnt[w][256] = 0;
    __syncthreads();
    for (int64_t r = begin; r < end; r += kThreads) {
        const int64_t e = r + threadIdx.x;
        const bool valid = e < end;
        uint32_t k = 0, v = 0, d = 256;
        if (valid) {
            k = kin[e];
            v = vin[e];
            d = (k >> shift) & 255u;
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t lt = peers & lanemask_lt();
        const uint32_t rank = __popc(lt);
        if (lt == 0) s_cnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            const int t = threadIdx.x;
            uint32_t acc = 0, base = s_base[t];
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) {
                uint32_t c = s_cnt[w][t];
                s_cnt[w][t] = base + acc;
                acc += c;
            }
            s_base[t] = base + acc;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = s_cnt[warp][d] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        for (int w = 0; w < kThreads / 32; ++w) s_cnt[w][threadIdx.x] = 0;
        if (threadIdx.x == 0)
            for (int w = 0; w < kThreads / 32; ++w) s_cnt[w][256] = 0;
        __syncthreads();
    }
    (void)lane;
}

}  // namespace

int64_t gsp_scan_temp_elems(int64_t n) { return gsp_scan_temp_elems_c(n); }

cudaError_t gsp_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* d_total,
                         uint32_t* temp, cudaStream_t st) {
    if (n <= 0) {
        if (d_total) return cudaMemsetAsync(d_total, 0, sizeof(uint32_t), st);
        return cudaSuccess;
    }
    const int64_t nb = (n + kTile - 1) / kTile;
    k_scan_reduce<<<(unsigned)nb, kThreads, 0, st>>>(in, n, temp);
    k_scan_blocks<<<1, kThreads, 0, st>>>(temp, nb, d_total);
    k_scan_down<<<(unsigned)nb, kThreads, 0, st>>>(in, out, n, temp);
    return cudaGetLastError();
}

int64_t gsp_sort_hist_elems() { return kGspSortHistElems; }

cudaError_t gsp_radix_sort_u32(uint32_t* ka, uint32_t* va, uint32_t* kb, uint32_t* vb,
                               const uint32_t* d_n, int bits, uint32_t* hist, uint32_t* temp,
                               cudaStream_t st, uint32_t** kout, uint32_t** vout) {
    for (int shift = 0; shift < bits; shift += 8) {
        k_sort_hist<<<kSortBlocks, kThreads, 0, st>>>(ka, d_n, shift, hist);
        cudaError_t e = gsp_scan_u32(hist, hist, gsp_sort_hist_elems(), nullptr, temp, st);
        if (e != cudaSuccess) return e;
        k_sort_scatter<<<kSortBlocks, kThreads, 0, st>>>(ka, va, kb, vb, d_n, shift, hist);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    *kout = ka;
    *vout = va;
    return cudaGetLastError();
}
