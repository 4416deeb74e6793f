// scan_sort.h -- device exclusive scan and stable radix sort used by the hash-grid deposit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// Launch constants that fix the scratch sizes below (scan_sort.cu checks that it uses them).
constexpr int64_t kGspScanTile = 256 * 8;  // elements one scan block reduces
constexpr int64_t kGspSortBlocks = 512;    // blocks of each radix-sort pass

// Scratch sizes (in uint32 elements) for gsp_scan_u32 over n elements.
constexpr int64_t gsp_scan_temp_elems_c(int64_t n) { return (n + kGspScanTile - 1) / kGspScanTile + 1; }
int64_t gsp_scan_temp_elems(int64_t n);

// Exclusive scan of in[0..n) into out[0..n); the total goes to *d_total if it is not null.
// `temp` needs gsp_scan_temp_elems(n) elements. n is known on the host.
cudaError_t gsp_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* d_total,
                         uint32_t* temp, cudaStream_t st);

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the key. The element
// count is read on the device from *d_n (at most `cap`). Uses two ping-pong buffer pairs;
// returns through *keys_out/*vals_out the pair that holds the result. `hist` needs
// gsp_sort_hist_elems() elements and `temp` gsp_scan_temp_elems(gsp_sort_hist_elems()).
constexpr int64_t kGspSortHistElems = 256 * kGspSortBlocks;
int64_t gsp_sort_hist_elems();
cudaError_t gsp_radix_sort_u32(uint32_t* keys_a, uint32_t* vals_a, uint32_t* keys_b,
                               uint32_t* vals_b, const uint32_t* d_n, int bits, uint32_t* hist,
                               uint32_t* temp, cudaStream_t st, uint32_t** keys_out,
                               uint32_t** vals_out);

// Scratch (uint32 words) of one exact hash-grid build over n points and T buckets: two key/value
// ping-pong pairs, the sort histogram, the larger of the two scans' partials, and 64 words for
// the device-side count.
constexpr int64_t gsp_grid_scratch_words_c(int64_t n, int64_t T) {
    return 4 * n + kGspSortHistElems +
           (gsp_scan_temp_elems_c(T) > gsp_scan_temp_elems_c(kGspSortHistElems) ? gsp_scan_temp_elems_c(T)
                                                                                 : gsp_scan_temp_elems_c(kGspSortHistElems)) +
           64;
}
