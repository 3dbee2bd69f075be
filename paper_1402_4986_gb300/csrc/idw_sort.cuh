// Stable least-significant-digit radix sort of (uint32 key, uint32 value)
// pairs on the device, and a device-wide exclusive scan of int32 counts.
// The deterministic gradient of the k-NN form uses it to turn the query-major
// list of (data point, query) selections into a point-major one whose
// queries stay in increasing order within each point (stability), so every
// point's terms are summed in one fixed order.
//
// One pass sorts on 8 bits:
//   1. count: each CTA counts the digits of its tile of kSortTile items
//      (shared-memory atomics: counts do not depend on order);
//   2. scan: the counts, laid out digit-major (digit d of tile b at
//      d * tiles + b), are scanned into each (digit, tile)'s first output
//      position;
//   3. scatter: each CTA walks its tile in rounds of 256 consecutive items
//      and ranks each item among the equal digits before it: lanes of a warp
//      by a match mask, warps of a round by per-warp digit counts, rounds by
//      a running count per digit.  Equal keys keep their input order.
#pragma once

#include <cstdint>
#include <utility>

#include <cuda_runtime.h>

namespace idw {
namespace sort_detail {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;  // 4096 items per CTA
constexpr int kRadix = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kSortThreads)
    radix_count_kernel(const uint32_t* __restrict__ keys, int64_t count, int shift,
                       int32_t* __restrict__ counts, int64_t tiles) {
  __shared__ int32_t h[kRadix];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t x = base + int64_t(r) * kSortThreads + threadIdx.x;
    if (x < count) atomicAdd(&h[(keys[x] >> shift) & (kRadix - 1)], 1);
  }
  __syncthreads();
  counts[int64_t(threadIdx.x) * tiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan, step 1: each CTA scans kScanThreads consecutive values in
// place and writes its total.
__global__ void __launch_bounds__(kScanThreads)
    scan_block_kernel(int32_t* __restrict__ v, int64_t count, int32_t* __restrict__ totals) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  const int64_t x = int64_t(blockIdx.x) * kScanThreads + threadIdx.x;
  const int32_t own = x < count ? v[x] : 0;
  int32_t incl = own;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int32_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  const int32_t before = (w > 0 ? warp_tot[w - 1] : 0) + incl - own;
  if (x < count) v[x] = before;
  if (threadIdx.x == kScanThreads - 1) totals[blockIdx.x] = warp_tot[kScanThreads / 32 - 1];
}

// Exclusive scan, step 3: adds each CTA's base (the scanned totals).
__global__ void __launch_bounds__(kScanThreads)
    scan_add_kernel(int32_t* __restrict__ v, int64_t count, const int32_t* __restrict__ bases) {
  const int64_t x = int64_t(blockIdx.x) * kScanThreads + threadIdx.x;
  if (x < count) v[x] += bases[blockIdx.x];
}

__global__ void __launch_bounds__(kSortThreads)
    radix_scatter_kernel(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                         int64_t count, int shift, const int32_t* __restrict__ offsets,
                         int64_t tiles, uint32_t* __restrict__ keys_out,
                         uint32_t* __restrict__ vals_out) {
  __shared__ int32_t running[kRadix];          // equal digits in earlier rounds
  __shared__ int32_t wcount[kSortWarps][kRadix];  // equal digits per warp, this round
  __shared__ int32_t first[kRadix];            // this tile's first position per digit
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  running[t] = 0;
  first[t] = offsets[int64_t(t) * tiles + blockIdx.x];
  for (int ww = 0; ww < kSortWarps; ++ww) wcount[ww][t] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t x = base + int64_t(r) * kSortThreads + t;
    const bool valid = x < count;
    const uint32_t key = valid ? keys_in[x] : 0u;
    const int d = valid ? int((key >> shift) & (kRadix - 1)) : kRadix;  // kRadix: no digit
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    if (valid && rank == 0) wcount[w][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int pos = first[d] + running[d] + rank;
      for (int ww = 0; ww < w; ++ww) pos += wcount[ww][d];
      keys_out[pos] = key;
      vals_out[pos] = vals_in[x];
    }
    __syncthreads();
    int add = 0;
    for (int ww = 0; ww < kSortWarps; ++ww) {
      add += wcount[ww][t];
      wcount[ww][t] = 0;
    }
    running[t] += add;
    __syncthreads();
  }
}

}  // namespace sort_detail

// Scratch (bytes) that exclusive_scan_i32 needs for `count` values.
inline size_t scan_scratch_bytes(int64_t count) {
  using namespace sort_detail;
  size_t b = 0;
  for (int64_t c = count; c > 1; c = (c + kScanThreads - 1) / kScanThreads)
    b += size_t((c + kScanThreads - 1) / kScanThreads) * sizeof(int32_t) + 256;
  return b + 256;
}

// In-place exclusive scan of `count` int32 values (sum < 2^31).
inline cudaError_t exclusive_scan_i32(int32_t* v, int64_t count, void* scratch, cudaStream_t s) {
  using namespace sort_detail;
  if (count <= 0) return cudaSuccess;
  const int64_t blocks = (count + kScanThreads - 1) / kScanThreads;
  int32_t* totals = static_cast<int32_t*>(scratch);
  scan_block_kernel<<<static_cast<unsigned>(blocks), kScanThreads, 0, s>>>(v, count, totals);
  if (blocks > 1) {
    unsigned char* next = static_cast<unsigned char*>(scratch) +
                          (size_t(blocks) * sizeof(int32_t) + 255) / 256 * 256;
    cudaError_t e = exclusive_scan_i32(totals, blocks, next, s);
    if (e != cudaSuccess) return e;
    scan_add_kernel<<<static_cast<unsigned>(blocks), kScanThreads, 0, s>>>(v, count, totals);
  }
  return cudaGetLastError();
}

// Scratch (bytes) radix_sort_pairs needs for `count` pairs: one more key and
// value buffer, the digit counts and the scan's scratch.
inline size_t radix_sort_scratch_bytes(int64_t count) {
  using namespace sort_detail;
  const int64_t tiles = (count + kSortTile - 1) / kSortTile;
  const size_t pairs = (size_t(count) * sizeof(uint32_t) + 255) / 256 * 256;
  const size_t counts = (size_t(tiles) * kRadix * sizeof(int32_t) + 255) / 256 * 256;
  return 2 * pairs + counts + scan_scratch_bytes(tiles * kRadix);
}

// Stable sort of (keys, vals) by the low `bits` bits of the keys.  The result
// ends in keys/vals (the scratch holds the other buffer of each pass).
inline cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, int64_t count, int bits,
                                    void* scratch, cudaStream_t s) {
  using namespace sort_detail;
  if (count <= 1) return cudaSuccess;
  const int64_t tiles = (count + kSortTile - 1) / kSortTile;
  const size_t pairs = (size_t(count) * sizeof(uint32_t) + 255) / 256 * 256;
  unsigned char* p = static_cast<unsigned char*>(scratch);
  uint32_t* k2 = reinterpret_cast<uint32_t*>(p);
  uint32_t* v2 = reinterpret_cast<uint32_t*>(p + pairs);
  int32_t* counts = reinterpret_cast<int32_t*>(p + 2 * pairs);
  void* scan_scratch = p + 2 * pairs + (size_t(tiles) * kRadix * sizeof(int32_t) + 255) / 256 * 256;
  uint32_t *ki = keys, *vi = vals, *ko = k2, *vo = v2;
  const int passes = (bits + 7) / 8;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = 8 * pass;
    radix_count_kernel<<<static_cast<unsigned>(tiles), kSortThreads, 0, s>>>(ki, count, shift,
                                                                             counts, tiles);
    cudaError_t e = exclusive_scan_i32(counts, tiles * kRadix, scan_scratch, s);
    if (e != cudaSuccess) return e;
    radix_scatter_kernel<<<static_cast<unsigned>(tiles), kSortThreads, 0, s>>>(
        ki, vi, count, shift, counts, tiles, ko, vo);
    std::swap(ki, ko);
    std::swap(vi, vo);
  }
  if (ki != keys) {  // an odd number of passes: copy back
    cudaError_t e = cudaMemcpyAsync(keys, ki, size_t(count) * sizeof(uint32_t),
                                    cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(vals, vi, size_t(count) * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace idw
