// Stable least-significant-digit radix sort of 64-bit items by the key in
// their high word (the low word is a payload that travels with it), and a
// device-wide exclusive scan of int32 counts.  The deterministic gradient of
// the k-NN form uses it to turn the query-major list of (data point, query)
// selections into a point-major one whose queries stay in increasing order
// within each point (stability), so every point's terms are summed in one
// fixed order.
//
// One pass sorts on 8 bits of the key:
//   1. count: each CTA counts the digits of its tile of kSortTile items
//      (shared-memory atomics: counts do not depend on order);
//   2. scan: the counts, laid out digit-major (digit d of tile b at
//      d * tiles + b), are scanned into each (digit, tile)'s first output
//      position;
//   3. scatter: each CTA loads its tile into registers, a contiguous slice
//      per warp, and ranks every item among the equal digits before it in
//      its warp's slice (lanes of a round by a match mask, rounds by the
//      warp's own digit counters, so no CTA barrier per round); the warps'
//      counts give each digit's start within the tile and each warp's
//      offset inside it; the items are placed in shared memory in digit
//      order and written out, a digit's items of one tile to consecutive
//      addresses, so the writes coalesce into runs instead of one scattered
//      8-byte store per item.  Equal keys keep their input order.
// Passes alternate between the caller's buffer and a scratch buffer; the
// sort returns whichever holds the result, so nothing is copied back.
#pragma once

#include <cstdint>
#include <utility>

#include <cuda_runtime.h>

namespace idw {
namespace sort_detail {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;  // 2048 items per CTA
constexpr int kRadix = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kScanThreads = 1024;
static_assert(kRadix == kSortThreads, "one digit per thread in the tile scan");

__device__ __forceinline__ int item_digit(uint64_t v, int shift) {
  return static_cast<int>((v >> (32 + shift)) & (kRadix - 1));
}

__global__ void __launch_bounds__(kSortThreads)
    radix_count_kernel(const uint64_t* __restrict__ items, int64_t count, int shift,
                       int32_t* __restrict__ counts, int64_t tiles) {
  __shared__ int32_t h[kRadix];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t x = base + int64_t(r) * kSortThreads + threadIdx.x;
    if (x < count) atomicAdd(&h[item_digit(items[x], shift)], 1);
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

__global__ void __launch_bounds__(kSortThreads, 4)
    radix_scatter_kernel(const uint64_t* __restrict__ in, int64_t count, int shift,
                         const int32_t* __restrict__ offsets, int64_t tiles,
                         uint64_t* __restrict__ out) {
  __shared__ uint64_t stage[kSortTile];           // the tile in digit order
  __shared__ int32_t wcount[kSortWarps][kRadix];  // per warp: digits seen, then its prefix
  __shared__ int32_t local[kRadix];               // each digit's start within the tile
  __shared__ int32_t first[kRadix];               // each digit's first output position
  __shared__ int32_t wsum[kSortWarps];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  const int in_tile = static_cast<int>(count - base < kSortTile ? count - base : kSortTile);
  first[t] = offsets[int64_t(t) * tiles + blockIdx.x];
  for (int ww = 0; ww < kSortWarps; ++ww) wcount[ww][t] = 0;
  __syncthreads();
  // Warp w owns items [w * 32 kSortRounds, (w + 1) * 32 kSortRounds) of the
  // tile, round r lane l holding item w * 32 kSortRounds + 32 r + l, so the
  // order (warp, round, lane) is the input order.  Its rank among the equal
  // digits before it within the warp: earlier rounds (the warp's own
  // counters) plus the lanes below it in its round (a match mask).
  uint64_t item[kSortRounds];
  int rank[kSortRounds];
  const int wbase = w * 32 * kSortRounds;
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int x = wbase + 32 * r + lane;
    item[r] = x < in_tile ? in[base + x] : 0ull;
  }
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int x = wbase + 32 * r + lane;
    const bool valid = x < in_tile;
    const int d = valid ? item_digit(item[r], shift) : kRadix;  // kRadix: no digit
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int below = __popc(peers & lt);
    const int seen = wcount[w][valid ? d : 0];
    rank[r] = valid ? seen + below : 0;
    __syncwarp();
    if (valid && below == 0) wcount[w][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // Digit t: the warps' counts become their exclusive prefix, and the tile's
  // total for the digit is scanned over the digits into its start.
  int32_t own = 0;
  for (int ww = 0; ww < kSortWarps; ++ww) {
    const int32_t c = wcount[ww][t];
    wcount[ww][t] = own;
    own += c;
  }
  int32_t incl = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  int32_t before = incl - own;
  for (int ww = 0; ww < w; ++ww) before += wsum[ww];
  local[t] = before;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int x = wbase + 32 * r + lane;
    if (x < in_tile) {
      const int d = item_digit(item[r], shift);
      stage[local[d] + wcount[w][d] + rank[r]] = item[r];
    }
  }
  __syncthreads();
  // Positions i .. of one digit are consecutive here and in the output.
  for (int i = t; i < in_tile; i += kSortThreads) {
    const uint64_t v = stage[i];
    const int d = item_digit(v, shift);
    out[first[d] + (i - local[d])] = v;
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

// Scratch (bytes) radix_sort_items needs for `count` items: the second item
// buffer, the digit counts and the scan's scratch.
inline size_t radix_sort_scratch_bytes(int64_t count) {
  using namespace sort_detail;
  const int64_t tiles = (count + kSortTile - 1) / kSortTile;
  const size_t items = (size_t(count) * sizeof(uint64_t) + 255) / 256 * 256;
  const size_t counts = (size_t(tiles) * kRadix * sizeof(int32_t) + 255) / 256 * 256;
  return items + counts + scan_scratch_bytes(tiles * kRadix);
}

// Stable sort of `count` items by the low `bits` bits of their high words.
// *result is set to the buffer that holds the sorted items: `items` after an
// even number of 8-bit passes, the scratch buffer after an odd one.
inline cudaError_t radix_sort_items(uint64_t* items, int64_t count, int bits, void* scratch,
                                    cudaStream_t s, uint64_t** result) {
  using namespace sort_detail;
  *result = items;
  if (count <= 1) return cudaSuccess;
  const int64_t tiles = (count + kSortTile - 1) / kSortTile;
  const size_t ibytes = (size_t(count) * sizeof(uint64_t) + 255) / 256 * 256;
  unsigned char* p = static_cast<unsigned char*>(scratch);
  uint64_t* other = reinterpret_cast<uint64_t*>(p);
  int32_t* counts = reinterpret_cast<int32_t*>(p + ibytes);
  void* scan_scratch = p + ibytes + (size_t(tiles) * kRadix * sizeof(int32_t) + 255) / 256 * 256;
  uint64_t *src = items, *dst = other;
  const int passes = (bits + 7) / 8;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = 8 * pass;
    radix_count_kernel<<<static_cast<unsigned>(tiles), kSortThreads, 0, s>>>(src, count, shift,
                                                                             counts, tiles);
    cudaError_t e = exclusive_scan_i32(counts, tiles * kRadix, scan_scratch, s);
    if (e != cudaSuccess) return e;
    radix_scatter_kernel<<<static_cast<unsigned>(tiles), kSortThreads, 0, s>>>(
        src, count, shift, counts, tiles, dst);
    std::swap(src, dst);
  }
  *result = src;
  return cudaGetLastError();
}

}  // namespace idw
