// Local (radius-limited) Shepard interpolation: Eq. 1 over the data points
// within distance R of each query.  This is the local variant of the IDW
// implementations the paper cites as related work (Sec. 1), not its global
// method.
//
// Pipeline (all on the caller's stream, no host synchronisation):
//   1. bounding box of the finite data points; the last block plans a
//      uniform grid of cells about R/2 wide, at most 2048 per axis and at
//      most one per two data points (coarser when the box needs it);
//   2. counting sort of the data AND of the queries into the cells
//      (histogram, exclusive scan, scatter of 16-byte records);
//   3. one thread per query, in cell order, walks the rows of cells that its
//      disc of radius R can reach (at most 5 rows of at most 5 cells), each
//      row one contiguous run of sorted data.
// Membership is decided in FP32 as d^2 = fmaf(dy, dy, fl32(dx dx)) <
// fl32(R^2) on the caller's unscaled coordinates.  Weights are FP32 (MUFU
// reciprocal at p = 2; 2^(-(p/2) log2 d^2) with an FMA-recovered exponent
// otherwise) and both sums are carried as compensated (hi, lo) FP32 pairs
// (Knuth's TwoSum per member), then divided with one residual correction.
// Sums that leave FP32's range, and queries that coincide with a data point
// (infinite weight), go to an FP64 pass: an exact hit takes the z of the
// lowest coincident index, other sums are redone with weights scaled by
// d2_min^(p/2).  An empty neighbourhood gives NaN.
//
// Cell positions are computed in FP32 as u(v) = fl(fl(fl(v/2) - fl(x0/2)) *
// inv2), inv2 = fl(2/h): halving is exact for normal floats and keeps the
// difference finite for any finite coordinates, and u is monotone in v.
// With at most 2048 cells per axis, u near the grid is off by at most
// 2^-23 (g + 2) ~ 2^-12 cells from (v - x0)/h.  A member lies less than
// R (1 + 2^-23) from its query (FP32 membership; R + 2^-74 where R^2 is
// subnormal, and h >= 2^-61), so in computed cell positions it lies within
// rho = (R/h)(1 + 2^-8) + 2^-8 of the query, which covers those errors and
// the FP32 rounding of the reach arithmetic.  With h >= R (1 + 2^-6)/2,
// rho < 2: a query scans rows floor(v_q) - 2 .. floor(v_q) + 2, and in each
// the columns floor(u_q - e) .. floor(u_q + e), e = sqrt(rho^2 - dy^2), dy
// the gap between v_q and the row.  Grids that need cells wider than 2^120
// (R or the data's extent near FP32's limit) fall back to a single cell.
// Scatter positions come from atomics, so the order of candidates within a
// cell (and with it the last bits of the compensated sums) can vary between
// calls.
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdint>

#include <algorithm>
#include <type_traits>

#include "idw.h"
#include "idw_device.cuh"
#include "idw_internal.h"
#include "idw_local.h"
#include "idw_sort.cuh"

namespace idw {
namespace {

constexpr int kScanBlock = 1024;            // threads of a scan block
constexpr int kScanTile = 4 * kScanBlock;  // entries of a scan tile (an int4 per thread)
constexpr int kLocalThreads = 256;
constexpr int kMaxCellsPerAxis = 2048;
constexpr int kBlockShift = 3;  // occupancy blocks of 8 x 8 cells (k-NN search)
constexpr int kMaxBlocksPerAxis = kMaxCellsPerAxis >> kBlockShift;
// A compensated weight sum below this per member may have lost flushed
// (FTZ) weights: such queries are redone in FP64.
constexpr float kTinyPerMember = 0x1p-100f;

// Index checks of a debug build (-DIDW_DEBUG_CHECKS): a failed check sets
// its site's bit in a device word and the access it guards is skipped; no
// trap.  Release builds compile every check to `true`.
enum DebugSite : unsigned {
  kSiteCell = 0,      // a cell index outside [0, cells]
  kSiteGather = 1,    // a sorted-data position outside [0, n)
  kSiteScatter = 2,   // a scatter position outside its array
  kSiteOutput = 3,    // an output row outside [0, m)
  kSiteHeap = 4,      // a heap slot outside [0, k)
  kSiteBlock = 5,     // an occupancy-block index outside the prefix table
  kSiteData = 6,      // a data index outside [0, n)
  kSiteTable = 7,     // a summed-area-table entry outside (gx + 1)(gy + 1)
};
#ifdef IDW_DEBUG_CHECKS
__device__ unsigned g_debug_failures;
__device__ __forceinline__ bool dcheck(bool ok, DebugSite site) {
  if (!ok) atomicOr(&g_debug_failures, 1u << site);
  return ok;
}
#else
__device__ __forceinline__ constexpr bool dcheck(bool, DebugSite) { return true; }
#endif

// Grid of cells, planned on the device.  Each call starts by setting every
// byte of it to 0xff (keys at their identity, tickets at -1).
struct GridDev {
  unsigned keys[4];      // min x, min y, ~max x, ~max y (order-preserving keys)
  unsigned box_ticket;   // blocks of the box kernel done, minus one
  unsigned scan_ticket;  // scan tiles done, minus one
  float hx0, hy0, inv2;  // cell position u(v) = fl(fl(fl(v/2) - h0) * inv2)
  float rho;             // reach of R in cells, with margin (< 2)
  int gx, gy, cells;
};

// Order-preserving unsigned key of a float (for atomic min).
__device__ __forceinline__ unsigned float_key(float f) {
  const unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__device__ __forceinline__ bool finite2(float x, float y) {
  return fabsf(x) <= FLT_MAX && fabsf(y) <= FLT_MAX;
}

// Ticket counter: atomic add with acquire-release semantics at GPU scope.
// Its release orders the caller's earlier writes before the increment; the
// caller that draws the last ticket acquires every earlier caller's writes.
__device__ __forceinline__ unsigned ticket_acq_rel(unsigned* counter) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
               : "=r"(old)
               : "l"(counter)
               : "memory");
  return old;
}

// Cell position along one axis (same arithmetic for data and queries).
__device__ __forceinline__ float cell_pos(float v, float h0, float inv2) {
  return __fmul_rn(__fsub_rn(__fmul_rn(0.5f, v), h0), inv2);
}
// floor(u) clamped to [lo, hi] (u may be +-inf for far queries, never NaN).
__device__ __forceinline__ int clamp_floor(float u, int lo, int hi) {
  return static_cast<int>(fminf(fmaxf(floorf(u), float(lo)), float(hi)));
}

// Grid for the box in grid->keys (one thread).  For the k-NN form
// (knn_k > 0) the cells are sized as for a radius holding k points at the
// data's mean density over the box, sqrt(k area / (pi n)); the radius only
// sets the cell size there, not the result.
__device__ void plan_grid(GridDev* grid, double radius, double inv_max_cells, int knn_k,
                          int64_t n) {
  const unsigned k0 = __ldcg(&grid->keys[0]), k1 = __ldcg(&grid->keys[1]);
  const unsigned k2 = __ldcg(&grid->keys[2]), k3 = __ldcg(&grid->keys[3]);
  int gx = 1, gy = 1;
  float hx0 = 0.f, hy0 = 0.f, inv2 = 0.f, rho = 1.f;  // inv2 = 0: one cell
  if (k0 != 0xffffffffu) {  // some finite data point
    const float xmin = key_float(k0), ymin = key_float(k1);
    const float xmax = key_float(~k2), ymax = key_float(~k3);
    const double ex = double(xmax) - xmin, ey = double(ymax) - ymin;
    if (knn_k > 0) {
      if (ex * ey > 0.0)
        radius = sqrt(double(knn_k) * ex * ey / (3.141592653589793 * double(n)));
      else if (fmax(ex, ey) > 0.0)
        radius = fmax(ex, ey) * double(knn_k) / (2.0 * double(n));  // points on a line
      else
        radius = 1.0;  // all points coincide: one cell
    }
    double h = fmax(fmax(radius * (0.5 + 0x1p-7), 0x1p-61),
                    fmax(ex * (1.0 / (kMaxCellsPerAxis - 1)), ey * (1.0 / (kMaxCellsPerAxis - 1))));
    h = fmax(h, sqrt(ex * ey * inv_max_cells));
    const float cap = float(kMaxCellsPerAxis - 1), max_cells = float(1.0 / inv_max_cells);
    for (int it = 0; it < 64 && h <= 0x1p120; ++it, h *= 1.25) {
      const float i2 = 2.f * __frcp_rn(__double2float_ru(h));
      const float ux = floorf(cell_pos(xmax, 0.5f * xmin, i2));
      const float uy = floorf(cell_pos(ymax, 0.5f * ymin, i2));
      if (ux <= cap && uy <= cap && (ux + 1.f) * (uy + 1.f) <= max_cells) {
        gx = int(ux) + 1;
        gy = int(uy) + 1;
        hx0 = 0.5f * xmin;
        hy0 = 0.5f * ymin;
        inv2 = i2;
        // h <= 2^120 and h >= R (1 + 2^-6)/2, so R fits a float.
        rho = __fmaf_ru(__fmul_ru(__double2float_ru(radius), i2), 0.5f + 0x1p-9f, 0x1p-8f);
        break;
      }
    }
  }
  grid->hx0 = hx0;
  grid->hy0 = hy0;
  grid->inv2 = inv2;
  grid->rho = rho;
  grid->gx = gx;
  grid->gy = gy;
  grid->cells = gx * gy;
}

// Bounding box of the finite data points; the last block to finish plans
// the grid.
__global__ void __launch_bounds__(256)
    box_plan_kernel(const float* __restrict__ data, int64_t n, GridDev* __restrict__ grid,
                    double radius, double inv_max_cells, int knn_k) {
  __shared__ unsigned part[4][8];
  __shared__ bool last;
  unsigned k0 = 0xffffffffu, k1 = 0xffffffffu, k2 = 0xffffffffu, k3 = 0xffffffffu;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    const float x = data[3 * i], y = data[3 * i + 1];
    if (finite2(x, y)) {
      k0 = min(k0, float_key(x));
      k1 = min(k1, float_key(y));
      k2 = min(k2, ~float_key(x));
      k3 = min(k3, ~float_key(y));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    k0 = min(k0, __shfl_xor_sync(0xffffffffu, k0, o));
    k1 = min(k1, __shfl_xor_sync(0xffffffffu, k1, o));
    k2 = min(k2, __shfl_xor_sync(0xffffffffu, k2, o));
    k3 = min(k3, __shfl_xor_sync(0xffffffffu, k3, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    part[0][wid] = k0;
    part[1][wid] = k1;
    part[2][wid] = k2;
    part[3][wid] = k3;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    unsigned k = 0xffffffffu;
    for (int w = 0; w < 8; ++w) k = min(k, part[threadIdx.x][w]);
    atomicMin(&grid->keys[threadIdx.x], k);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&grid->box_ticket, 1u) + 1u == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    plan_grid(grid, radius, inv_max_cells, knn_k, n);
  }
}

// Zeroes both histograms over cells + 1 entries rounded up to a multiple of
// four (the scan reads them as int4).
__global__ void __launch_bounds__(256)
    zero_counts_kernel(const GridDev* __restrict__ grid, int32_t* __restrict__ counts_d,
                       int32_t* __restrict__ counts_q) {
  const int len = (grid->cells + 1 + 3) & ~3;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
    counts_d[i] = 0;
    counts_q[i] = 0;
  }
}

// Cell of a data point (-1: a non-finite point, in no cell) and sorting
// bucket of a query (its cell clamped into the grid).
__device__ __forceinline__ int data_cell(const GridDev& g, float x, float y) {
  if (!finite2(x, y)) return -1;
  const int cx = clamp_floor(cell_pos(x, g.hx0, g.inv2), 0, g.gx - 1);
  const int cy = clamp_floor(cell_pos(y, g.hy0, g.inv2), 0, g.gy - 1);
  return cy * g.gx + cx;
}
__device__ __forceinline__ int query_bucket(const GridDev& g, float x, float y) {
  if (!finite2(x, y)) return 0;
  const int cx = clamp_floor(cell_pos(x, g.hx0, g.inv2), 0, g.gx - 1);
  const int cy = clamp_floor(cell_pos(y, g.hy0, g.inv2), 0, g.gy - 1);
  return cy * g.gx + cx;
}

// Threads [0, n) count data points, [n, n + m) count queries.
__global__ void __launch_bounds__(256)
    count_kernel(const GridDev* __restrict__ grid, const float* __restrict__ data, int64_t n,
                 const float* __restrict__ queries, int64_t m, int32_t* __restrict__ counts_d,
                 int32_t* __restrict__ counts_q) {
  const GridDev g = *grid;
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    const int c = data_cell(g, data[3 * i], data[3 * i + 1]);
    if (c >= 0) atomicAdd(&counts_d[c], 1);
  } else if (i < n + m) {
    const int64_t j = i - n;
    atomicAdd(&counts_q[query_bucket(g, queries[2 * j], queries[2 * j + 1])], 1);
  }
}

// Exclusive scan of one value per thread over a kScanBlock-thread block;
// `total` receives the block's sum.  `warp_tot` holds kScanBlock / 32 ints.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t* warp_tot,
                                                        int32_t& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int32_t w = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    warp_tot[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  total = warp_tot[kScanBlock / 32 - 1];
  return (wid > 0 ? warp_tot[wid - 1] : 0) + incl - v;
}

// Exclusive scan of the histograms (half = first + blockIdx.y: 0 data,
// 1 queries; launched with gridDim.y = 2 for both, 1 for one), one tile of
// kScanTile entries per block (four consecutive entries per thread), over
// cells + 1 entries.  Each tile writes its local prefix to starts[],
// clears the counts (they become the scatter cursors) and records its total;
// the block that finishes last turns the totals into tile bases (exclusive
// scan in place), so that a cell starts at starts[i] + base[i / kScanTile].
// The histogram arrays hold a multiple of four entries, 16-byte aligned.
__global__ void __launch_bounds__(kScanBlock)
    scan_kernel(GridDev* __restrict__ grid, int32_t* __restrict__ counts_d,
                int32_t* __restrict__ counts_q, int32_t* __restrict__ starts_d,
                int32_t* __restrict__ starts_q, int32_t* __restrict__ sums, int max_tiles,
                int first) {
  __shared__ int32_t warp_tot[kScanBlock / 32];
  __shared__ bool last;
  const int len = grid->cells + 1;
  const int ntiles = (len + kScanTile - 1) / kScanTile;
  if (int(blockIdx.x) >= ntiles) return;  // tile beyond the grid
  const int half = first + int(blockIdx.y);
  int4* in = reinterpret_cast<int4*>(half ? counts_q : counts_d);
  int4* out = reinterpret_cast<int4*>(half ? starts_q : starts_d);
  const int i4 = blockIdx.x * kScanBlock + threadIdx.x;  // int4 index
  int4 v = make_int4(0, 0, 0, 0);
  if (4 * i4 < len) {
    v = in[i4];
    in[i4] = make_int4(0, 0, 0, 0);
  }
  // Entries past len are zero: the arrays are cleared up to a multiple of 4.
  int32_t total;
  const int32_t before = block_exclusive_scan(v.x + v.y + v.z + v.w, warp_tot, total);
  if (4 * i4 < len)
    out[i4] = make_int4(before, before + v.x, before + v.x + v.y, before + v.x + v.y + v.z);
  if (threadIdx.x == 0) {
    sums[half * max_tiles + blockIdx.x] = total;  // published by the ticket
    last = ticket_acq_rel(&grid->scan_ticket) + 1u == unsigned(int(gridDim.y) * ntiles - 1);
  }
  __syncthreads();  // the last block's threads read after thread 0's acquire
  if (!last) return;
  const int per = (ntiles + kScanBlock - 1) / kScanBlock;
  for (int y = first; y < first + int(gridDim.y); ++y) {
    int32_t* sb = sums + y * max_tiles;
    const int b0 = min(ntiles, int(threadIdx.x) * per), b1 = min(ntiles, b0 + per);
    int32_t acc = 0;
    for (int b = b0; b < b1; ++b) acc += __ldcg(&sb[b]);
    __syncthreads();  // warp_tot is reused
    int32_t run = block_exclusive_scan(acc, warp_tot, total);
    for (int b = b0; b < b1; ++b) {
      const int32_t t = __ldcg(&sb[b]);
      sb[b] = run;
      run += t;
    }
  }
}

__device__ __forceinline__ int cell_start(const int32_t* __restrict__ starts,
                                          const int32_t* __restrict__ base, int i, int cells) {
  if (!dcheck(i >= 0 && i <= cells, kSiteCell)) return 0;
  return starts[i] + base[i / kScanTile];
}

// Occupancy of 8 x 8-cell blocks for the k-NN search: for block row by,
// bpre[by * (kMaxBlocksPerAxis + 1) + bx] is the number of data points in
// blocks 0 .. bx - 1 of that row.  One CTA per block row, one thread per
// block; runs after the scan (cell starts are final).
__global__ void __launch_bounds__(kMaxBlocksPerAxis)
    block_prefix_kernel(const GridDev* __restrict__ grid, const int32_t* __restrict__ starts,
                        const int32_t* __restrict__ base, int32_t* __restrict__ bpre) {
  __shared__ int32_t warp_tot[kMaxBlocksPerAxis / 32];
  const GridDev g = *grid;
  const int bgx = (g.gx + 7) >> kBlockShift, bgy = (g.gy + 7) >> kBlockShift;
  const int by = blockIdx.x;
  if (by >= bgy) return;
  const int bx = threadIdx.x;
  int32_t c = 0;
  if (bx < bgx) {
    const int x0 = bx << kBlockShift, x1 = min(g.gx - 1, x0 + 7);
    const int y0 = by << kBlockShift, y1 = min(g.gy - 1, y0 + 7);
    for (int yy = y0; yy <= y1; ++yy)
      c += cell_start(starts, base, yy * g.gx + x1 + 1, g.cells) -
           cell_start(starts, base, yy * g.gx + x0, g.cells);
  }
  // Exclusive scan over the row's blocks (kMaxBlocksPerAxis threads).
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  int32_t before = incl - c;
  for (int w = 0; w < wid; ++w) before += warp_tot[w];
  int32_t* row = bpre + by * (kMaxBlocksPerAxis + 1);
  if (bx < bgx) row[bx] = before;
  if (bx == bgx - 1) row[bgx] = before + c;  // the row total
}

// Summed-area table of the data cells for the k-NN search: with W = gx + 1,
// sat[y * W + x] is the number of data points in rows 0 .. y - 1 and columns
// 0 .. x - 1, so any rectangle of cells is counted from four entries.  A
// CTA takes 32 columns; its warp w sums rows w C .. (w + 1) C - 1 of each
// column (C = ceil(gy / 32)), the warps' totals are scanned through shared
// memory, and each warp writes its rows.  Launched with enough CTAs for
// 2049 columns; those past gx + 1 return at once (the plan is on the
// device).
constexpr int kSatCols = 32, kSatWarps = 32;
__global__ void __launch_bounds__(kSatCols * kSatWarps)
    sat_kernel(const GridDev* __restrict__ grid, const int32_t* __restrict__ starts,
               const int32_t* __restrict__ base, int32_t* __restrict__ sat) {
  __shared__ int32_t part[kSatWarps][kSatCols];
  const GridDev g = *grid;
  if (int(blockIdx.x) * kSatCols > g.gx) return;  // the whole CTA: no barrier is reached
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int W = g.gx + 1, x = blockIdx.x * kSatCols + lane;
  const int chunk = (g.gy + kSatWarps - 1) / kSatWarps;
  const int y0 = min(g.gy, w * chunk), y1 = min(g.gy, y0 + chunk);
  // Points of row y in columns 0 .. x - 1 (x = gx: the whole row).
  auto row_prefix = [&](int y) {
    return cell_start(starts, base, y * g.gx + x, g.cells) -
           cell_start(starts, base, y * g.gx, g.cells);
  };
  int32_t s = 0;
  if (x < W)
    for (int y = y0; y < y1; ++y) s += row_prefix(y);
  part[w][lane] = s;
  __syncthreads();
  int32_t acc = 0;
  for (int i = 0; i < w; ++i) acc += part[i][lane];
  if (x < W) {
    if (w == 0) sat[x] = 0;
    for (int y = y0; y < y1; ++y) {
      acc += row_prefix(y);
      if (dcheck(y + 1 <= g.gy, kSiteTable)) sat[(y + 1) * W + x] = acc;
    }
  }
}

// Query records in the caller's order, (x, y, index, 0): used in place of
// the query sort when the caller's order is kept.
__global__ void __launch_bounds__(256)
    query_identity_kernel(const float* __restrict__ queries, int64_t m,
                          float4* __restrict__ qrec) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= m) return;
  qrec[j] = make_float4(queries[2 * j], queries[2 * j + 1], __int_as_float(static_cast<int>(j)),
                        0.f);
}

// Threads [0, n) place data points as (x, y, z, index), [n, n + m) place
// queries as (x, y, index, 0).
__global__ void __launch_bounds__(256)
    scatter_kernel(const GridDev* __restrict__ grid, const float* __restrict__ data, int64_t n,
                   const float* __restrict__ queries, int64_t m,
                   const int32_t* __restrict__ starts_d, const int32_t* __restrict__ starts_q,
                   const int32_t* __restrict__ sums, int max_tiles,
                   int32_t* __restrict__ cursor_d, int32_t* __restrict__ cursor_q,
                   float4* __restrict__ sorted, float4* __restrict__ qrec) {
  const GridDev g = *grid;
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) {
    const float x = data[3 * i], y = data[3 * i + 1];
    const int c = data_cell(g, x, y);
    if (c < 0) return;
    const int pos = cell_start(starts_d, sums, c, g.cells) + atomicAdd(&cursor_d[c], 1);
    if (!dcheck(pos >= 0 && pos < n, kSiteScatter)) return;
    sorted[pos] = make_float4(x, y, data[3 * i + 2], __int_as_float(static_cast<int>(i)));
  } else if (i < n + m) {
    const int64_t j = i - n;
    const float x = queries[2 * j], y = queries[2 * j + 1];
    const int b = query_bucket(g, x, y);
    const int pos = cell_start(starts_q, sums + max_tiles, b, g.cells) + atomicAdd(&cursor_q[b], 1);
    if (!dcheck(pos >= 0 && pos < m, kSiteScatter)) return;
    qrec[pos] = make_float4(x, y, __int_as_float(static_cast<int>(j)), 0.f);
  }
}

template <int MODE>
__device__ __forceinline__ float local_weight(float d2, float hp, float nhp) {
  if (MODE == kPow2) return rcp_approx(d2);
  const float L = lg2_approx(d2);
  const float th = L * nhp;
  const float tl = fmaf(L, nhp, L * hp);  // exact rounding error of th
  const float e = ex2_approx(th);
  return fmaf(e, tl * 0.6931471805599453f, e);
}

// MUFU square root (relative error ~2^-22, subnormal input flushed to 0).
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float fp32_d2(float qx, float qy, float x, float y) {
  const float dx = __fsub_rn(qx, x), dy = __fsub_rn(qy, y);
  return __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
}

// The runs of sorted data a query's disc of radius R can reach: at most
// five rows, each one contiguous run [a[r], b[r]) (empty runs have a == b).
// All runs are looked up before any is walked, so their loads overlap.
// The reach e of a row comes from the MUFU square root: its error (and a
// flushed subnormal rho^2 - dy^2, where no member can lie) is far inside
// rho's margin.
struct Runs {
  int a[5], b[5];

  __device__ __forceinline__ Runs(const GridDev& g, float qx, float qy,
                                  const int32_t* __restrict__ starts,
                                  const int32_t* __restrict__ base) {
    int y0 = 0, y1 = -1;
    float u = 0.f, v = 0.f;
    if (finite2(qx, qy)) {
      u = cell_pos(qx, g.hx0, g.inv2);
      v = cell_pos(qy, g.hy0, g.inv2);
      const int cy = clamp_floor(v, -3, g.gy + 2);
      y0 = cy - 2;
      y1 = min(g.gy - 1, cy + 2);
    }
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      const int yy = y0 + r;
      const float dy = fmaxf(0.f, fmaxf(float(yy) - v, v - float(yy + 1)));
      const float e = sqrt_approx(fmaxf(0.f, __fmaf_rn(-dy, dy, g.rho * g.rho)));
      const int xa = clamp_floor(u - e, 0, g.gx), xb = clamp_floor(u + e, -1, g.gx - 1);
      a[r] = b[r] = 0;
      if (yy >= 0 && yy <= y1 && dy < g.rho && xa <= xb) {
        a[r] = cell_start(starts, base, yy * g.gx + xa, g.cells);
        b[r] = cell_start(starts, base, yy * g.gx + xb + 1, g.cells);
      }
    }
  }
};

// One thread per query, in cell order.  The fast loop takes every candidate
// with d^2 < r2t, r2t = fl32(R^2) (or the least subnormal when that is 0,
// so that only d^2 == 0 passes), and sums its FP32 weight.  A coincident
// point (d^2 == 0) has an infinite or NaN weight, so a query with an exact
// hit, or with sums outside FP32's range, falls through to the FP64 pass,
// which takes the z of the lowest coincident index or recomputes the sums
// with weights scaled by d2_min^(p/2).
// Weights of the radius form: d^-p (kWeightShepard) or the modified
// Shepard weights ((R - d)/(R d))^p = (1/d - 1/R)^p (kWeightModified), which
// fall to 0 at d = R.  The modified base comes from the MUFU reciprocal
// square root (relative error ~2^-22) and is clamped at 0 for members that
// rounding puts at the boundary; a coincident point gives an infinite base.
constexpr int kWeightShepard = 0, kWeightModified = 1;
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
template <int MODE>
__device__ __forceinline__ float modified_weight(float d2, float inv_r, float pw) {
  const float t = fmaxf(rsqrt_approx(d2) - inv_r, 0.f);
  if (MODE == kPow2) return t * t;
  return ex2_approx(pw * lg2_approx(t));
}

template <int MODE, int WMODE = kWeightShepard>
__global__ void __launch_bounds__(kLocalThreads)
    local_query_kernel(const GridDev* __restrict__ grid, const float4* __restrict__ sorted,
                       int64_t n, const int32_t* __restrict__ starts,
                       const int32_t* __restrict__ base, const float4* __restrict__ qrec,
                       int64_t m, double p, float r2f, float r2t, float* __restrict__ out,
                       int32_t* __restrict__ count_out, double radius = 0.0) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const float4 r = qrec[t];
  const float qx = r.x, qy = r.y;
  const int j = __float_as_int(r.z);
  if (!dcheck(j >= 0 && j < m, kSiteOutput)) return;
  const Runs runs(*grid, qx, qy, starts, base);
  const float hp = static_cast<float>(0.5 * p), nhp = -hp;
  const float pw = static_cast<float>(p);
  const float inv_r = WMODE == kWeightModified ? static_cast<float>(1.0 / radius) : 0.f;

  // (sum w, sum w z) and their TwoSum errors.  The products w z are rounded
  // once (2^-24), below the error of the MUFU weights themselves (2^-23).
  u64 hi = 0, lo = 0;
  int cnt = 0;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
#pragma unroll 2
    for (int k = runs.a[r]; k < runs.b[r]; ++k) {
      if (!dcheck(k >= 0 && k < n, kSiteGather)) break;
      const float4 v = sorted[k];
      const float d2 = fp32_d2(qx, qy, v.x, v.y);
      if (d2 < r2t) {
        const float w = WMODE == kWeightModified ? modified_weight<MODE>(d2, inv_r, pw)
                                                 : local_weight<MODE>(d2, hp, nhp);
        two_sum_acc(hi, lo, pk(w, __fmul_rn(w, v.z)));
        ++cnt;
      }
    }
  }
  if (cnt == 0) {  // no member and no coincident point
    out[j] = __int_as_float(0x7fc00000);
    if (count_out) count_out[j] = 0;
    return;
  }
  float h0, h1, l0, l1;
  upk(hi, h0, h1);
  upk(lo, l0, l1);
  if (h0 >= kTinyPerMember * float(cnt) && h0 <= FLT_MAX && fabsf(h1) <= FLT_MAX &&
      fabsf(l1) <= FLT_MAX) {
    // Z = (h1 + l1) / (h0 + l0): quotient, then one residual correction.
    const float z0 = __fdiv_rn(h1, h0);
    const float res = __fadd_rn(__fmaf_rn(-z0, h0, h1), __fmaf_rn(-z0, l0, l1));
    out[j] = __fmaf_rn(res, rcp_approx(h0), z0);
    if (count_out) count_out[j] = cnt;
    return;
  }
  // FP64 pass: exact hits first, then the members' d2_min (or, for the
  // modified weights, their largest base (R - d)/(R d), clamped at 0).
  int best = INT_MAX, members = 0;
  float bestz = 0.f;
  double dmin = INFINITY, tmax = 0.0;
  auto base64 = [&](double e2) {
    const double d = sqrt(e2);
    const double t = isinf(radius) ? 1.0 / d : (radius - d) / (radius * d);
    return t > 0.0 ? t : 0.0;
  };
#pragma unroll
  for (int r = 0; r < 5; ++r)
    for (int k = runs.a[r]; k < runs.b[r]; ++k) {
      const float4 v = sorted[k];
      if (v.x == qx && v.y == qy) {
        const int idx = __float_as_int(v.w);
        if (idx < best) {
          best = idx;
          bestz = v.z;
        }
      } else if (fp32_d2(qx, qy, v.x, v.y) < r2f) {
        const double ex = double(qx) - v.x, ey = double(qy) - v.y;
        dmin = fmin(dmin, ex * ex + ey * ey);
        if (WMODE == kWeightModified) tmax = fmax(tmax, base64(ex * ex + ey * ey));
        ++members;
      }
    }
  if (best != INT_MAX || members == 0 || (WMODE == kWeightModified && !(tmax > 0.0))) {
    out[j] = best != INT_MAX ? bestz : __int_as_float(0x7fc00000);
    if (count_out) count_out[j] = best != INT_MAX ? -1 : members;
    return;
  }
  double s0 = 0.0, s1 = 0.0;
#pragma unroll
  for (int r = 0; r < 5; ++r)
    for (int k = runs.a[r]; k < runs.b[r]; ++k) {
      const float4 v = sorted[k];
      if (fp32_d2(qx, qy, v.x, v.y) < r2f) {
        const double ex = double(qx) - v.x, ey = double(qy) - v.y;
        const double w = WMODE == kWeightModified ? pow(base64(ex * ex + ey * ey) / tmax, p)
                                                  : pow(dmin / (ex * ex + ey * ey), 0.5 * p);
        s0 += w;
        s1 += w * double(v.z);
      }
    }
  out[j] = static_cast<float>(s1 / s0);
  if (count_out) count_out[j] = members;
}

// ------------------------------------------------- local-form gradients
//
// dL/d(inputs) of L = sum_j g_j Z(q_j) for the radius form.  Each query's
// membership set is held fixed (it is piecewise constant in every input), so
// every derivative is the global one (the chain rule on Eq. 1) summed over
// the members:
//   dZ/dz_i = w_i / S0,   dZ/dx_i = (p / S0)(z_i - Z) w_i (q - x_i) / d_i^2,
//   dZ/dq = -sum_i dZ/dx_i,   dZ/dp = -(1 / (2 S0)) sum_i (z_i - Z) w_i ln d_i^2.
// Weights are scaled by the members' smallest d^2 (w_i = (d2_min / d_i^2)^(p/2)
// <= 1): every formula is a ratio in w / S0, so the factor cancels, and
// nothing overflows.  Since sum_i (z_i - Z) w_i = 0, ln d_i^2 may be taken
// relative to d2_min.  An exact hit passes g_j to dL/dz of its point only; a
// query without members contributes nothing.
//
// Two kernels share one record per sorted query:
//   1. per query (in cell order): hit and members, the sums, Z, dL/dq and
//      the query's share of dL/dp (a warp sum, then one FP64 atomic);
//   2. per data point (in cell order): walks the sorted queries whose disc
//      can reach it (the grid's coverage argument is symmetric in the two
//      points) with the same FP32 membership test, and sums dL/dz_i and
//      dL/dx_i in registers: one write per point, no atomics.
// FP32 throughout, except queries whose d2_min is below 2^-100 (or zero
// without a coincident point) or whose FP32 sums are not finite: those use
// FP64 on both sides.
// The record read for every (point, query) candidate is 16 bytes of FP32
// (FP64-to-FP32 conversions run at the FP64 rate on this part); queries on
// the FP64 path keep their values in a second array read only for them.
struct LocalGradRec {
  float d2min;  // the weights' scale (FP32 path): the members' smallest d^2, or
                // for the modified weights their largest base 1/d - 1/R
  float c;      // g_j / S0 (scaled), or g_j at an exact hit
  float z;      // Z_j
  int code;     // >= 0: exact hit (data index); -1: nothing; -2: FP32; -3: FP64
};
struct LocalGradRec64 {
  double d2min, c, z;  // FP64 path only
};
constexpr int kGradHitNone = -1, kGradF32 = -2, kGradF64 = -3;

// Scaled FP32 weight (d2min / d2)^(p/2); lmin = log2(d2min) for general p.
template <int MODE>
__device__ __forceinline__ float grad_weight(float d2, float d2min, float lmin, float hp) {
  if (MODE == kPow2) return __fmul_rn(d2min, rcp_approx(d2));
  return ex2_approx(-hp * (lg2_approx(d2) - lmin));
}

// The FP64 path of one query (weights scaled by its exact d2_min^(p/2)):
// dL/dq, its dL/dp share and the record the data-side kernel reads.  Out of
// line, so that the rare FP64 branch adds no registers to the FP32 loops.
struct GradF64 {
  float gqx, gqy;
  double gp;
  LocalGradRec64 rec;
};
// FP64 weight terms of one member at squared distance e2 under the scale:
// the weight w, the pair factor f (w / d^2, or for the modified weights
// w / (t d^3)) and the dL/dp log term (ln of d^2 / d2_min, or of t / t_max).
struct GradTerms64 {
  double w, f, l;
};
__device__ __forceinline__ GradTerms64 grad_terms64(double e2, double scale, double p,
                                                    bool modified, double radius) {
  if (!modified) {
    const double w = pow(scale / e2, 0.5 * p);
    return GradTerms64{w, w / e2, log(e2 / scale)};
  }
  const double d = sqrt(e2);
  const double t = isinf(radius) ? 1.0 / d : (radius - d) / (radius * d);
  if (!(t > 0.0)) return GradTerms64{0.0, 0.0, 0.0};
  const double w = pow(t / scale, p);
  return GradTerms64{w, w / (t * e2 * d), log(t / scale)};
}

__device__ __noinline__ GradF64 grad_query_f64(const Runs runs, const float4* __restrict__ sorted,
                                               float qx, float qy, float r2f, double p,
                                               float gj, bool modified, double radius) {
  double scale = modified ? 0.0 : INFINITY;  // d2_min, or the largest base t
  for (int rr = 0; rr < 5; ++rr)
    for (int k = runs.a[rr]; k < runs.b[rr]; ++k) {
      const float4 v = sorted[k];
      if (!(fp32_d2(qx, qy, v.x, v.y) < r2f)) continue;
      const double ex = double(qx) - v.x, ey = double(qy) - v.y, e2 = ex * ex + ey * ey;
      if (modified) {
        const double d = sqrt(e2);
        scale = fmax(scale, isinf(radius) ? 1.0 / d : (radius - d) / (radius * d));
      } else {
        scale = fmin(scale, e2);
      }
    }
  GradF64 r{0.f, 0.f, 0.0, LocalGradRec64{0.0, 0.0, 0.0}};
  if (!(scale > 0.0)) return r;  // no member of positive weight: no gradient
  double s0 = 0.0, s1 = 0.0;
  for (int rr = 0; rr < 5; ++rr)
    for (int k = runs.a[rr]; k < runs.b[rr]; ++k) {
      const float4 v = sorted[k];
      if (!(fp32_d2(qx, qy, v.x, v.y) < r2f)) continue;
      const double ex = double(qx) - v.x, ey = double(qy) - v.y;
      const double w = grad_terms64(ex * ex + ey * ey, scale, p, modified, radius).w;
      s0 += w;
      s1 += w * double(v.z);
    }
  const double Z = s1 / s0;
  double ax = 0.0, ay = 0.0, al = 0.0;
  for (int rr = 0; rr < 5; ++rr)
    for (int k = runs.a[rr]; k < runs.b[rr]; ++k) {
      const float4 v = sorted[k];
      if (!(fp32_d2(qx, qy, v.x, v.y) < r2f)) continue;
      const double ex = double(qx) - v.x, ey = double(qy) - v.y;
      const GradTerms64 g = grad_terms64(ex * ex + ey * ey, scale, p, modified, radius);
      const double dz = double(v.z) - Z;
      ax += dz * g.f * ex;
      ay += dz * g.f * ey;
      al += dz * g.w * g.l;
    }
  r.gqx = static_cast<float>(-double(gj) * p / s0 * ax);
  r.gqy = static_cast<float>(-double(gj) * p / s0 * ay);
  r.gp = (modified ? 1.0 : -0.5) * double(gj) * al / s0;
  r.rec = LocalGradRec64{scale, double(gj) / s0, Z};
  return r;
}

// (a / b)^p for the modified weights (lb = log2 b; p = 2 needs no log).
template <int MODE>
__device__ __forceinline__ float modified_ratio(float a, float b, float lb, float pf) {
  if (MODE == kPow2) {
    const float r = a * rcp_approx(b);
    return r * r;
  }
  return ex2_approx(pf * (lg2_approx(a) - lb));
}

template <int MODE, int WMODE = kWeightShepard>
__global__ void __launch_bounds__(kLocalThreads)
    local_grad_query_kernel(const GridDev* __restrict__ grid, const float4* __restrict__ sorted,
                            int64_t n, const int32_t* __restrict__ starts,
                            const int32_t* __restrict__ base, const float4* __restrict__ qrec,
                            int64_t m, double p, float r2f, float r2t,
                            const float* __restrict__ grad_out, float* __restrict__ grad_q,
                            double* __restrict__ grad_p, LocalGradRec* __restrict__ rec,
                            LocalGradRec64* __restrict__ rec64, double radius) {
  constexpr bool kMod = WMODE == kWeightModified;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  double gp = 0.0;  // this query's share of dL/dp (every lane joins the warp sum)
  if (t < m) {
    const float4 r = qrec[t];
    const float qx = r.x, qy = r.y;
    const int j = __float_as_int(r.z);
    if (dcheck(j >= 0 && j < m, kSiteOutput)) {
      const float gj = grad_out[j];
      const Runs runs(*grid, qx, qy, starts, base);
      // One pass: hit, members, and the sums with weights scaled by the
      // heaviest member so far (the smallest d^2, or for the modified
      // weights the largest base 1/d - 1/R), rescaled as in an online softmax
      // when a heavier one appears, so every scaled weight stays <= 1.
      const float hp = static_cast<float>(0.5 * p), pf = static_cast<float>(p);
      const float inv_r = kMod ? static_cast<float>(1.0 / radius) : 0.f;
      int best = INT_MAX, members = 0;
      float d2min = INFINITY, scale = kMod ? 0.f : INFINITY, lsc = 0.f;
      // (sum w, sum w z) as a compensated pair, as in the forward pass: Z
      // and g / S0 then stay accurate however many members a query has.
      u64 hi = 0, lo = 0;
#pragma unroll
      for (int rr = 0; rr < 5; ++rr)
        for (int k = runs.a[rr]; k < runs.b[rr]; ++k) {
          if (!dcheck(k >= 0 && k < n, kSiteGather)) break;
          const float4 v = sorted[k];
          const float d2 = fp32_d2(qx, qy, v.x, v.y);
          if (!(d2 < r2t)) continue;
          if (v.x == qx && v.y == qy) {
            best = min(best, __float_as_int(v.w));
            continue;
          }
          if (!(d2 < r2f)) continue;
          ++members;
          d2min = fminf(d2min, d2);
          float w;
          if (kMod) {
            const float tb = fmaxf(rsqrt_approx(d2) - inv_r, 0.f);
            if (!(tb > 0.f)) continue;  // zero weight
            if (tb > scale) {
              const float l = MODE == kPow2 ? 0.f : lg2_approx(tb);
              if (scale > 0.f) {
                const float f = modified_ratio<MODE>(scale, tb, l, pf);  // (t_old / t)^p
                hi = mul2(hi, pk(f, f));
                lo = mul2(lo, pk(f, f));
              }
              scale = tb;
              lsc = l;
            }
            w = modified_ratio<MODE>(tb, scale, lsc, pf);
          } else {
            if (d2 < scale) {
              const float l = MODE == kPow2 ? 0.f : lg2_approx(d2);
              if (members > 1) {
                const float f = grad_weight<MODE>(scale, d2, l, hp);  // (d2 / d2min_old)^(p/2)
                hi = mul2(hi, pk(f, f));
                lo = mul2(lo, pk(f, f));
              }
              scale = d2;
              lsc = l;
            }
            w = grad_weight<MODE>(d2, scale, lsc, hp);
          }
          two_sum_acc(hi, lo, pk(w, __fmul_rn(w, v.z)));
        }
      float h0, h1, l0, l1;
      upk(hi, h0, h1);
      upk(lo, l0, l1);
      const float s0 = h0 + l0;
      LocalGradRec out{0.f, 0.f, 0.f, kGradHitNone};
      float gqx = 0.f, gqy = 0.f;
      if (best != INT_MAX) {
        out.code = best;
        out.c = gj;
      } else if (members > 0 && (!kMod || scale > 0.f)) {
        bool f32 = d2min >= 0x1p-100f;
        if (f32) {
          // Z = (h1 + l1) / (h0 + l0): quotient, then one residual correction.
          const float z0 = __fdiv_rn(h1, h0);
          const float Z = __fmaf_rn(__fadd_rn(__fmaf_rn(-z0, h0, h1), __fmaf_rn(-z0, l0, l1)),
                                    rcp_approx(h0), z0);
          const float lsc2 = lg2_approx(scale);
          float ax = 0.f, ay = 0.f, al = 0.f;
#pragma unroll
          for (int rr = 0; rr < 5; ++rr)
            for (int k = runs.a[rr]; k < runs.b[rr]; ++k) {
              const float4 v = sorted[k];
              const float dx = __fsub_rn(qx, v.x), dy = __fsub_rn(qy, v.y);
              const float d2 = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
              if (!(d2 < r2f)) continue;
              float w, ar, lt;
              if (kMod) {
                const float id = rsqrt_approx(d2);
                const float tb = fmaxf(id - inv_r, 0.f);
                if (!(tb > 0.f)) continue;
                w = modified_ratio<MODE>(tb, scale, lsc, pf);
                ar = (v.z - Z) * w * (id * id) * (id * rcp_approx(tb));  // / (t d^3)
                lt = lg2_approx(tb) - lsc2;
              } else {
                w = grad_weight<MODE>(d2, scale, lsc, hp);
                ar = (v.z - Z) * w * rcp_approx(d2);  // / d^2
                lt = lg2_approx(d2) - lsc2;
              }
              ax = fmaf(ar, dx, ax);
              ay = fmaf(ar, dy, ay);
              al = fmaf((v.z - Z) * w, lt, al);
            }
          const float c = gj / s0, k1 = c * pf;
          gqx = -k1 * ax;
          gqy = -k1 * ay;
          // dL/dp share in FP32 (no FP64 divide): -ln2/2 c al for d^-p,
          // +ln2 c al for the modified weights (dw/dp = w ln t).
          const float gpf = (kMod ? 0.6931471805599453f : -0.5f * 0.6931471805599453f) * c * al;
          gp = gpf;
          out.code = kGradF32;
          out.c = c;
          out.z = Z;
          out.d2min = scale;
          f32 = isfinite(Z) && isfinite(gqx) && isfinite(gqy) && isfinite(gpf) && isfinite(c);
        }
        if (!f32) {  // FP64: weights scaled by the exact scale
          const GradF64 r64 = grad_query_f64(runs, sorted, qx, qy, r2f, p, gj, kMod, radius);
          gqx = r64.gqx;
          gqy = r64.gqy;
          gp = r64.gp;
          out.code = r64.rec.c == 0.0 && r64.rec.d2min == 0.0 ? kGradHitNone : kGradF64;
          rec64[t] = r64.rec;
        }
      }
      rec[t] = out;
      if (grad_q) {
        grad_q[2 * int64_t(j)] = gqx;
        grad_q[2 * int64_t(j) + 1] = gqy;
      }
    }
  }
  if (grad_p) {
    gp = warp_sum(gp);
    if ((threadIdx.x & 31) == 0 && gp != 0.0) atomicAdd(grad_p, gp);
  }
}

// The FP64 path's share of one (point, query) pair: (dL/dz, dL/dx, dL/dy).
// Out of line, so that the rare FP64 branch adds no registers to the loop.
// One instance per weight mode, so the plain one passes no radius.
__device__ __forceinline__ float3 grad_pair_f64_terms(LocalGradRec64 D, float qx, float qy,
                                                      float4 v, double p, bool modified,
                                                      double radius) {
  const double ex = double(qx) - v.x, ey = double(qy) - v.y;
  const GradTerms64 g = grad_terms64(ex * ex + ey * ey, D.d2min, p, modified, radius);
  const double a = D.c * p * (double(v.z) - D.z) * g.f;
  return make_float3(static_cast<float>(D.c * g.w), static_cast<float>(a * ex),
                     static_cast<float>(a * ey));
}
__device__ __noinline__ float3 grad_pair_f64(LocalGradRec64 D, float qx, float qy, float4 v,
                                             double p) {
  return grad_pair_f64_terms(D, qx, qy, v, p, false, 0.0);
}
__device__ __noinline__ float3 grad_pair_f64_modified(LocalGradRec64 D, float qx, float qy,
                                                      float4 v, double p, double radius) {
  return grad_pair_f64_terms(D, qx, qy, v, p, true, radius);
}

template <int MODE, int WMODE = kWeightShepard>
__global__ void __launch_bounds__(kLocalThreads)
    local_grad_data_kernel(const GridDev* __restrict__ grid, const float4* __restrict__ sorted,
                           int64_t n, const int32_t* __restrict__ starts_d,
                           const int32_t* __restrict__ base_d,
                           const int32_t* __restrict__ starts_q,
                           const int32_t* __restrict__ base_q, const float4* __restrict__ qrec,
                           int64_t m, const LocalGradRec* __restrict__ rec,
                           const LocalGradRec64* __restrict__ rec64, double p, float r2f,
                           float* __restrict__ grad_z, float* __restrict__ grad_xy,
                           double radius) {
  constexpr bool kMod = WMODE == kWeightModified;
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const GridDev g = *grid;
  if (k >= cell_start(starts_d, base_d, g.cells, g.cells)) return;  // placed (finite) points
  if (!dcheck(k < n, kSiteGather)) return;
  const float4 v = sorted[k];
  const int idx = __float_as_int(v.w);
  if (!dcheck(idx >= 0 && idx < n, kSiteData)) return;
  const Runs runs(g, v.x, v.y, starts_q, base_q);
  const float hp = static_cast<float>(0.5 * p), pf = static_cast<float>(p);
  const float inv_r = kMod ? static_cast<float>(1.0 / radius) : 0.f;
  float gz = 0.f, gx = 0.f, gy = 0.f;
#pragma unroll
  for (int rr = 0; rr < 5; ++rr)
#pragma unroll 2
    for (int t = runs.a[rr]; t < runs.b[rr]; ++t) {
      if (!dcheck(t >= 0 && t < m, kSiteGather)) break;
      const LocalGradRec R = rec[t];  // both loads issue before any branch
      const float4 q = qrec[t];
      if (R.code == kGradHitNone) continue;
      if (R.code >= 0) {
        if (R.code == idx) gz += R.c;
        continue;
      }
      const float dx = __fsub_rn(q.x, v.x), dy = __fsub_rn(q.y, v.y);
      const float d2 = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
      if (!(d2 < r2f)) continue;  // the query's membership test, bit for bit
      if (R.code == kGradF32) {
        const float lsc = MODE == kPow2 ? 0.f : lg2_approx(R.d2min);
        float w, fac;
        if (kMod) {  // the scale is the query's largest base t
          const float id = rsqrt_approx(d2);
          const float tb = fmaxf(id - inv_r, 0.f);
          if (!(tb > 0.f)) continue;
          w = modified_ratio<MODE>(tb, R.d2min, lsc, pf);
          fac = (id * id) * (id * rcp_approx(tb));  // 1 / (t d^3)
        } else {
          w = grad_weight<MODE>(d2, R.d2min, lsc, hp);
          fac = rcp_approx(d2);  // 1 / d^2
        }
        gz = fmaf(R.c, w, gz);
        const float a = R.c * pf * (v.z - R.z) * w * fac;
        gx = fmaf(a, dx, gx);
        gy = fmaf(a, dy, gy);
      } else {
        const float3 f = kMod ? grad_pair_f64_modified(rec64[t], q.x, q.y, v, p, radius)
                              : grad_pair_f64(rec64[t], q.x, q.y, v, p);
        gz += f.x;
        gx += f.y;
        gy += f.z;
      }
    }
  if (grad_z) grad_z[idx] = gz;
  if (grad_xy) {
    grad_xy[2 * int64_t(idx)] = gx;
    grad_xy[2 * int64_t(idx) + 1] = gy;
  }
}

// ------------------------------------------------------------- k-NN form
//
// One thread per query, in cell order, grows a square of cells around the
// grid cell nearest to it (radius 0, 1, 2, 3, 4, 6, 9, ...: r += max(1, r/2),
// the step halved while the added cells would hold more than 4k points; the
// cells added at each step are walked as row runs) and keeps the k
// smallest keys in a max-heap in shared memory.  A key is the FP32 d^2's
// bits (non-negative, so they order as an unsigned integer) above the data
// index: one 64-bit compare ranks by (d^2, index).  After each step the
// search stops once the k-th key's d^2 is below a lower bound on the d^2 of
// any point not yet seen.  Such a point lies in the grid's box and outside
// the square, beyond one of its sides that still has grid cells; with ax, ay
// the query's distance to the box along each axis and D the distance to
// that side (cell units, each minus a margin mg = (|u| + |v|) 2^-22 + 2^-9
// for the cell-position errors), its true distance is at least
// h sqrt(max(ax, D)^2 + ay^2) (or the y analogue), and its FP32 d^2 at least
// that squared times (1 - 2^-18), minus 2^-126.  The bound is strict, so an
// unseen point can neither beat nor tie the k-th key.

// One warp per block: a block whose slowest query is still searching holds
// only its own warp's heaps in shared memory.
constexpr int kKnnThreads = 32;

__device__ __forceinline__ u64 knn_key(float d2, int idx) {
  return (u64(__float_as_uint(d2)) << 32) | u64(unsigned(idx));
}
__device__ __forceinline__ float key_d2(u64 key) { return __uint_as_float(unsigned(key >> 32)); }
__device__ __forceinline__ int key_index(u64 key) { return int(unsigned(key)); }

// 4-ary max-heap of this thread's keys: slot s at h[s * kKnnThreads]
// (conflict-free); the children of slot a are 4a + 1 .. 4a + 4, so a sift
// is at most 3 levels deep for k <= 64 and each level's loads issue together.
struct KnnHeap {
  u64* h;
  int size = 0;

  __device__ __forceinline__ u64 top() const { return h[0]; }
  __device__ __forceinline__ void push(u64 key) {
    int at = size++;
    while (at > 0) {
      const int parent = (at - 1) >> 2;
      const u64 pk = h[parent * kKnnThreads];
      if (pk >= key) break;
      h[at * kKnnThreads] = pk;
      at = parent;
    }
    h[at * kKnnThreads] = key;
  }
  // Replaces the largest key by a smaller one (keys are distinct).
  __device__ __forceinline__ void replace_top(u64 key, int n) { sift_down(0, key, n); }
  // Puts `key` at slot `at` of the first n slots and sifts it down, the
  // subtree below `at` being a heap already.
  __device__ __forceinline__ void sift_down(int at, u64 key, int n) {
    for (;;) {
      const int c0 = 4 * at + 1;
      if (c0 >= n) break;
      u64 bk = h[c0 * kKnnThreads];
      int big = c0;
#pragma unroll
      for (int c = 1; c < 4; ++c) {
        if (c0 + c < n) {
          const u64 ck = h[(c0 + c) * kKnnThreads];
          if (ck > bk) {
            bk = ck;
            big = c0 + c;
          }
        }
      }
      if (bk <= key) break;
      h[at * kKnnThreads] = bk;
      at = big;
    }
    h[at * kKnnThreads] = key;
  }
  // Floyd's bottom-up construction of a heap over the first n slots.
  __device__ void heapify(int n) {
    for (int a = (n - 2) >> 2; a >= 0; --a) sift_down(a, h[a * kKnnThreads], n);
  }
};

// Writes one query's k-NN result from its heap: Z (the z of the lowest
// coincident index, or Eq. 1 over the selection with compensated FP32 sums,
// or FP64 when those leave FP32's range; NaN when nothing is selected), the
// hit index, the k-th key's d^2 and the neighbour row (key order when
// sort_rows, else heap order).  Shared by both search kernels.
template <int MODE>
__device__ __forceinline__ void knn_write_result(KnnHeap& hp, int best_hit, float qx, float qy,
                                                 int j, const float* __restrict__ data,
                                                 int64_t n, double p, int k,
                                                 float* __restrict__ out,
                                                 int32_t* __restrict__ nbr_out,
                                                 float* __restrict__ kd2_out,
                                                 int32_t* __restrict__ hit_out, bool sort_rows) {
  const int size = hp.size;
  if (kd2_out) kd2_out[j] = size > 0 ? key_d2(hp.top()) : __int_as_float(0x7fc00000);
  float zv = __int_as_float(0x7fc00000);  // NaN: nothing selected
  if (best_hit != INT_MAX) {
    if (dcheck(best_hit >= 0 && best_hit < n, kSiteData)) zv = data[3 * int64_t(best_hit) + 2];
  } else if (size > 0) {
    const float hpw = static_cast<float>(0.5 * p), nhp = -hpw;
    u64 hi = 0, lo = 0;
    for (int s = 0; s < size; ++s) {
      const u64 key = hp.h[s * kKnnThreads];
      const float w = local_weight<MODE>(key_d2(key), hpw, nhp);
      two_sum_acc(hi, lo, pk(w, __fmul_rn(w, data[3 * int64_t(key_index(key)) + 2])));
    }
    float h0, h1, l0, l1;
    upk(hi, h0, h1);
    upk(lo, l0, l1);
    if (h0 >= kTinyPerMember * float(size) && h0 <= FLT_MAX && fabsf(h1) <= FLT_MAX &&
        fabsf(l1) <= FLT_MAX) {
      const float z0 = __fdiv_rn(h1, h0);
      const float res = __fadd_rn(__fmaf_rn(-z0, h0, h1), __fmaf_rn(-z0, l0, l1));
      zv = __fmaf_rn(res, rcp_approx(h0), z0);
    } else {
      // Outside FP32's range: FP64 over the selected points, scaled by
      // d2_min^(p/2).
      double dmin = INFINITY;
      for (int s = 0; s < size; ++s) {
        const float* x = data + 3 * int64_t(key_index(hp.h[s * kKnnThreads]));
        const double ex = double(qx) - x[0], ey = double(qy) - x[1];
        dmin = fmin(dmin, ex * ex + ey * ey);
      }
      double s0 = 0.0, s1 = 0.0;
      for (int s = 0; s < size; ++s) {
        const float* x = data + 3 * int64_t(key_index(hp.h[s * kKnnThreads]));
        const double ex = double(qx) - x[0], ey = double(qy) - x[1];
        const double w = pow(dmin / (ex * ex + ey * ey), 0.5 * p);
        s0 += w;
        s1 += w * double(x[2]);
      }
      zv = static_cast<float>(s1 / s0);
    }
  }
  out[j] = zv;
  if (hit_out) hit_out[j] = best_hit != INT_MAX ? best_hit : -1;
  if (nbr_out) {
    int32_t* row = nbr_out + int64_t(j) * k;
    for (int s = size; s < k; ++s) row[s] = -1;
    if (!sort_rows) {  // the selection in heap order (the gradient needs no order)
      for (int s = 0; s < size; ++s) row[s] = key_index(hp.h[s * kKnnThreads]);
      return;
    }
    // Heap sort: the largest remaining key goes to the end of the row.
    for (int n = size; n > 0; --n) {
      const u64 top = hp.top();
      row[n - 1] = key_index(top);
      const u64 last = hp.h[(n - 1) * kKnnThreads];
      if (n > 1) hp.replace_top(last, n - 1);
    }
  }
}

// At most 64 registers (32 one-warp blocks per SM); left to itself the
// compiler settles on fewer and spills.
template <int MODE>
__global__ void __maxnreg__(64)
    knn_query_kernel(const GridDev* __restrict__ grid, const float4* __restrict__ sorted,
                     const int32_t* __restrict__ starts, const int32_t* __restrict__ base,
                     const int32_t* __restrict__ bpre, const int32_t* __restrict__ sat,
                     const float4* __restrict__ qrec, const float* __restrict__ data, int64_t n,
                     int64_t m,
                     double p, int k, float* __restrict__ out, int32_t* __restrict__ nbr_out,
                     float* __restrict__ kd2_out, int32_t* __restrict__ hit_out,
                     bool sort_rows) {
  extern __shared__ __align__(16) unsigned char knn_smem[];
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= m) return;  // no block-wide barrier in this kernel
  KnnHeap hp;
  hp.h = reinterpret_cast<u64*>(knn_smem) + threadIdx.x;
  const GridDev g = *grid;
  const float4 rq = qrec[t];
  const float qx = rq.x, qy = rq.y;
  const int j = __float_as_int(rq.z);
  if (!dcheck(j >= 0 && j < m, kSiteOutput)) return;
  int best_hit = INT_MAX;
  u64 worst = ~u64(0);  // the heap's largest key once it holds k, else above every key

  auto run = [&](int yy, int xa, int xb) {
    const int a = cell_start(starts, base, yy * g.gx + xa, g.cells);
    const int b = cell_start(starts, base, yy * g.gx + xb + 1, g.cells);
    // Each candidate's record is loaded one iteration ahead, so that its
    // latency overlaps the previous candidate's heap work.
    float4 nv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a < b && dcheck(a >= 0 && a < n, kSiteGather)) nv = sorted[a];
    for (int q = a; q < b; ++q) {
      if (!dcheck(q >= 0 && q < n, kSiteGather)) break;
      const float4 v = nv;
      if (q + 1 < b && dcheck(q + 1 < n, kSiteGather)) nv = sorted[q + 1];
      const float d2 = fp32_d2(qx, qy, v.x, v.y);
      const int idx = __float_as_int(v.w);
      if (d2 == 0.f && v.x == qx && v.y == qy) best_hit = min(best_hit, idx);
      const u64 key = knn_key(d2, idx);
      if (key < worst) {  // worst stays ~0 (all ones) until the heap is full
        if (!dcheck(hp.size <= k && idx >= 0 && idx < n, kSiteHeap)) continue;
        if (hp.size < k) {
          hp.push(key);
          if (hp.size == k) worst = hp.top();
        } else {
          hp.replace_top(key, k);
          worst = hp.top();
        }
      }
    }
  };

  if (finite2(qx, qy)) {
    const float u = cell_pos(qx, g.hx0, g.inv2), v = cell_pos(qy, g.hy0, g.inv2);
    const int cx = clamp_floor(u, 0, g.gx - 1), cy = clamp_floor(v, 0, g.gy - 1);
    const float mg = __fmaf_ru(fabsf(u) + fabsf(v), 0x1p-22f, 0x1p-9f);
    const float ax = fmaxf(0.f, fmaxf(u - float(g.gx), -u) - mg);
    const float ay = fmaxf(0.f, fmaxf(v - float(g.gy), -v) - mg);
    const float hh = g.inv2 > 0.f ? 2.f / g.inv2 : 0.f;
    const float h2 = __fmul_rd(hh, hh) * (1.f - 0x1p-18f);
    const float ih2 = __frcp_ru(h2);  // +inf for the one-cell grid: nothing is clipped
    // Once the heap holds k keys, a cell can only matter if the stop test's
    // lower bound for its points, (gap_x^2 + gap_y^2) h2 - 2^-126 with each
    // gap reduced by mg, is at most the k-th key's d^2: gap_x^2 + gap_y^2 <=
    // reach2() (rounded up; +inf or NaN clips nothing).
    auto reach2 = [&]() {
      return __fmul_ru(__fadd_ru(key_d2(worst), 0x1p-126f), ih2);
    };
    // Narrows a range [lo, hi] to the cells t whose gap from c (reduced by
    // mg) is at most e: t <= c + mg + e and t + 1 >= c - mg - e, rounded
    // outwards.  An empty range is left as it is; otherwise the result lies
    // in [lo, hi] or is empty (lo > hi).  NaN bounds clip nothing.
    auto clip = [&](float c, float e, int& lo, int& hi) {
      if (lo > hi) return;
      const float a = ceilf(__fsub_rd(__fsub_rd(__fsub_rd(c, mg), e), 1.f));
      const float b = floorf(__fadd_ru(__fadd_ru(c, mg), e));
      const int nlo = int(fminf(fmaxf(float(lo), a), float(hi) + 1.f));
      const int nhi = int(fmaxf(fminf(float(hi), b), float(lo) - 1.f));
      lo = nlo;
      hi = nhi;
    };
    // Points in the square of radius rr around (cx, cy), from the table.
    auto square_count = [&](int rr) {
      const int ya = max(0, cy - rr), yb = min(g.gy - 1, cy + rr);
      const int xa = max(0, cx - rr), xb = min(g.gx - 1, cx + rr);
      const int W = g.gx + 1;
      if (!dcheck(ya >= 0 && xa >= 0 && yb < g.gy && xb < g.gx, kSiteTable)) return 0;
      return sat[(yb + 1) * W + xb + 1] - sat[ya * W + xb + 1] - sat[(yb + 1) * W + xa] +
             sat[ya * W + xa];
    };
    int in_square = -1;  // points in the square of radius r, once counted
    // r = -1 stands for the query's own cell; then square r grows to r2.
    for (int r = -1;;) {
      if (r >= 0) {
        const bool open_l = cx - r > 0, open_r = cx + r < g.gx - 1;
        const bool open_b = cy - r > 0, open_t = cy + r < g.gy - 1;
        if (!(open_l || open_r || open_b || open_t)) break;  // the square covers the grid
        if (hp.size == k) {
          float l2 = INFINITY;
          if (open_l) {
            const float dx = fmaxf(ax, fmaxf(0.f, (u - float(cx - r)) - mg));
            l2 = fminf(l2, __fmaf_rd(dx, dx, __fmul_rd(ay, ay)));
          }
          if (open_r) {
            const float dx = fmaxf(ax, fmaxf(0.f, (float(cx + r + 1) - u) - mg));
            l2 = fminf(l2, __fmaf_rd(dx, dx, __fmul_rd(ay, ay)));
          }
          if (open_b) {
            const float dy = fmaxf(ay, fmaxf(0.f, (v - float(cy - r)) - mg));
            l2 = fminf(l2, __fmaf_rd(dy, dy, __fmul_rd(ax, ax)));
          }
          if (open_t) {
            const float dy = fmaxf(ay, fmaxf(0.f, (float(cy + r + 1) - v) - mg));
            l2 = fminf(l2, __fmaf_rd(dy, dy, __fmul_rd(ax, ax)));
          }
          if (key_d2(worst) < __fmul_rd(l2, h2) - 0x1p-126f) break;
        }
      }
      // Grow by max(1, r/2), halved while the band would hold more than 4k
      // points (a step from empty space into a dense cluster stays short).
      // From r = 4 on (steps of 2 or more), the band's count comes from the
      // summed-area table and an empty band is not walked.
      int r2 = r + max(1, r >> 1);
      bool walk = true;
      if (r >= 4) {
        if (in_square < 0) in_square = square_count(r);
        int c2 = square_count(r2);
        while (c2 - in_square > 4 * k && r2 > r + 1) {
          r2 = r + max(1, (r2 - r) >> 1);
          c2 = square_count(r2);
        }
        walk = c2 != in_square;
        in_square = c2;
      }
      // The cells between squares r and r2 in four parts: the side strips of
      // the rows already in the square, then the new rows below and above.
      // One loop walks every part, so the candidate code exists once.
#pragma unroll 1
      for (int part = 0; walk && part < 4; ++part) {
        int ya, yb, xa, xb;
        if (r < 0) {
          if (part > 0) break;
          ya = yb = cy;
          xa = xb = cx;
        } else if (part < 2) {
          ya = max(0, cy - r);
          yb = min(g.gy - 1, cy + r);
          xa = part == 0 ? max(0, cx - r2) : cx + r + 1;
          xb = part == 0 ? cx - r - 1 : min(g.gx - 1, cx + r2);
        } else {
          xa = max(0, cx - r2);
          xb = min(g.gx - 1, cx + r2);
          ya = part == 2 ? max(0, cy - r2) : cy + r + 1;
          yb = part == 2 ? cy - r - 1 : min(g.gy - 1, cy + r2);
        }
        if (xa > xb || ya > yb) continue;  // then 0 <= ya <= yb < gy, 0 <= xa <= xb < gx
        // With a full heap, rows and columns beyond the k-th key's reach are
        // dropped first (the ranges only narrow, or empty).
        if (hp.size == k) {
          const float e = __fsqrt_ru(reach2());
          clip(v, e, ya, yb);
          clip(u, e, xa, xb);
          if (xa > xb || ya > yb) continue;
        }
        // Once the square is 8 cells out, each stretch of 8 rows whose
        // occupancy blocks over xa..xb hold no point is skipped.
        const bool check_blocks = r >= 8;
        for (int y8 = ya; y8 <= yb;) {
          const int y1 = check_blocks ? min(yb, y8 | 7) : yb;
          bool occupied = true;
          if (check_blocks) {
            const int by = y8 >> kBlockShift;
            const int32_t* bp = bpre + by * (kMaxBlocksPerAxis + 1);
            occupied = dcheck(by < kMaxBlocksPerAxis && (xb >> kBlockShift) < kMaxBlocksPerAxis,
                              kSiteBlock) &&
                       bp[(xb >> kBlockShift) + 1] != bp[xa >> kBlockShift];
          }
          for (int yy = y8; occupied && yy <= y1; ++yy) {
            int ra = xa, rb = xb;
            if (hp.size == k) {  // the columns this row's chord reaches
              const float gap = fmaxf(0.f, fmaxf(float(yy) - v, v - float(yy + 1)) - mg);
              const float w2 = reach2(), g2 = __fmul_rd(gap, gap);
              if (g2 > w2) continue;
              clip(u, __fsqrt_ru(__fsub_ru(w2, g2)), ra, rb);
              if (ra > rb) continue;
            }
            run(yy, ra, rb);
          }
          y8 = y1 + 1;
        }
      }
      r = r2;
    }
  }
  knn_write_result<MODE>(hp, best_hit, qx, qy, j, data, n, p, k, out, nbr_out, kd2_out, hit_out,
                         sort_rows);
}

// ------------------------------------------- k-NN, warp-synchronous
//
// The same search as knn_query_kernel, one thread per query, with the 32
// lanes of a warp kept in step so that they diverge far less:
// * every lane grows its square by the same step at the same time (the
//   smallest of the lanes' step choices; a lane whose stop test has held
//   idles until the warp's last lane stops);
// * a band's rows are taken in the same order by every lane (row offsets
//   -r2 .. r2 from the lane's own cell row), each lane listing its
//   non-empty row runs (clipped to its disc) in shared memory first, then
//   walking its listed runs as one flat stream of candidates, so a lane
//   waits only when its whole stream is shorter than another's;
// * keys that beat a lane's k-th key are appended to its k slots while it
//   fills and to a short pending list after that; the warp merges the
//   pending lists into the lanes' heaps together (building each heap, by
//   Floyd's method, once its k slots are full) whenever a lane's list is
//   nearly full and at the end of each step, where the stop test needs the
//   exact k-th key.
// Every cell the single-query search walks is walked here too, or lies
// beyond the lane's k-th key, so the selection is the same: the k smallest
// keys.
// It is an option, not the default: the lanes do keep more in step (16.7
// of 32 threads per instruction against 12.0 at k = 32), but the lockstep
// control costs about as many warp instructions as the divergence it
// removes, the run lists cut the warps an SM holds, and on clustered data
// the lanes of a warp need very different numbers of steps.

constexpr int kSyncRuns = 8;     // row runs a lane lists before walking them
constexpr int kSyncPending = 4;  // keys a lane holds back before the warp merges

// Shared memory of one warp: (k + kSyncPending) key slots and kSyncRuns
// runs per lane, lane-interleaved.
size_t knn_sync_smem_bytes(int k) {
  return size_t(k + kSyncPending) * kKnnThreads * sizeof(u64) +
         size_t(kSyncRuns) * kKnnThreads * sizeof(int2);
}

template <int MODE>
__global__ void __launch_bounds__(kKnnThreads)
    knn_sync_kernel(const GridDev* __restrict__ grid, const float4* __restrict__ sorted,
                    const int32_t* __restrict__ starts, const int32_t* __restrict__ base,
                    const int32_t* __restrict__ bpre, const int32_t* __restrict__ sat,
                    const float4* __restrict__ qrec, const float* __restrict__ data, int64_t n,
                    int64_t m, double p, int k, float* __restrict__ out,
                    int32_t* __restrict__ nbr_out, float* __restrict__ kd2_out,
                    int32_t* __restrict__ hit_out, bool sort_rows) {
  extern __shared__ __align__(16) unsigned char knn_smem[];
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x;
  const int64_t t = int64_t(blockIdx.x) * kKnnThreads + lane;
  KnnHeap hp;
  hp.h = reinterpret_cast<u64*>(knn_smem) + lane;
  int2* runs = reinterpret_cast<int2*>(knn_smem + size_t(k + kSyncPending) * kKnnThreads *
                                                      sizeof(u64)) + lane;
  const GridDev g = *grid;
  float qx = 0.f, qy = 0.f;
  int j = -1;
  if (t < m) {
    const float4 rq = qrec[t];
    qx = rq.x;
    qy = rq.y;
    j = __float_as_int(rq.z);
    if (!dcheck(j >= 0 && j < m, kSiteOutput)) j = -1;
  }
  const bool searching = j >= 0 && finite2(qx, qy);
  int best_hit = INT_MAX;
  // The heap's largest key once it is built, else above every key; zero
  // (nothing is taken) for a lane that does not search.
  u64 worst = searching ? ~u64(0) : u64(0);
  bool heaped = false;  // the k slots are full and form a heap
  int np = 0;           // keys pending after the k slots
  auto flush = [&]() {
    if (!heaped && hp.size == k) {
      hp.heapify(k);
      heaped = true;
      worst = hp.top();
    }
#pragma unroll 1
    for (int i = 0; i < kSyncPending; ++i) {
      if (i < np) {
        const u64 key = hp.h[(k + i) * kKnnThreads];
        if (key < worst) {
          hp.replace_top(key, k);
          worst = hp.top();
        }
      }
    }
    np = 0;
  };
  int nr = 0;  // runs listed
  // Keys one candidate record against the lane's query.
  auto consider = [&](const float4 c) {
    const float d2 = fp32_d2(qx, qy, c.x, c.y);
    const int idx = __float_as_int(c.w);
    if (d2 == 0.f && c.x == qx && c.y == qy) best_hit = min(best_hit, idx);
    const u64 key = knn_key(d2, idx);
    if (key < worst) {  // to the k slots while filling, else pending
      const bool fill = hp.size < k;
      const int slot = fill ? hp.size : k + np;
      if (dcheck(slot < k + kSyncPending && idx >= 0 && idx < n, kSiteHeap)) {
        hp.h[slot * kKnnThreads] = key;
        hp.size += fill;
        np += !fill;
      }
    }
  };
  // Walks the listed runs as one stream, two candidates per lane per pass,
  // both records loaded before either is keyed (a pass adds at most two
  // pending keys, so the warp merges when a lane holds more than
  // kSyncPending - 2).
  auto walk_runs = [&]() {
    int ri = 0, q = 0, b = 0;
    auto take = [&]() {  // the lane's next candidate, or -1
      if (q >= b && ri < nr) {
        const int2 rr = runs[ri * kKnnThreads];
        ++ri;
        q = rr.x;
        b = rr.y;
      }
      return q < b ? q++ : -1;
    };
    for (;;) {
      const int c0 = take(), c1 = take();
      float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
      const bool t0 = c0 >= 0 && dcheck(c0 < n, kSiteGather);
      const bool t1 = c1 >= 0 && dcheck(c1 < n, kSiteGather);
      if (t0) v0 = sorted[c0];
      if (t1) v1 = sorted[c1];
      if (t0) consider(v0);
      if (t1) consider(v1);
      // Merged before the loop can end, so that every lane leaves with at
      // most kSyncPending - 2 keys pending and the next pass has room.
      if (__any_sync(kFull, np > kSyncPending - 2)) flush();
      if (!__any_sync(kFull, q < b || ri < nr)) break;
    }
    nr = 0;
  };

  const float u = searching ? cell_pos(qx, g.hx0, g.inv2) : 0.f;
  const float v = searching ? cell_pos(qy, g.hy0, g.inv2) : 0.f;
  const int cx = clamp_floor(u, 0, g.gx - 1), cy = clamp_floor(v, 0, g.gy - 1);
  const float mg = __fmaf_ru(fabsf(u) + fabsf(v), 0x1p-22f, 0x1p-9f);
  const float ax = fmaxf(0.f, fmaxf(u - float(g.gx), -u) - mg);
  const float ay = fmaxf(0.f, fmaxf(v - float(g.gy), -v) - mg);
  const float hh = g.inv2 > 0.f ? 2.f / g.inv2 : 0.f;
  const float h2 = __fmul_rd(hh, hh) * (1.f - 0x1p-18f);
  const float ih2 = __frcp_ru(h2);
  auto reach2 = [&]() { return __fmul_ru(__fadd_ru(key_d2(worst), 0x1p-126f), ih2); };
  auto clip = [&](float c, float e, int& lo, int& hi) {
    if (lo > hi) return;
    const float a = ceilf(__fsub_rd(__fsub_rd(__fsub_rd(c, mg), e), 1.f));
    const float b = floorf(__fadd_ru(__fadd_ru(c, mg), e));
    const int nlo = int(fminf(fmaxf(float(lo), a), float(hi) + 1.f));
    const int nhi = int(fmaxf(fminf(float(hi), b), float(lo) - 1.f));
    lo = nlo;
    hi = nhi;
  };
  auto square_count = [&](int rr) {
    const int ya = max(0, cy - rr), yb = min(g.gy - 1, cy + rr);
    const int xa = max(0, cx - rr), xb = min(g.gx - 1, cx + rr);
    const int W = g.gx + 1;
    if (!dcheck(ya >= 0 && xa >= 0 && yb < g.gy && xb < g.gx, kSiteTable)) return 0;
    return sat[(yb + 1) * W + xb + 1] - sat[ya * W + xb + 1] - sat[(yb + 1) * W + xa] +
           sat[ya * W + xa];
  };
  // Lists run [xa, xb] of row yy (already clipped) when it holds points.
  auto list_run = [&](int yy, int xa, int xb) {
    if (xa > xb) return;
    const int a = cell_start(starts, base, yy * g.gx + xa, g.cells);
    const int b = cell_start(starts, base, yy * g.gx + xb + 1, g.cells);
    if (a < b && dcheck(nr < kSyncRuns, kSiteTable)) runs[nr++ * kKnnThreads] = make_int2(a, b);
  };

  bool finished = !searching;
  int in_square = -1;  // points in this lane's square of radius r, once counted
  for (int r = -1;;) {
    if (r >= 0) {
      flush();  // the stop test and the clipping use the exact k-th key
      if (!finished) {
        const bool open_l = cx - r > 0, open_r = cx + r < g.gx - 1;
        const bool open_b = cy - r > 0, open_t = cy + r < g.gy - 1;
        if (!(open_l || open_r || open_b || open_t)) {
          finished = true;  // the square covers the grid
        } else if (heaped) {
          float l2 = INFINITY;
          if (open_l) {
            const float dx = fmaxf(ax, fmaxf(0.f, (u - float(cx - r)) - mg));
            l2 = fminf(l2, __fmaf_rd(dx, dx, __fmul_rd(ay, ay)));
          }
          if (open_r) {
            const float dx = fmaxf(ax, fmaxf(0.f, (float(cx + r + 1) - u) - mg));
            l2 = fminf(l2, __fmaf_rd(dx, dx, __fmul_rd(ay, ay)));
          }
          if (open_b) {
            const float dy = fmaxf(ay, fmaxf(0.f, (v - float(cy - r)) - mg));
            l2 = fminf(l2, __fmaf_rd(dy, dy, __fmul_rd(ax, ax)));
          }
          if (open_t) {
            const float dy = fmaxf(ay, fmaxf(0.f, (float(cy + r + 1) - v) - mg));
            l2 = fminf(l2, __fmaf_rd(dy, dy, __fmul_rd(ax, ax)));
          }
          if (key_d2(worst) < __fmul_rd(l2, h2) - 0x1p-126f) finished = true;
        }
      }
      if (__all_sync(kFull, finished)) break;
    }
    // The step: each searching lane chooses as the single-query search does
    // (from r = 4 on, halved while its band would hold more than 4k points,
    // counted from the summed-area table); the warp takes the smallest.
    int r2 = r + max(1, r >> 1);
    bool walk = !finished;
    if (r >= 4) {
      int mine = INT_MAX;
      if (!finished) {
        if (in_square < 0) in_square = square_count(r);
        mine = r2;
        int c2 = square_count(mine);
        while (c2 - in_square > 4 * k && mine > r + 1) {
          mine = r + max(1, (mine - r) >> 1);
          c2 = square_count(mine);
        }
      }
      r2 = __reduce_min_sync(kFull, mine);
      if (!finished) {
        const int c2 = square_count(r2);
        walk = c2 != in_square;  // an empty band is not walked
        in_square = c2;
      }
    }
    if (r < 0) {
      if (walk) list_run(cy, cx, cx);  // the lane's own cell
    } else {
      // Row offsets -r2 .. r2 from the lane's own row, the same for every
      // lane: within r a row holds the band's two side strips, beyond it a
      // whole row of the band.
      const bool check_blocks = r >= 8;
#pragma unroll 1
      for (int s = -r2; s <= r2; ++s) {
        if (__any_sync(kFull, nr > kSyncRuns - 2)) walk_runs();
        const int yy = cy + s;
        if (!walk || yy < 0 || yy >= g.gy) continue;
        int xa = max(0, cx - r2), xb = min(g.gx - 1, cx + r2);
        if (heaped) {  // the columns this row's chord reaches
          const float gap = fmaxf(0.f, fmaxf(float(yy) - v, v - float(yy + 1)) - mg);
          const float w2 = reach2(), g2 = __fmul_rd(gap, gap);
          if (g2 > w2) continue;
          clip(u, __fsqrt_ru(__fsub_ru(w2, g2)), xa, xb);
          if (xa > xb) continue;
        }
        if (check_blocks) {  // the row's stretch of 8 x 8-cell blocks holds no point
          const int by = yy >> kBlockShift;
          const int32_t* bp = bpre + by * (kMaxBlocksPerAxis + 1);
          if (!dcheck(by < kMaxBlocksPerAxis && (xb >> kBlockShift) < kMaxBlocksPerAxis,
                      kSiteBlock) ||
              bp[(xb >> kBlockShift) + 1] == bp[xa >> kBlockShift])
            continue;
        }
        if (s >= -r && s <= r) {
          list_run(yy, xa, min(xb, cx - r - 1));
          list_run(yy, max(xa, cx + r + 1), xb);
        } else {
          list_run(yy, xa, xb);
        }
      }
    }
    walk_runs();
    r = r2;
  }
  flush();
  if (!heaped) hp.heapify(hp.size);  // fewer than k points
  if (j >= 0)
    knn_write_result<MODE>(hp, best_hit, qx, qy, j, data, n, p, k, out, nbr_out, kd2_out,
                           hit_out, sort_rows);
}

// ------------------------------------------------------ k-NN gradients
//
// The k-NN form's gradients hold each query's selection fixed (it is
// piecewise constant in every input): the derivatives of Eq. 1 summed over
// the selected points, as for the radius form.  The search runs first, with
// neighbour lists and hits kept in the workspace; then one thread per query
// (cell order, so neighbouring threads share points) walks its list, left
// in heap order (the search skips the heap sort): one pass finds d2_min and
// the sums of the scaled weights (d2_min / d^2)^(p/2), rescaling them when a
// smaller d^2 appears, a second the gradients.  A selection is not
// bounded by a fixed radius, so the data-side terms (dL/dz, dL/dx, dL/dy)
// are added to a per-point float4 with one 16-byte vector atomic per pair
// (a third of the L2 operations of three scalar ones; their order, and so
// the last bits, can vary between calls), then copied out.

// The FP64 path of one k-NN query: adds its data-side terms, returns
// (dL/dqx, dL/dqy) and its dL/dp share.  Out of line (rare).
struct KnnGradF64 {
  float gqx, gqy;
  double gp;
  double Z, c, dmin;  // what the pair terms are computed from
};
__device__ __noinline__ KnnGradF64 knn_grad_query_f64(const int32_t* __restrict__ row, int cnt,
                                                      const float* __restrict__ data, float qx,
                                                      float qy, double p, float gj,
                                                      float4* __restrict__ acc) {
  double dmin = INFINITY;
  for (int s = 0; s < cnt; ++s) {
    const float* x = data + 3 * int64_t(row[s]);
    const double ex = double(qx) - x[0], ey = double(qy) - x[1];
    dmin = fmin(dmin, ex * ex + ey * ey);
  }
  double s0 = 0.0, s1 = 0.0;
  for (int s = 0; s < cnt; ++s) {
    const float* x = data + 3 * int64_t(row[s]);
    const double ex = double(qx) - x[0], ey = double(qy) - x[1];
    const double w = pow(dmin / (ex * ex + ey * ey), 0.5 * p);
    s0 += w;
    s1 += w * double(x[2]);
  }
  const double Z = s1 / s0, c = double(gj) / s0;
  double ax = 0.0, ay = 0.0, al = 0.0;
  for (int s = 0; s < cnt; ++s) {
    const int64_t i = row[s];
    const float* x = data + 3 * i;
    const double ex = double(qx) - x[0], ey = double(qy) - x[1], e2 = ex * ex + ey * ey;
    const double w = pow(dmin / e2, 0.5 * p);
    const double a = (double(x[2]) - Z) * w;
    ax += a * ex / e2;
    ay += a * ey / e2;
    al += a * log(e2 / dmin);
    if (acc)
      atomicAdd(&acc[i], make_float4(static_cast<float>(c * w), static_cast<float>(c * p * a * ex / e2),
                                     static_cast<float>(c * p * a * ey / e2), 0.f));
  }
  KnnGradF64 r;
  r.gqx = static_cast<float>(-c * p * ax);
  r.gqy = static_cast<float>(-c * p * ay);
  r.gp = -0.5 * c * al;
  r.Z = Z;
  r.c = c;
  r.dmin = dmin;
  return r;
}

// Per-query state of a deterministic k-NN gradient: the data-side pass
// recomputes each (point, query) term from it, point by point.
enum KnnQMode : int { kKnnQNone = 0, kKnnQF32 = 1, kKnnQF64 = 2, kKnnQHit = 3 };
struct KnnQState {
  double Z, c, d2min;  // FP32 path: exact widenings of its float values
  float lmin;          // log2 d2min (general p, FP32 path)
  int mode;            // KnnQMode
};
static_assert(sizeof(KnnQState) == 32, "query state layout");

template <int MODE>
__global__ void __launch_bounds__(kLocalThreads)
    knn_grad_kernel(const float4* __restrict__ qrec, int64_t m, const float* __restrict__ data,
                    int64_t n, const int32_t* __restrict__ nbr, const int32_t* __restrict__ hit,
                    int k, double p, const float* __restrict__ grad_out,
                    float4* __restrict__ acc, float* __restrict__ grad_q,
                    double* __restrict__ grad_p, KnnQState* __restrict__ qstate,
                    double* __restrict__ gp_query) {
  // qstate (deterministic mode): each query's state is recorded for the
  // point-major pass, acc is null, and dL/dp goes per query to gp_query.
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  double gp = 0.0;  // every lane joins the warp sum
  if (t < m) {
    const float4 r = qrec[t];
    const float qx = r.x, qy = r.y;
    const int j = __float_as_int(r.z);
    if (dcheck(j >= 0 && j < m, kSiteOutput)) {
      const float gj = grad_out[j];
      const int32_t* row = nbr + int64_t(j) * k;
      const int h = hit[j];
      int cnt = 0;
      while (cnt < k && row[cnt] >= 0) ++cnt;
      float gqx = 0.f, gqy = 0.f;
      KnnQState qs{0.0, 0.0, 0.0, 0.f, kKnnQNone};
      if (h >= 0) {
        if (acc && dcheck(h < n, kSiteData)) atomicAdd(&acc[h], make_float4(gj, 0.f, 0.f, 0.f));
        qs.mode = kKnnQHit;
      } else if (cnt > 0) {
        const float hp = static_cast<float>(0.5 * p), pf = static_cast<float>(p);
        // One pass: d2_min and the sums with weights scaled by the smallest
        // d^2 so far, rescaled when a smaller one appears (the row is in
        // heap order).
        float d2min = INFINITY, lmin = 0.f, s0 = 0.f, s1 = 0.f;
        for (int s = 0; s < cnt; ++s) {
          const float* x = data + 3 * int64_t(row[s]);
          const float d2 = fp32_d2(qx, qy, x[0], x[1]);
          if (d2 < d2min) {
            const float l = MODE == kPow2 ? 0.f : lg2_approx(d2);
            if (s > 0) {
              const float f = grad_weight<MODE>(d2min, d2, l, hp);  // (d2 / d2min_old)^(p/2)
              s0 *= f;
              s1 *= f;
            }
            d2min = d2;
            lmin = l;
          }
          const float w = grad_weight<MODE>(d2, d2min, lmin, hp);
          s0 += w;
          s1 = fmaf(w, x[2], s1);
        }
        bool f32 = d2min >= 0x1p-100f;
        if (f32) {
          const float Z = s1 / s0, c = gj / s0;
          const float lmin2 = lg2_approx(d2min);
          f32 = isfinite(Z) && isfinite(c);
          if (f32) {
            float ax = 0.f, ay = 0.f, al = 0.f;
            for (int s = 0; s < cnt; ++s) {
              const int64_t i = row[s];
              if (!dcheck(i >= 0 && i < n, kSiteData)) continue;
              const float* x = data + 3 * i;
              const float dx = __fsub_rn(qx, x[0]), dy = __fsub_rn(qy, x[1]);
              const float d2 = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
              const float w = grad_weight<MODE>(d2, d2min, lmin, hp);
              const float a = (x[2] - Z) * w, ar = a * rcp_approx(d2);
              ax = fmaf(ar, dx, ax);
              ay = fmaf(ar, dy, ay);
              al = fmaf(a, lg2_approx(d2) - lmin2, al);
              if (acc) {
                const float b = c * pf * ar;
                atomicAdd(&acc[i], make_float4(c * w, b * dx, b * dy, 0.f));
              }
            }
            gqx = -c * pf * ax;
            gqy = -c * pf * ay;
            const float gpf = (-0.5f * 0.6931471805599453f) * c * al;
            gp = gpf;
            qs = KnnQState{double(Z), double(c), double(d2min), lmin, kKnnQF32};
          }
        }
        if (!f32) {
          const KnnGradF64 r64 =
              knn_grad_query_f64(row, cnt, data, qx, qy, p, gj, acc);
          gqx = r64.gqx;
          gqy = r64.gqy;
          gp = r64.gp;
          qs = KnnQState{r64.Z, r64.c, r64.dmin, 0.f, kKnnQF64};
        }
      }
      if (grad_q) {
        grad_q[2 * int64_t(j)] = gqx;
        grad_q[2 * int64_t(j) + 1] = gqy;
      }
      if (qstate) qstate[j] = qs;
      if (gp_query) gp_query[j] = gp;
    }
  }
  if (grad_p && !gp_query) {
    gp = warp_sum(gp);
    if ((threadIdx.x & 31) == 0 && gp != 0.0) atomicAdd(grad_p, gp);
  }
}

// ----------------------------------------- deterministic k-NN gradients
//
// Point-major data-side terms in a fixed order: every (point, query)
// selection becomes one 64-bit item, the point index above the query index,
// listed query-major; a stable radix sort by point keeps each point's
// queries in increasing order; 8 lanes per point (a whole warp for a point
// with many terms) then recompute its terms from the queries' states and
// sum them lane-strided and by a fixed shuffle tree.
// dL/dp is summed over queries in index order by a fixed two-level tree.
// Nothing depends on the order in which threads or atomics ran, so two calls
// on the same inputs give the same bits.

// Pair (x = j k + s), packed as key << 32 | j: key = the selected point
// (the hit index for slot 0 of a hit query), or n for an empty slot.
__global__ void __launch_bounds__(256)
    knn_pairs_kernel(const int32_t* __restrict__ nbr, const int32_t* __restrict__ hit,
                     const KnnQState* __restrict__ qstate, int64_t m, int k, int64_t n,
                     uint64_t* __restrict__ items) {
  const int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (x >= m * k) return;
  const int64_t j = x / k;
  const int sl = static_cast<int>(x - j * k);
  const int mode = qstate[j].mode;
  int64_t key = n;
  if (mode == kKnnQHit) {
    if (sl == 0 && dcheck(hit[j] >= 0 && hit[j] < n, kSiteData)) key = hit[j];
  } else if (mode == kKnnQF32 || mode == kKnnQF64) {
    const int32_t i = nbr[x];
    if (i >= 0 && dcheck(i < n, kSiteData)) key = i;
  }
  items[x] = (uint64_t(key) << 32) | uint64_t(uint32_t(j));
}

// First and one-past-last position of each point's run of sorted keys (the
// caller zeroes both arrays: a point no query selected has an empty run).
__global__ void __launch_bounds__(256)
    knn_runs_kernel(const uint64_t* __restrict__ items, int64_t count, int64_t n,
                    int32_t* __restrict__ first, int32_t* __restrict__ last) {
  const int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (x >= count) return;
  const uint32_t key = uint32_t(items[x] >> 32);
  if (key >= n) return;
  if (x == 0 || uint32_t(items[x - 1] >> 32) != key) first[key] = static_cast<int32_t>(x);
  if (x == count - 1 || uint32_t(items[x + 1] >> 32) != key)
    last[key] = static_cast<int32_t>(x + 1);
}

// The data-side terms (dL/dz, dL/dx, dL/dy) of point (x0, y0, zi) for the
// query of pair item q, recomputed as the query-major kernel computes them,
// added to (gz, gx, gy).
template <int MODE>
__device__ __forceinline__ void knn_point_term(uint64_t item, const KnnQState* __restrict__ qstate,
                                               const float* __restrict__ queries,
                                               const float* __restrict__ grad_out, float x0,
                                               float y0, float zi, double p, float hp, float pf,
                                               float& gz, float& gx, float& gy) {
  const int64_t j = uint32_t(item);  // the pair's query
  const KnnQState st = qstate[j];
  const float gj = grad_out[j];
  const float qx = queries[2 * j], qy = queries[2 * j + 1];
  if (st.mode == kKnnQHit) {
    gz += gj;
  } else if (st.mode == kKnnQF32) {
    const float Z = static_cast<float>(st.Z), c = static_cast<float>(st.c);
    const float d2min = static_cast<float>(st.d2min);
    const float dx = __fsub_rn(qx, x0), dy = __fsub_rn(qy, y0);
    const float d2 = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
    const float w = grad_weight<MODE>(d2, d2min, st.lmin, hp);
    const float ar = (zi - Z) * w * rcp_approx(d2);
    const float bb = c * pf * ar;
    gz += c * w;
    gx += bb * dx;
    gy += bb * dy;
  } else if (st.mode == kKnnQF64) {
    const double ex = double(qx) - x0, ey = double(qy) - y0, e2 = ex * ex + ey * ey;
    const double w = pow(st.d2min / e2, 0.5 * p);
    const double av = (double(zi) - st.Z) * w;
    gz += static_cast<float>(st.c * w);
    gx += static_cast<float>(st.c * p * av * ex / e2);
    gy += static_cast<float>(st.c * p * av * ey / e2);
  }
}

// A warp takes kPointsPerWarp consecutive data points and sums each one's
// terms in increasing query order: normally kPointLanes lanes per point,
// lane l summing the point's terms l, l + kPointLanes, ... and the lanes'
// sums joined by a fixed shuffle tree (about k terms per point when m = n,
// so a whole warp per point would leave most lanes one term and the warp
// waiting on it); if one of its points has more than kHeavyTerms terms
// (clustered data: a point inside a blob), all 32 lanes take the warp's
// points one after the other the same way.  The choice depends only on the
// counts, so a point's order of summation is the same in every call.
constexpr int kPointLanes = 8;
constexpr int kPointsPerWarp = 32 / kPointLanes;
constexpr int kHeavyTerms = 16 * kPointLanes;
template <int MODE>
__global__ void __launch_bounds__(256)
    knn_point_grad_kernel(const int32_t* __restrict__ first, const int32_t* __restrict__ last,
                          const uint64_t* __restrict__ items, const KnnQState* __restrict__ qstate,
                          const float* __restrict__ queries, const float* __restrict__ data,
                          int64_t n, double p, const float* __restrict__ grad_out,
                          float* __restrict__ grad_z, float* __restrict__ grad_xy) {
  constexpr unsigned kFull = 0xffffffffu;
  const int lane32 = threadIdx.x & 31;
  const int64_t i0 = ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * kPointsPerWarp;
  const int g = lane32 / kPointLanes, lane = lane32 % kPointLanes;
  const int64_t i = i0 + g;
  const bool own = i < n;  // every lane stays for the shuffles
  float x0 = 0.f, y0 = 0.f, zi = 0.f;
  int a = 0, b = 0;
  if (own) {
    x0 = data[3 * i];
    y0 = data[3 * i + 1];
    zi = data[3 * i + 2];
    a = first[i];
    b = last[i];
  }
  const float hp = static_cast<float>(0.5 * p), pf = static_cast<float>(p);
  auto put = [&](int64_t pi, float gz, float gx, float gy) {
    if (grad_z) grad_z[pi] = gz;
    if (grad_xy) reinterpret_cast<float2*>(grad_xy)[pi] = make_float2(gx, gy);
  };
  if (!__any_sync(kFull, b - a > kHeavyTerms)) {
    float gz = 0.f, gx = 0.f, gy = 0.f;
    for (int q = a + lane; q < b; q += kPointLanes)
      knn_point_term<MODE>(items[q], qstate, queries, grad_out, x0, y0, zi, p, hp, pf, gz, gx, gy);
#pragma unroll
    for (int o = kPointLanes / 2; o > 0; o >>= 1) {
      gz += __shfl_xor_sync(kFull, gz, o);
      gx += __shfl_xor_sync(kFull, gx, o);
      gy += __shfl_xor_sync(kFull, gy, o);
    }
    if (own && lane == 0) put(i, gz, gx, gy);
    return;
  }
  for (int h = 0; h < kPointsPerWarp; ++h) {  // the whole warp on each point
    const int src = h * kPointLanes;
    const float hx = __shfl_sync(kFull, x0, src), hy = __shfl_sync(kFull, y0, src);
    const float hz = __shfl_sync(kFull, zi, src);
    const int ha = __shfl_sync(kFull, a, src), hb = __shfl_sync(kFull, b, src);
    float gz = 0.f, gx = 0.f, gy = 0.f;
    for (int q = ha + lane32; q < hb; q += 32)
      knn_point_term<MODE>(items[q], qstate, queries, grad_out, hx, hy, hz, p, hp, pf, gz, gx, gy);
    gz = warp_sum(gz);
    gx = warp_sum(gx);
    gy = warp_sum(gy);
    if (lane32 == 0 && i0 + h < n) put(i0 + h, gz, gx, gy);
  }
}

// Fixed-order sum of v[0 .. count): CTA b sums its contiguous slice (thread
// t takes every 256th value from t, then a fixed shuffle and shared-memory
// tree), then one CTA sums the CTA totals the same way.
constexpr int kDetSumCtas = 256;
__global__ void __launch_bounds__(256)
    fixed_sum_kernel(const double* __restrict__ v, int64_t count, double* __restrict__ out) {
  __shared__ double part[8];
  const int64_t per = (count + gridDim.x - 1) / gridDim.x;
  const int64_t lo = int64_t(blockIdx.x) * per, hi = min(count, lo + per);
  double acc = 0.0;
  for (int64_t x = lo + threadIdx.x; x < hi; x += blockDim.x) acc += v[x];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < 8; ++w) tot += part[w];
    out[blockIdx.x] = tot;
  }
}

// Copies the per-point accumulators out to the caller's gradient arrays.
__global__ void __launch_bounds__(256)
    knn_grad_copy_kernel(const float4* __restrict__ acc, int64_t n, float* __restrict__ grad_z,
                         float* __restrict__ grad_xy) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 v = acc[i];
  if (grad_z) grad_z[i] = v.x;
  if (grad_xy) reinterpret_cast<float2*>(grad_xy)[i] = make_float2(v.y, v.z);
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int scan_tiles_of(int64_t max_cells) {
  return static_cast<int>((max_cells + 1 + kScanTile - 1) / kScanTile);
}

}  // namespace

// At least two data points per cell on average: finer cells cost more row
// lookups per query than the candidates they save.
int64_t local_max_cells(int64_t n) {
  return std::min<int64_t>(int64_t(kMaxCellsPerAxis) * kMaxCellsPerAxis,
                           std::max<int64_t>(1024, n / 2));
}

LocalLayout local_layout(int64_t n, int64_t m, int64_t max_cells) {
  LocalLayout L;
  L.max_cells = max_cells;
  const size_t len = size_t(max_cells + 1 + 3) / 4 * 16;  // whole int4s
  size_t off = 0;
  L.off_grid = off;       off += round_up(sizeof(GridDev), 256);
  L.off_counts_d = off;   off += round_up(len, 256);
  L.off_counts_q = off;   off += round_up(len, 256);
  L.off_starts_d = off;   off += round_up(len, 256);
  L.off_starts_q = off;   off += round_up(len, 256);
  L.off_sums = off;       off += round_up(size_t(2 * scan_tiles_of(max_cells)) * 4, 256);
  L.off_sorted = off;     off += round_up(size_t(n) * 16, 256);
  L.off_qrec = off;       off += round_up(size_t(m) * 16, 256);
  L.off_bpre = off;
  off += round_up(size_t(kMaxBlocksPerAxis) * (kMaxBlocksPerAxis + 1) * 4, 256);
  // (gx + 1)(gy + 1) = cells + gx + gy + 1 entries, cells <= max_cells.
  L.off_sat = off;
  off += round_up(size_t(max_cells + 2 * kMaxCellsPerAxis + 1) * 4, 256);
  L.bytes = off;
  return L;
}

namespace {

// Enqueues the grid build shared by both local forms: bounding box and plan,
// histograms, scans, scatter of data and queries into cell order.
cudaError_t launch_grid_sort(const float* data, int64_t n, const float* queries, int64_t m,
                             double radius, int knn_k, void* workspace, const LocalLayout& L,
                             int sm_count, cudaStream_t s, bool sort_queries = true) {
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  GridDev* grid = reinterpret_cast<GridDev*>(ws + L.off_grid);
  int32_t* counts_d = reinterpret_cast<int32_t*>(ws + L.off_counts_d);
  int32_t* counts_q = reinterpret_cast<int32_t*>(ws + L.off_counts_q);
  int32_t* starts_d = reinterpret_cast<int32_t*>(ws + L.off_starts_d);
  int32_t* starts_q = reinterpret_cast<int32_t*>(ws + L.off_starts_q);
  int32_t* sums = reinterpret_cast<int32_t*>(ws + L.off_sums);
  float4* sorted = reinterpret_cast<float4*>(ws + L.off_sorted);
  float4* qrec = reinterpret_cast<float4*>(ws + L.off_qrec);
  const int max_tiles = scan_tiles_of(L.max_cells);

  cudaError_t e = cudaMemsetAsync(grid, 0xff, sizeof(GridDev), s);
  if (e != cudaSuccess) return e;
  const unsigned bgrid = static_cast<unsigned>(
      std::max<int64_t>(1, std::min<int64_t>(int64_t(sm_count) * 4, (n + 255) / 256)));
  box_plan_kernel<<<bgrid, 256, 0, s>>>(data, n, grid, radius, 1.0 / double(L.max_cells), knn_k);
  const unsigned zgrid = static_cast<unsigned>(
      std::min<int64_t>(int64_t(sm_count) * 8, (L.max_cells + 4 + 255) / 256));
  zero_counts_kernel<<<zgrid, 256, 0, s>>>(grid, counts_d, counts_q);
  // Without the query sort, the queries join none of the three passes and
  // their records are written in the caller's order.
  const int64_t mq = sort_queries ? m : 0;
  const unsigned pgrid = static_cast<unsigned>((n + mq + 255) / 256);
  count_kernel<<<pgrid, 256, 0, s>>>(grid, data, n, queries, mq, counts_d, counts_q);
  scan_kernel<<<dim3(max_tiles, sort_queries ? 2 : 1), kScanBlock, 0, s>>>(
      grid, counts_d, counts_q, starts_d, starts_q, sums, max_tiles, 0);
  scatter_kernel<<<pgrid, 256, 0, s>>>(grid, data, n, queries, mq, starts_d, starts_q, sums,
                                       max_tiles, counts_d, counts_q, sorted, qrec);
  if (!sort_queries && m > 0)
    query_identity_kernel<<<static_cast<unsigned>((m + 255) / 256), 256, 0, s>>>(queries, m, qrec);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_local(const float* data, int64_t n, const float* queries, int64_t m, double p,
                         double radius, float* out, int32_t* count_out, void* workspace,
                         const LocalLayout& L, int sm_count, cudaStream_t s, bool sort_queries,
                         bool modified) {
  cudaError_t e = launch_grid_sort(data, n, queries, m, radius, 0, workspace, L, sm_count, s,
                                   sort_queries);
  if (e != cudaSuccess) return e;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  const GridDev* grid = reinterpret_cast<const GridDev*>(ws + L.off_grid);
  const int32_t* starts_d = reinterpret_cast<const int32_t*>(ws + L.off_starts_d);
  const int32_t* sums = reinterpret_cast<const int32_t*>(ws + L.off_sums);
  const float4* sorted = reinterpret_cast<const float4*>(ws + L.off_sorted);
  const float4* qrec = reinterpret_cast<const float4*>(ws + L.off_qrec);
  const float r2f = static_cast<float>(radius * radius);
  const float r2t = r2f > 0.f ? r2f : 0x1p-149f;
  const unsigned qgrid = static_cast<unsigned>((m + kLocalThreads - 1) / kLocalThreads);
  if (modified) {
    if (p == 2.0)
      local_query_kernel<kPow2, kWeightModified><<<qgrid, kLocalThreads, 0, s>>>(
          grid, sorted, n, starts_d, sums, qrec, m, p, r2f, r2t, out, count_out, radius);
    else
      local_query_kernel<kPowGeneral, kWeightModified><<<qgrid, kLocalThreads, 0, s>>>(
          grid, sorted, n, starts_d, sums, qrec, m, p, r2f, r2t, out, count_out, radius);
  } else if (p == 2.0) {
    local_query_kernel<kPow2><<<qgrid, kLocalThreads, 0, s>>>(
        grid, sorted, n, starts_d, sums, qrec, m, p, r2f, r2t, out, count_out);
  } else {
    local_query_kernel<kPowGeneral><<<qgrid, kLocalThreads, 0, s>>>(
        grid, sorted, n, starts_d, sums, qrec, m, p, r2f, r2t, out, count_out);
  }
  return cudaGetLastError();
}

size_t local_grad_record_bytes(int64_t m) {
  return round_up(size_t(m) * sizeof(LocalGradRec), 256) +
         round_up(size_t(m) * sizeof(LocalGradRec64), 256);
}

cudaError_t launch_local_backward(const float* data, int64_t n, const float* queries, int64_t m,
                                  double p, double radius, const float* grad_out, float* grad_z,
                                  float* grad_xy, float* grad_q, double* grad_p, void* workspace,
                                  const LocalLayout& L, int sm_count, cudaStream_t s,
                                  bool modified) {
  cudaError_t e = launch_grid_sort(data, n, queries, m, radius, 0, workspace, L, sm_count, s);
  if (e != cudaSuccess) return e;
  if (grad_z && (e = cudaMemsetAsync(grad_z, 0, size_t(n) * 4, s)) != cudaSuccess) return e;
  if (grad_xy && (e = cudaMemsetAsync(grad_xy, 0, size_t(n) * 8, s)) != cudaSuccess) return e;
  if (grad_p && (e = cudaMemsetAsync(grad_p, 0, sizeof(double), s)) != cudaSuccess) return e;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  const GridDev* grid = reinterpret_cast<const GridDev*>(ws + L.off_grid);
  const int32_t* starts_d = reinterpret_cast<const int32_t*>(ws + L.off_starts_d);
  const int32_t* starts_q = reinterpret_cast<const int32_t*>(ws + L.off_starts_q);
  const int32_t* sums = reinterpret_cast<const int32_t*>(ws + L.off_sums);
  const int32_t* sums_q = sums + scan_tiles_of(L.max_cells);
  const float4* sorted = reinterpret_cast<const float4*>(ws + L.off_sorted);
  const float4* qrec = reinterpret_cast<const float4*>(ws + L.off_qrec);
  LocalGradRec* rec = reinterpret_cast<LocalGradRec*>(ws + L.bytes);
  LocalGradRec64* rec64 = reinterpret_cast<LocalGradRec64*>(
      ws + L.bytes + round_up(size_t(m) * sizeof(LocalGradRec), 256));
  const float r2f = static_cast<float>(radius * radius);
  const float r2t = r2f > 0.f ? r2f : 0x1p-149f;
  const unsigned qgrid = static_cast<unsigned>((m + kLocalThreads - 1) / kLocalThreads);
  const unsigned dgrid = static_cast<unsigned>((n + kLocalThreads - 1) / kLocalThreads);
  const bool data_side = grad_z || grad_xy;
  auto run = [&](auto mode, auto wmode) {
    constexpr int M = decltype(mode)::value, W = decltype(wmode)::value;
    local_grad_query_kernel<M, W><<<qgrid, kLocalThreads, 0, s>>>(
        grid, sorted, n, starts_d, sums, qrec, m, p, r2f, r2t, grad_out, grad_q, grad_p, rec,
        rec64, radius);
    if (data_side)
      local_grad_data_kernel<M, W><<<dgrid, kLocalThreads, 0, s>>>(
          grid, sorted, n, starts_d, sums, starts_q, sums_q, qrec, m, rec, rec64, p, r2f, grad_z,
          grad_xy, radius);
  };
  using P2 = std::integral_constant<int, kPow2>;
  using PG = std::integral_constant<int, kPowGeneral>;
  using WS = std::integral_constant<int, kWeightShepard>;
  using WM = std::integral_constant<int, kWeightModified>;
  if (modified) {
    if (p == 2.0) run(P2{}, WM{}); else run(PG{}, WM{});
  } else {
    if (p == 2.0) run(P2{}, WS{}); else run(PG{}, WS{});
  }
  return cudaGetLastError();
}

size_t knn_grad_scratch_bytes(int64_t n, int64_t m, int k, bool deterministic) {
  size_t b = round_up(size_t(m) * 4, 256) * 2 + round_up(size_t(m) * size_t(k) * 4, 256) +
             round_up(size_t(n) * 16, 256);
  if (deterministic) {
    const int64_t pairs = m * int64_t(k);
    b += round_up(size_t(pairs) * 8, 256) + radix_sort_scratch_bytes(pairs) +
         2 * round_up(size_t(n) * 4, 256) + round_up(size_t(m) * sizeof(KnnQState), 256) +
         round_up(size_t(m) * 8, 256) + round_up(size_t(kDetSumCtas) * 8, 256);
  }
  return b;
}

namespace {
// The deterministic k-NN gradient after the search (rows sorted by key):
// query-major kernel without atomics (states, dL/dq, per-query dL/dp), the
// pair list, its stable sort by point, the runs, the point-major kernel and
// the fixed-order dL/dp sum.
cudaError_t launch_knn_backward_fixed_order(const float* data, int64_t n, const float* queries,
                                            int64_t m, double p, int k, const float* grad_out,
                                            float* grad_z, float* grad_xy, float* grad_q,
                                            double* grad_p, unsigned char* ws,
                                            const LocalLayout& L, const int32_t* hit,
                                            const int32_t* nbr, cudaStream_t s) {
  const int64_t pairs = m * int64_t(k);
  size_t off = L.bytes + round_up(size_t(m) * 4, 256) * 2 + round_up(size_t(pairs) * 4, 256) +
               round_up(size_t(n) * 16, 256);
  auto take = [&](size_t bytes) {
    unsigned char* ptr = ws + off;
    off += round_up(bytes, 256);
    return ptr;
  };
  uint64_t* items = reinterpret_cast<uint64_t*>(take(size_t(pairs) * 8));
  void* sort_scratch = take(radix_sort_scratch_bytes(pairs));
  int32_t* first = reinterpret_cast<int32_t*>(take(size_t(n) * 4));
  int32_t* last = reinterpret_cast<int32_t*>(take(size_t(n) * 4));
  KnnQState* qstate = reinterpret_cast<KnnQState*>(take(size_t(m) * sizeof(KnnQState)));
  double* gpq = reinterpret_cast<double*>(take(size_t(m) * 8));
  double* gpart = reinterpret_cast<double*>(take(size_t(kDetSumCtas) * 8));

  const float4* qrec = reinterpret_cast<const float4*>(ws + L.off_qrec);
  const unsigned qgrid = static_cast<unsigned>((m + kLocalThreads - 1) / kLocalThreads);
  if (p == 2.0)
    knn_grad_kernel<kPow2><<<qgrid, kLocalThreads, 0, s>>>(qrec, m, data, n, nbr, hit, k, p,
                                                           grad_out, nullptr, grad_q, grad_p,
                                                           qstate, gpq);
  else
    knn_grad_kernel<kPowGeneral><<<qgrid, kLocalThreads, 0, s>>>(qrec, m, data, n, nbr, hit, k,
                                                                 p, grad_out, nullptr, grad_q,
                                                                 grad_p, qstate, gpq);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (grad_p) {
    fixed_sum_kernel<<<kDetSumCtas, 256, 0, s>>>(gpq, m, gpart);
    fixed_sum_kernel<<<1, 256, 0, s>>>(gpart, kDetSumCtas, grad_p);
  }
  if (!grad_z && !grad_xy) return cudaGetLastError();
  knn_pairs_kernel<<<static_cast<unsigned>((pairs + 255) / 256), 256, 0, s>>>(
      nbr, hit, qstate, m, k, n, items);
  int bits = 1;
  while (bits < 32 && (uint64_t(1) << bits) <= uint64_t(n)) ++bits;  // keys in [0, n]
  uint64_t* sorted_items = nullptr;
  if ((e = radix_sort_items(items, pairs, bits, sort_scratch, s, &sorted_items)) != cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(first, 0, size_t(n) * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(last, 0, size_t(n) * 4, s)) != cudaSuccess) return e;
  knn_runs_kernel<<<static_cast<unsigned>((pairs + 255) / 256), 256, 0, s>>>(sorted_items, pairs, n,
                                                                             first, last);
  const unsigned pgrid =
      static_cast<unsigned>(((n + kPointsPerWarp - 1) / kPointsPerWarp * 32 + 255) / 256);
  if (p == 2.0)
    knn_point_grad_kernel<kPow2><<<pgrid, 256, 0, s>>>(first, last, sorted_items, qstate, queries,
                                                       data, n, p, grad_out, grad_z, grad_xy);
  else
    knn_point_grad_kernel<kPowGeneral><<<pgrid, 256, 0, s>>>(first, last, sorted_items, qstate,
                                                             queries, data, n, p, grad_out,
                                                             grad_z, grad_xy);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_knn_backward(const float* data, int64_t n, const float* queries, int64_t m,
                                double p, int k, const float* grad_out, float* grad_z,
                                float* grad_xy, float* grad_q, double* grad_p, void* workspace,
                                const LocalLayout& L, int sm_count, cudaStream_t s,
                                bool sort_queries, bool deterministic, bool warp_search) {
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  float* zbuf = reinterpret_cast<float*>(ws + L.bytes);
  int32_t* hit = reinterpret_cast<int32_t*>(ws + L.bytes + round_up(size_t(m) * 4, 256));
  int32_t* nbr = reinterpret_cast<int32_t*>(ws + L.bytes + 2 * round_up(size_t(m) * 4, 256));
  // Deterministic mode: rows in key order, so each query's own sums run in
  // one fixed order too.
  cudaError_t e = launch_knn(data, n, queries, m, p, k, zbuf, nbr, nullptr, workspace, L, sm_count,
                             s, hit, sort_queries, deterministic, warp_search);
  if (e != cudaSuccess) return e;
  if (deterministic)
    return launch_knn_backward_fixed_order(data, n, queries, m, p, k, grad_out, grad_z, grad_xy,
                                           grad_q, grad_p, ws, L, hit, nbr, s);
  const bool data_side = grad_z || grad_xy;
  float4* acc = data_side ? reinterpret_cast<float4*>(ws + L.bytes + 2 * round_up(size_t(m) * 4, 256) +
                                                      round_up(size_t(m) * size_t(k) * 4, 256))
                          : nullptr;
  if (acc && (e = cudaMemsetAsync(acc, 0, size_t(n) * 16, s)) != cudaSuccess) return e;
  if (grad_p && (e = cudaMemsetAsync(grad_p, 0, sizeof(double), s)) != cudaSuccess) return e;
  const float4* qrec = reinterpret_cast<const float4*>(ws + L.off_qrec);
  const unsigned qgrid = static_cast<unsigned>((m + kLocalThreads - 1) / kLocalThreads);
  if (p == 2.0)
    knn_grad_kernel<kPow2><<<qgrid, kLocalThreads, 0, s>>>(qrec, m, data, n, nbr, hit, k, p,
                                                           grad_out, acc, grad_q, grad_p,
                                                           nullptr, nullptr);
  else
    knn_grad_kernel<kPowGeneral><<<qgrid, kLocalThreads, 0, s>>>(qrec, m, data, n, nbr, hit, k,
                                                                 p, grad_out, acc, grad_q, grad_p,
                                                                 nullptr, nullptr);
  if (acc)
    knn_grad_copy_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(acc, n, grad_z,
                                                                               grad_xy);
  return cudaGetLastError();
}

cudaError_t debug_check_failures(unsigned* sites, bool* enabled) {
#ifdef IDW_DEBUG_CHECKS
  *enabled = true;
  cudaError_t e = cudaMemcpyFromSymbol(sites, g_debug_failures, sizeof(unsigned));
  const unsigned zero = 0;
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_debug_failures, &zero, sizeof(unsigned));
  return e;
#else
  *enabled = false;
  *sites = 0;
  return cudaSuccess;
#endif
}

size_t knn_smem_bytes(int k) { return size_t(k) * kKnnThreads * sizeof(u64); }


cudaError_t launch_knn(const float* data, int64_t n, const float* queries, int64_t m, double p,
                       int k, float* out, int32_t* nbr_out, float* kd2_out, void* workspace,
                       const LocalLayout& L, int sm_count, cudaStream_t s, int32_t* hit_out,
                       bool sort_queries, bool sort_rows, bool warp_search) {
  const size_t smem = warp_search ? knn_sync_smem_bytes(k) : knn_smem_bytes(k);
  cudaError_t e = cudaSuccess;
  if (warp_search) {
    e = cudaFuncSetAttribute(knn_sync_kernel<kPow2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(knn_sync_kernel<kPowGeneral>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  } else {
    e = cudaFuncSetAttribute(knn_query_kernel<kPow2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(knn_query_kernel<kPowGeneral>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  }
  if (e != cudaSuccess) return e;
  e = launch_grid_sort(data, n, queries, m, 0.0, k, workspace, L, sm_count, s, sort_queries);
  if (e != cudaSuccess) return e;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  const GridDev* grid = reinterpret_cast<const GridDev*>(ws + L.off_grid);
  const int32_t* starts_d = reinterpret_cast<const int32_t*>(ws + L.off_starts_d);
  const int32_t* sums = reinterpret_cast<const int32_t*>(ws + L.off_sums);
  const float4* sorted = reinterpret_cast<const float4*>(ws + L.off_sorted);
  const float4* qrec = reinterpret_cast<const float4*>(ws + L.off_qrec);
  int32_t* bpre = reinterpret_cast<int32_t*>(ws + L.off_bpre);
  int32_t* sat = reinterpret_cast<int32_t*>(ws + L.off_sat);
  block_prefix_kernel<<<kMaxBlocksPerAxis, kMaxBlocksPerAxis, 0, s>>>(grid, starts_d, sums, bpre);
  sat_kernel<<<(kMaxCellsPerAxis + 1 + kSatCols - 1) / kSatCols, kSatCols * kSatWarps, 0, s>>>(
      grid, starts_d, sums, sat);
  const unsigned qgrid = static_cast<unsigned>((m + kKnnThreads - 1) / kKnnThreads);
  auto kernel = warp_search ? (p == 2.0 ? knn_sync_kernel<kPow2> : knn_sync_kernel<kPowGeneral>)
                            : (p == 2.0 ? knn_query_kernel<kPow2> : knn_query_kernel<kPowGeneral>);
  kernel<<<qgrid, kKnnThreads, smem, s>>>(grid, sorted, starts_d, sums, bpre, sat, qrec, data, n,
                                          m, p, k, out, nbr_out, kd2_out, hit_out, sort_rows);
  return cudaGetLastError();
}

namespace {

// Copies an index's plan into a query call's scratch with the tickets reset.
// For the radius form (radius > 0) the reach is recomputed for the call's
// radius, which the host has checked is at most the build radius, so rho
// stays below 2 and the coverage argument of the plan still holds.
__global__ void index_prep_kernel(const GridDev* __restrict__ src, GridDev* __restrict__ dst,
                                  double radius) {
  GridDev g = *src;
  g.box_ticket = 0xffffffffu;
  g.scan_ticket = 0xffffffffu;
  if (radius > 0.0 && g.inv2 > 0.f)
    g.rho = __fmaf_ru(__fmul_ru(__double2float_ru(radius), g.inv2), 0.5f + 0x1p-9f, 0x1p-8f);
  *dst = g;
}

// Query side of a call on a prepared index: plan copy, then the counting
// sort of the queries alone (the scan runs its query half only).
cudaError_t launch_query_sort(const GridDev* xgrid, const float* queries, int64_t m, double radius,
                              int64_t max_cells, void* workspace, const QueryLayout& Q,
                              int sm_count, cudaStream_t s, bool sort_queries) {
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  GridDev* grid = reinterpret_cast<GridDev*>(ws + Q.off_grid);
  int32_t* counts = reinterpret_cast<int32_t*>(ws + Q.off_counts);
  int32_t* starts = reinterpret_cast<int32_t*>(ws + Q.off_starts);
  int32_t* sums = reinterpret_cast<int32_t*>(ws + Q.off_sums);
  float4* qrec = reinterpret_cast<float4*>(ws + Q.off_qrec);
  const int max_tiles = scan_tiles_of(max_cells);
  index_prep_kernel<<<1, 1, 0, s>>>(xgrid, grid, radius);
  if (!sort_queries) {
    query_identity_kernel<<<static_cast<unsigned>((m + 255) / 256), 256, 0, s>>>(queries, m, qrec);
    return cudaGetLastError();
  }
  const unsigned zgrid = static_cast<unsigned>(
      std::min<int64_t>(int64_t(sm_count) * 8, (max_cells + 4 + 255) / 256));
  zero_counts_kernel<<<zgrid, 256, 0, s>>>(grid, counts, counts);
  const unsigned qgrid = static_cast<unsigned>((m + 255) / 256);
  count_kernel<<<qgrid, 256, 0, s>>>(grid, nullptr, 0, queries, m, counts, counts);
  scan_kernel<<<dim3(max_tiles, 1), kScanBlock, 0, s>>>(grid, counts, counts, starts, starts, sums,
                                                        max_tiles, 1);
  scatter_kernel<<<qgrid, 256, 0, s>>>(grid, nullptr, 0, queries, m, starts, starts, sums,
                                       max_tiles, counts, counts, nullptr, qrec);
  return cudaGetLastError();
}

}  // namespace

IndexLayout index_layout(int64_t n, bool knn) {
  IndexLayout X;
  X.n = n;
  X.knn = knn;
  X.max_cells = local_max_cells(n);
  const size_t len = size_t(X.max_cells + 1 + 3) / 4 * 16;  // whole int4s
  size_t off = 0;
  X.off_grid = off;    off += round_up(sizeof(GridDev), 256);
  X.off_counts = off;  off += round_up(len, 256);
  X.off_starts = off;  off += round_up(len, 256);
  X.off_sums = off;    off += round_up(size_t(scan_tiles_of(X.max_cells)) * 4, 256);
  X.off_sorted = off;  off += round_up(size_t(n) * 16, 256);
  if (knn) {
    X.off_data = off;  off += round_up(size_t(n) * 12, 256);
    X.off_bpre = off;  off += round_up(size_t(kMaxBlocksPerAxis) * (kMaxBlocksPerAxis + 1) * 4, 256);
    X.off_sat = off;   off += round_up(size_t(X.max_cells + 2 * kMaxCellsPerAxis + 1) * 4, 256);
  }
  X.bytes = off;
  return X;
}

QueryLayout query_layout(int64_t m, int64_t max_cells) {
  QueryLayout Q;
  const size_t len = size_t(max_cells + 1 + 3) / 4 * 16;
  size_t off = 0;
  Q.off_grid = off;    off += round_up(sizeof(GridDev), 256);
  Q.off_counts = off;  off += round_up(len, 256);
  Q.off_starts = off;  off += round_up(len, 256);
  Q.off_sums = off;    off += round_up(size_t(2 * scan_tiles_of(max_cells)) * 4, 256);
  Q.off_qrec = off;    off += round_up(size_t(m) * 16, 256);
  Q.bytes = off;
  return Q;
}

cudaError_t launch_index_build(const float* data, int64_t n, double radius, int knn_k,
                               void* index_mem, const IndexLayout& X, int sm_count,
                               cudaStream_t s) {
  unsigned char* mem = static_cast<unsigned char*>(index_mem);
  GridDev* grid = reinterpret_cast<GridDev*>(mem + X.off_grid);
  int32_t* counts = reinterpret_cast<int32_t*>(mem + X.off_counts);
  int32_t* starts = reinterpret_cast<int32_t*>(mem + X.off_starts);
  int32_t* sums = reinterpret_cast<int32_t*>(mem + X.off_sums);
  float4* sorted = reinterpret_cast<float4*>(mem + X.off_sorted);
  const int max_tiles = scan_tiles_of(X.max_cells);
  cudaError_t e = cudaMemsetAsync(grid, 0xff, sizeof(GridDev), s);
  if (e != cudaSuccess) return e;
  const unsigned bgrid = static_cast<unsigned>(
      std::max<int64_t>(1, std::min<int64_t>(int64_t(sm_count) * 4, (n + 255) / 256)));
  box_plan_kernel<<<bgrid, 256, 0, s>>>(data, n, grid, radius, 1.0 / double(X.max_cells), knn_k);
  const unsigned zgrid = static_cast<unsigned>(
      std::min<int64_t>(int64_t(sm_count) * 8, (X.max_cells + 4 + 255) / 256));
  zero_counts_kernel<<<zgrid, 256, 0, s>>>(grid, counts, counts);
  const unsigned dgrid = static_cast<unsigned>((n + 255) / 256);
  count_kernel<<<dgrid, 256, 0, s>>>(grid, data, n, nullptr, 0, counts, counts);
  scan_kernel<<<dim3(max_tiles, 1), kScanBlock, 0, s>>>(grid, counts, counts, starts, starts, sums,
                                                        max_tiles, 0);
  scatter_kernel<<<dgrid, 256, 0, s>>>(grid, data, n, nullptr, 0, starts, starts, sums, max_tiles,
                                       counts, counts, sorted, nullptr);
  if (X.knn) {
    e = cudaMemcpyAsync(mem + X.off_data, data, size_t(n) * 12, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    int32_t* bpre = reinterpret_cast<int32_t*>(mem + X.off_bpre);
    int32_t* sat = reinterpret_cast<int32_t*>(mem + X.off_sat);
    block_prefix_kernel<<<kMaxBlocksPerAxis, kMaxBlocksPerAxis, 0, s>>>(grid, starts, sums, bpre);
    sat_kernel<<<(kMaxCellsPerAxis + 1 + kSatCols - 1) / kSatCols, kSatCols * kSatWarps, 0, s>>>(
        grid, starts, sums, sat);
  }
  return cudaGetLastError();
}

cudaError_t launch_index_local(const void* index_mem, const IndexLayout& X, const float* queries,
                               int64_t m, double p, double radius, float* out, int32_t* count_out,
                               void* workspace, const QueryLayout& Q, int sm_count,
                               cudaStream_t s, bool sort_queries, bool modified) {
  const unsigned char* mem = static_cast<const unsigned char*>(index_mem);
  const GridDev* xgrid = reinterpret_cast<const GridDev*>(mem + X.off_grid);
  cudaError_t e = launch_query_sort(xgrid, queries, m, radius, X.max_cells, workspace, Q, sm_count,
                                    s, sort_queries);
  if (e != cudaSuccess) return e;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  const GridDev* grid = reinterpret_cast<const GridDev*>(ws + Q.off_grid);
  const float4* qrec = reinterpret_cast<const float4*>(ws + Q.off_qrec);
  const int32_t* starts = reinterpret_cast<const int32_t*>(mem + X.off_starts);
  const int32_t* sums = reinterpret_cast<const int32_t*>(mem + X.off_sums);
  const float4* sorted = reinterpret_cast<const float4*>(mem + X.off_sorted);
  const float r2f = static_cast<float>(radius * radius);
  const float r2t = r2f > 0.f ? r2f : 0x1p-149f;
  const unsigned qgrid = static_cast<unsigned>((m + kLocalThreads - 1) / kLocalThreads);
  if (modified) {
    if (p == 2.0)
      local_query_kernel<kPow2, kWeightModified><<<qgrid, kLocalThreads, 0, s>>>(
          grid, sorted, X.n, starts, sums, qrec, m, p, r2f, r2t, out, count_out, radius);
    else
      local_query_kernel<kPowGeneral, kWeightModified><<<qgrid, kLocalThreads, 0, s>>>(
          grid, sorted, X.n, starts, sums, qrec, m, p, r2f, r2t, out, count_out, radius);
  } else if (p == 2.0) {
    local_query_kernel<kPow2><<<qgrid, kLocalThreads, 0, s>>>(
        grid, sorted, X.n, starts, sums, qrec, m, p, r2f, r2t, out, count_out);
  } else {
    local_query_kernel<kPowGeneral><<<qgrid, kLocalThreads, 0, s>>>(
        grid, sorted, X.n, starts, sums, qrec, m, p, r2f, r2t, out, count_out);
  }
  return cudaGetLastError();
}

cudaError_t launch_index_knn(const void* index_mem, const IndexLayout& X, const float* queries,
                             int64_t m, double p, int k, float* out, int32_t* nbr_out,
                             float* kd2_out, void* workspace, const QueryLayout& Q, int sm_count,
                             cudaStream_t s, bool sort_queries) {
  const size_t smem = knn_smem_bytes(k);
  cudaError_t e = cudaFuncSetAttribute(knn_query_kernel<kPow2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(knn_query_kernel<kPowGeneral>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  const unsigned char* mem = static_cast<const unsigned char*>(index_mem);
  const GridDev* xgrid = reinterpret_cast<const GridDev*>(mem + X.off_grid);
  e = launch_query_sort(xgrid, queries, m, 0.0, X.max_cells, workspace, Q, sm_count, s,
                        sort_queries);
  if (e != cudaSuccess) return e;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  const GridDev* grid = reinterpret_cast<const GridDev*>(ws + Q.off_grid);
  const float4* qrec = reinterpret_cast<const float4*>(ws + Q.off_qrec);
  const int32_t* starts = reinterpret_cast<const int32_t*>(mem + X.off_starts);
  const int32_t* sums = reinterpret_cast<const int32_t*>(mem + X.off_sums);
  const float4* sorted = reinterpret_cast<const float4*>(mem + X.off_sorted);
  const float* data = reinterpret_cast<const float*>(mem + X.off_data);
  const int32_t* bpre = reinterpret_cast<const int32_t*>(mem + X.off_bpre);
  const int32_t* sat = reinterpret_cast<const int32_t*>(mem + X.off_sat);
  const unsigned qgrid = static_cast<unsigned>((m + kKnnThreads - 1) / kKnnThreads);
  if (p == 2.0)
    knn_query_kernel<kPow2><<<qgrid, kKnnThreads, smem, s>>>(
        grid, sorted, starts, sums, bpre, sat, qrec, data, X.n, m, p, k, out, nbr_out, kd2_out,
        nullptr, true);
  else
    knn_query_kernel<kPowGeneral><<<qgrid, kKnnThreads, smem, s>>>(
        grid, sorted, starts, sums, bpre, sat, qrec, data, X.n, m, p, k, out, nbr_out, kd2_out,
        nullptr, true);
  return cudaGetLastError();
}

}  // namespace idw
