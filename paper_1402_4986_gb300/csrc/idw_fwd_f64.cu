// Plain FP64 forward pass of global Shepard IDW (Sec. 2.1, Eq. 1): the
// comparison form.  Same tiling and stream-K split as the FP32 form, but
// every operation is plain double precision: d^2 by DFMA, w = 1/d^2 (p = 2)
// or pow(d^2, -p/2) through the compiler's own division and pow, and plain
// running sums per thread.  Data tiles are staged in the paper's Hybrid
// layout (Sec. 3.5) by default, an array of (x, y) pairs beside an array of
// z, or in aligned (x, y, z, pad) records or plain SoA for the layout
// ablation; the arithmetic, and so the result, is the same in every layout.
#include <cmath>

#include "idw_device.cuh"
#include "idw_f64_layout.h"
#include "idw_internal.h"
#include "idw_slowpath.cuh"

namespace idw {
namespace {

constexpr int NT = kThreadsF64;
constexpr int QP = kQueriesF64;
constexpr int QT = kQueriesPerCtaF64;
constexpr int TB = kRecordsF64;
constexpr int ST = kStagesF64;
template <int LAYOUT>
__host__ __device__ constexpr uint32_t tile_bytes() {
  return LAYOUT == kF64Aoas ? uint32_t(TB) * 32u : static_cast<uint32_t>(kTileBytesF64);
}
static_assert(tile_bytes<kF64Hybrid>() % 16 == 0 && tile_bytes<kF64Aoas>() % 16 == 0,
              "bulk copies move multiples of 16 bytes");

// Record r of a staged tile.
template <int LAYOUT>
__device__ __forceinline__ void tile_record(const unsigned char* tile, int r, double& x, double& y,
                                            double& z) {
  if (LAYOUT == kF64Aoas) {
    const double4 v = reinterpret_cast<const double4*>(tile)[r];
    x = v.x;
    y = v.y;
    z = v.z;
  } else if (LAYOUT == kF64Soa) {
    const double* a = reinterpret_cast<const double*>(tile);
    x = a[r];
    y = a[TB + r];
    z = a[2 * TB + r];
  } else {
    const double2 xy = reinterpret_cast<const double2*>(tile)[r];
    x = xy.x;
    y = xy.y;
    z = reinterpret_cast<const double*>(tile + TB * 16)[r];
  }
}

struct FwdArgs {
  const unsigned char* tiles;
  const double* queries;
  int64_t m;
  int64_t data_tiles;
  int64_t units;
  int grid;
  double neg_half_p;
  double2* partial;  // partial_slots x QT (S0, S1)
  unsigned* err;
};

template <int LAYOUT>
__global__ void stage_f64_kernel(const double* __restrict__ data, int64_t n, int64_t data_tiles,
                                 unsigned char* __restrict__ tiles) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= data_tiles * TB) return;
  const int64_t t = r / TB;
  const int k = static_cast<int>(r % TB);
  double x = INFINITY, y = INFINITY, z = 0.0;
  if (r < n) {
    x = data[3 * r];
    y = data[3 * r + 1];
    z = data[3 * r + 2];
  }
  unsigned char* base = tiles + t * tile_bytes<LAYOUT>();
  if (LAYOUT == kF64Aoas) {
    reinterpret_cast<double4*>(base)[k] = make_double4(x, y, z, 0.0);
  } else if (LAYOUT == kF64Soa) {
    double* a = reinterpret_cast<double*>(base);
    a[k] = x;
    a[TB + k] = y;
    a[2 * TB + k] = z;
  } else {
    reinterpret_cast<double2*>(base)[k] = make_double2(x, y);
    reinterpret_cast<double*>(base + TB * 16)[k] = z;
  }
}

template <int MODE, int LAYOUT>
__global__ void __launch_bounds__(NT) fwd_f64_kernel(const FwdArgs a) {
  constexpr uint32_t kTileBytes = tile_bytes<LAYOUT>();
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long full_bar[ST];

  const int tid = threadIdx.x;
  const int64_t g = blockIdx.x;
  const int64_t u0 = unit_begin(g, a.units, a.grid);
  const int64_t total = unit_begin(g + 1, a.units, a.grid) - u0;
  if (total <= 0) return;

  if (tid == 0) {
    for (int s = 0; s < ST; ++s) mbar_init(smem_u32(&full_bar[s]), 1);
    fence_barrier_init();
  }
  __syncthreads();

  int64_t issued = 0;
  auto issue = [&](int64_t local) {
    const int s = static_cast<int>(local % ST);
    const int64_t dt = (u0 + local) % a.data_tiles;
    bulk_load(smem_u32(smem + s * kTileBytes), a.tiles + dt * kTileBytes, kTileBytes,
              smem_u32(&full_bar[s]));
  };
  if (tid == 0) {
    for (; issued < ST && issued < total; ++issued) issue(issued);
  }

  int64_t i = 0;
  bool aborted = false;
  while (i < total) {
    const int64_t qt = (u0 + i) / a.data_tiles;
    const int64_t seg_end = min(total, (qt + 1) * a.data_tiles - u0);
    double qx[QP], qy[QP], s0[QP], s1[QP];
#pragma unroll
    for (int k = 0; k < QP; ++k) {
      const int64_t j = qt * QT + k * NT + tid;
      qx[k] = j < a.m ? a.queries[2 * j] : 0.0;
      qy[k] = j < a.m ? a.queries[2 * j + 1] : 0.0;
      s0[k] = 0.0;
      s1[k] = 0.0;
    }
    for (; i < seg_end; ++i) {
      const int s = static_cast<int>(i % ST);
      const bool ok =
          mbar_wait_bounded(smem_u32(&full_bar[s]), static_cast<uint32_t>((i / ST) & 1), a.err);
      if (ok) {
        const unsigned char* tile = smem + s * kTileBytes;
#pragma unroll 4
        for (int r = 0; r < TB; ++r) {
          double x, y, z;
          tile_record<LAYOUT>(tile, r, x, y, z);
#pragma unroll
          for (int k = 0; k < QP; ++k) {
            const double dx = qx[k] - x;
            const double dy = qy[k] - y;
            const double d2 = fma(dy, dy, dx * dx);
            const double w = (MODE == kPow2) ? 1.0 / d2 : pow(d2, a.neg_half_p);
            s0[k] += w;
            s1[k] = fma(w, z, s1[k]);
          }
        }
      }
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      if (tid == 0 && issued < total) {
        issue(issued);
        ++issued;
      }
    }
    if (aborted) break;
    double2* P = a.partial + (qt + g) * QT;
#pragma unroll
    for (int k = 0; k < QP; ++k) P[k * NT + tid] = make_double2(s0[k], s1[k]);
  }
  if (aborted && tid == 0) {
    for (int64_t k = i; k < issued; ++k)
      mbar_wait_bounded(smem_u32(&full_bar[k % ST]), static_cast<uint32_t>((k / ST) & 1), a.err);
  }
}

__global__ void combine_f64_kernel(const double2* __restrict__ partial, int64_t m,
                                   int64_t data_tiles, int64_t units, int grid,
                                   double* __restrict__ out, double* __restrict__ s0_out,
                                   int32_t* __restrict__ hit_out, Control* __restrict__ ctrl,
                                   int32_t* __restrict__ list) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int64_t qt = j / QT, lq = j % QT;
  const int64_t g0 = cta_of_unit(qt * data_tiles, units, grid);
  const int64_t g1 = cta_of_unit((qt + 1) * data_tiles - 1, units, grid);
  double s0 = 0.0, s1 = 0.0;
  for (int64_t g = g0; g <= g1; ++g) {
    const double2 v = partial[(qt + g) * QT + lq];
    s0 += v.x;
    s1 += v.y;
  }
  if (!(s0 > 0.0) || !isfinite(s0) || !isfinite(s1)) {
    const unsigned slot = atomicAdd(&ctrl->flagged, 1u);
    list[slot] = static_cast<int32_t>(j);
    return;
  }
  out[j] = s1 / s0;
  if (s0_out) s0_out[j] = s0;
  if (hit_out) hit_out[j] = kNoHit;
}

}  // namespace

namespace {

template <int LAYOUT>
int occupancy_layout() {
  int blocks = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fwd_f64_kernel<kPow2, LAYOUT>, NT,
                                                size_t(ST) * tile_bytes<LAYOUT>());
  return blocks > 0 ? blocks : 1;
}

template <int LAYOUT>
cudaError_t launch_layout(const F64Problem& pb, const Plan& plan, void* workspace, Control* ctrl,
                          int sm_count, const SweepEvents* ev, cudaStream_t stream) {
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  double2* partial = reinterpret_cast<double2*>(ws + plan.staged_bytes);
  int32_t* list = reinterpret_cast<int32_t*>(ws + plan.staged_bytes + plan.partial_bytes);
  const int64_t staged = plan.data_tiles * TB;
  stage_f64_kernel<LAYOUT><<<static_cast<unsigned>((staged + 255) / 256), 256, 0, stream>>>(
      pb.data, pb.n, plan.data_tiles, ws);
  cudaError_t e = cudaMemsetAsync(&ctrl->flagged, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  FwdArgs a;
  a.tiles = ws;
  a.queries = pb.queries;
  a.m = pb.m;
  a.data_tiles = plan.data_tiles;
  a.units = plan.units;
  a.grid = plan.grid;
  a.neg_half_p = -0.5 * pb.p;
  a.partial = partial;
  a.err = &ctrl->error;
  const size_t smem = size_t(ST) * tile_bytes<LAYOUT>();
  if (ev && (e = cudaEventRecord(ev->start, stream)) != cudaSuccess) return e;
  if (pb.p == 2.0)
    fwd_f64_kernel<kPow2, LAYOUT><<<plan.grid, NT, smem, stream>>>(a);
  else
    fwd_f64_kernel<kPowGeneral, LAYOUT><<<plan.grid, NT, smem, stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev->stop, stream)) != cudaSuccess) return e;
  combine_f64_kernel<<<static_cast<unsigned>((pb.m + 255) / 256), 256, 0, stream>>>(
      partial, pb.m, plan.data_tiles, plan.units, plan.grid, pb.out, pb.s0_out, pb.hit_out, ctrl,
      list);
  slow_path_kernel<double, double><<<2 * sm_count, kSlowThreads, 0, stream>>>(
      pb.data, pb.n, pb.queries, pb.p, ctrl, list, pb.out, pb.s0_out, pb.hit_out);
  return cudaGetLastError();
}

}  // namespace

size_t f64_tile_bytes(int layout) {
  return layout == kF64Aoas ? tile_bytes<kF64Aoas>() : tile_bytes<kF64Hybrid>();
}

int occupancy_forward_f64_layout(int layout) {
  switch (layout) {
    case kF64Aoas: return occupancy_layout<kF64Aoas>();
    case kF64Soa: return occupancy_layout<kF64Soa>();
    default: return occupancy_layout<kF64Hybrid>();
  }
}

int occupancy_forward_f64() { return occupancy_forward_f64_layout(kF64Hybrid); }

cudaError_t launch_forward_f64_layout(const F64Problem& pb, const Plan& plan, int layout,
                                      void* workspace, Control* ctrl, int sm_count,
                                      const SweepEvents* ev, cudaStream_t stream) {
  switch (layout) {
    case kF64Aoas: return launch_layout<kF64Aoas>(pb, plan, workspace, ctrl, sm_count, ev, stream);
    case kF64Soa: return launch_layout<kF64Soa>(pb, plan, workspace, ctrl, sm_count, ev, stream);
    default: return launch_layout<kF64Hybrid>(pb, plan, workspace, ctrl, sm_count, ev, stream);
  }
}

cudaError_t launch_forward_f64(const F64Problem& pb, const Plan& plan, void* workspace,
                               Control* ctrl, int sm_count, const SweepEvents* ev,
                               cudaStream_t stream) {
  return launch_forward_f64_layout(pb, plan, kF64Hybrid, workspace, ctrl, sm_count, ev, stream);
}

}  // namespace idw
