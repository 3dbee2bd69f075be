// FP32-compensated forward pass of global Shepard IDW (Sec. 2.1, Eq. 1).
//
// Pipeline (one call): stage data -> persistent all-pairs sweep -> FP64
// combine -> FP64 slow path for flagged queries.
//
// The sweep is the paper's tiled kernel (Sec. 4.2: a block loads a tile of
// data points into shared memory and every thread sweeps it) rebuilt for
// sm_103a:
//   * each thread holds 2*kQueryPairsF32 queries in registers as pairs, so
//     every FP32 operation is a packed fp32x2 instruction over two queries;
//   * data tiles stream global -> shared by 1-D bulk TMA into a ring of
//     stages guarded by mbarriers (bounded waits), and every warp reads the
//     same record (a broadcast shared load);
//   * the record is staged pre-duplicated as (x,x,y,y)+(z,z) so it feeds the
//     packed instructions with no register moves (the paper's aligned AoS
//     record, Sec. 3.3, widened for pair arithmetic);
//   * w = d^-p without a square root: p = 2 is one MUFU reciprocal of d^2;
//     general p is 2^(-(p/2) log2 d^2) with the product's rounding error
//     recovered by an FMA and applied to first order;
//   * sums run in chunks of kChunkF32 points, and each chunk sum is folded
//     into (hi, lo) pairs by Knuth's TwoSum, so the rounding error does not
//     grow with n;
//   * the (query tile, data tile) work units are split evenly over a grid of
//     co-resident CTAs (stream-K); pieces of a query tile are summed in FP64
//     by the combine, which plays the role of the paper's in-block
//     reduction of the improved CDP kernel (Sec. 3.1).
#include <cmath>

#include "idw_device.cuh"
#include "idw_internal.h"
#include "idw_slowpath.cuh"

namespace idw {
namespace {

constexpr int NT = kThreadsF32;
constexpr int KP = kQueryPairsF32;
constexpr int QT = kQueriesPerCtaF32;
constexpr int TB = kRecordsF32;
constexpr int ST = kStagesF32;
constexpr int CH = kChunkF32;
constexpr uint32_t kTileBytes = static_cast<uint32_t>(kTileBytesF32);
static_assert(kTileBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
static_assert(TB % CH == 0, "chunks tile the data tile");

struct FwdArgs {
  const unsigned char* tiles;  // data_tiles x kTileBytes
  const float* queries;        // m x 2
  int64_t m;
  int64_t data_tiles;
  int64_t units;
  int grid;
  float half_p;
  float neg_half_p;
  float4* partial;  // partial_slots x QT records (S0 hi, S0 lo, S1 hi, S1 lo)
  unsigned* err;
};

// Stages the caller's n x 3 rows into tiles of TB records: TB x (x,x,y,y)
// then TB x (z,z).  Padding records sit at +inf with z = 0, so their weight
// is exactly 0 in both weight forms.
__global__ void stage_f32_kernel(const float* __restrict__ data, int64_t n, int64_t data_tiles,
                                 unsigned char* __restrict__ tiles) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= data_tiles * TB) return;
  const int64_t t = r / TB;
  const int k = static_cast<int>(r % TB);
  float x = INFINITY, y = INFINITY, z = 0.f;
  if (r < n) {
    x = data[3 * r];
    y = data[3 * r + 1];
    z = data[3 * r + 2];
  }
  unsigned char* base = tiles + t * kTileBytes;
  reinterpret_cast<float4*>(base)[k] = make_float4(x, x, y, y);
  reinterpret_cast<float2*>(base + TB * 16)[k] = make_float2(z, z);
}

template <int MODE>
__device__ __forceinline__ u64 weight_pair(u64 d2, u64 half_p2, u64 neg_half_p2) {
  float a, b;
  upk(d2, a, b);
  if (MODE == kPow2) {
    return pk(rcp_approx(a), rcp_approx(b));
  } else {
    // L = log2 d^2, clamped so that +inf (padding) stays finite below.
    const float la = fminf(lg2_approx(a), 1048576.f);
    const float lb = fminf(lg2_approx(b), 1048576.f);
    const u64 L = pk(la, lb);
    const u64 th = mul2(L, neg_half_p2);      // t = -(p/2) L, rounded
    const u64 nth = mul2(L, half_p2);         // -t exactly
    const u64 tl = fma2(L, neg_half_p2, nth); // exact rounding error of t
    float ta, tb;
    upk(th, ta, tb);
    const u64 e = pk(ex2_approx(ta), ex2_approx(tb));
    const u64 c = mul2(tl, pk(0.6931471805599453f, 0.6931471805599453f));
    return fma2(e, c, e);                     // 2^(th + tl) to first order in tl
  }
}

template <int MODE>
__global__ void __launch_bounds__(NT, 2) fwd_f32_kernel(const FwdArgs a) {
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

  int64_t issued = 0;  // meaningful in thread 0 only
  auto issue = [&](int64_t local) {
    const int s = static_cast<int>(local % ST);
    const int64_t dt = (u0 + local) % a.data_tiles;
    bulk_load(smem_u32(smem + s * kTileBytes), a.tiles + dt * kTileBytes, kTileBytes,
              smem_u32(&full_bar[s]));
  };
  if (tid == 0) {
    for (; issued < ST && issued < total; ++issued) issue(issued);
  }

  const u64 hp2 = pk(a.half_p, a.half_p);
  const u64 nhp2 = pk(a.neg_half_p, a.neg_half_p);
  int64_t i = 0;
  bool aborted = false;
  while (i < total) {
    const int64_t qt = (u0 + i) / a.data_tiles;
    const int64_t seg_end = min(total, (qt + 1) * a.data_tiles - u0);

    u64 QX[KP], QY[KP], H0[KP], L0[KP], H1[KP], L1[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const int64_t ja = qt * QT + (2 * k) * NT + tid;
      const int64_t jb = ja + NT;
      const float xa = ja < a.m ? a.queries[2 * ja] : 0.f;
      const float ya = ja < a.m ? a.queries[2 * ja + 1] : 0.f;
      const float xb = jb < a.m ? a.queries[2 * jb] : 0.f;
      const float yb = jb < a.m ? a.queries[2 * jb + 1] : 0.f;
      QX[k] = pk(xa, xb);
      QY[k] = pk(ya, yb);
      H0[k] = L0[k] = H1[k] = L1[k] = 0ull;
    }

    for (; i < seg_end; ++i) {
      const int s = static_cast<int>(i % ST);
      const uint32_t parity = static_cast<uint32_t>((i / ST) & 1);
      const bool ok = mbar_wait_bounded(smem_u32(&full_bar[s]), parity, a.err);
      if (ok) {
        const ulonglong2* XY = reinterpret_cast<const ulonglong2*>(smem + s * kTileBytes);
        const u64* ZZ = reinterpret_cast<const u64*>(smem + s * kTileBytes + TB * 16);
#pragma unroll 1
        for (int c = 0; c < TB; c += CH) {
          u64 C0[KP], C1[KP];
#pragma unroll
          for (int r = 0; r < CH; ++r) {
            const ulonglong2 xy = XY[c + r];
            const u64 zz = ZZ[c + r];
#pragma unroll
            for (int k = 0; k < KP; ++k) {
              const u64 dx = sub2f(QX[k], xy.x);
              const u64 dy = sub2f(QY[k], xy.y);
              const u64 d2 = fma2f(dy, dy, mul2f(dx, dx));
              const u64 w = weight_pair<MODE>(d2, hp2, nhp2);
              if (r == 0) {
                C0[k] = w;
                C1[k] = mul2(w, zz);
              } else {
                C0[k] = add2(C0[k], w);
                C1[k] = fma2(w, zz, C1[k]);
              }
            }
          }
#pragma unroll
          for (int k = 0; k < KP; ++k) {
            two_sum_acc(H0[k], L0[k], C0[k]);
            two_sum_acc(H1[k], L1[k], C1[k]);
          }
        }
      }
      // Every thread is done with stage s (and agrees on whether to stop).
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

    float4* P = a.partial + (qt + g) * QT;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      float h0a, h0b, l0a, l0b, h1a, h1b, l1a, l1b;
      upk(H0[k], h0a, h0b);
      upk(L0[k], l0a, l0b);
      upk(H1[k], h1a, h1b);
      upk(L1[k], l1a, l1b);
      P[(2 * k) * NT + tid] = make_float4(h0a, l0a, h1a, l1a);
      P[(2 * k + 1) * NT + tid] = make_float4(h0b, l0b, h1b, l1b);
    }
  }

  if (aborted && tid == 0) {
    // Let every copy still in flight land before the CTA's shared memory
    // is released (each wait is bounded as well).
    for (int64_t k = i; k < issued; ++k)
      mbar_wait_bounded(smem_u32(&full_bar[k % ST]), static_cast<uint32_t>((k / ST) & 1), a.err);
  }
}

// FP64 combine of the pieces of each query: Z = S1 / S0, or a flag that
// routes the query to the slow path (exact hit or FP32 range exceeded).
__global__ void combine_f32_kernel(const float4* __restrict__ partial, int64_t m,
                                   int64_t data_tiles, int64_t units, int grid, double tiny,
                                   float* __restrict__ out, double* __restrict__ s0_out,
                                   int32_t* __restrict__ hit_out, Control* __restrict__ ctrl,
                                   int32_t* __restrict__ list) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int64_t qt = j / QT, lq = j % QT;
  const int64_t g0 = cta_of_unit(qt * data_tiles, units, grid);
  const int64_t g1 = cta_of_unit((qt + 1) * data_tiles - 1, units, grid);
  double s0 = 0.0, s1 = 0.0;
  for (int64_t g = g0; g <= g1; ++g) {
    const float4 v = partial[(qt + g) * QT + lq];
    s0 += double(v.x) + double(v.y);
    s1 += double(v.z) + double(v.w);
  }
  if (!(s0 > tiny) || !isfinite(s0) || !isfinite(s1)) {
    const unsigned slot = atomicAdd(&ctrl->flagged, 1u);
    list[slot] = static_cast<int32_t>(j);
    return;
  }
  out[j] = static_cast<float>(s1 / s0);
  if (s0_out) s0_out[j] = s0;
  if (hit_out) hit_out[j] = kNoHit;
}

template <int MODE>
cudaError_t launch_sweep(const FwdArgs& a, cudaStream_t stream) {
  const size_t smem = size_t(ST) * kTileBytes;
  fwd_f32_kernel<MODE><<<a.grid, NT, smem, stream>>>(a);
  return cudaGetLastError();
}

// One thread waits, with the sweep kernels' bounded wait, on a barrier whose
// phase nothing completes; it gives up and records kErrWaitTimeout.
__global__ void bounded_wait_selftest_kernel(unsigned* err) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    fence_barrier_init();
    mbar_wait_bounded(smem_u32(&bar), 0, err);
  }
}

}  // namespace

cudaError_t launch_bounded_wait_selftest(Control* ctrl, cudaStream_t stream) {
  bounded_wait_selftest_kernel<<<1, 32, 0, stream>>>(&ctrl->error);
  return cudaGetLastError();
}

int occupancy_forward_f32(bool general_p) {
  int blocks = 0;
  const size_t smem = size_t(ST) * kTileBytes;
  if (general_p)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fwd_f32_kernel<kPowGeneral>, NT, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fwd_f32_kernel<kPow2>, NT, smem);
  return blocks > 0 ? blocks : 1;
}

cudaError_t launch_forward_f32(const F32Problem& pb, const Plan& plan, void* workspace,
                               Control* ctrl, int sm_count, const SweepEvents* ev,
                               cudaStream_t stream) {
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  unsigned char* tiles = ws;
  float4* partial = reinterpret_cast<float4*>(ws + plan.staged_bytes);
  int32_t* list = reinterpret_cast<int32_t*>(ws + plan.staged_bytes + plan.partial_bytes);

  const int64_t staged = plan.data_tiles * TB;
  stage_f32_kernel<<<static_cast<unsigned>((staged + 255) / 256), 256, 0, stream>>>(
      pb.data, pb.n, plan.data_tiles, tiles);
  cudaError_t e = cudaMemsetAsync(&ctrl->flagged, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;

  FwdArgs a;
  a.tiles = tiles;
  a.queries = pb.queries;
  a.m = pb.m;
  a.data_tiles = plan.data_tiles;
  a.units = plan.units;
  a.grid = plan.grid;
  a.half_p = static_cast<float>(0.5 * pb.p);
  a.neg_half_p = -a.half_p;
  a.partial = partial;
  a.err = &ctrl->error;
  if (ev && (e = cudaEventRecord(ev->start, stream)) != cudaSuccess) return e;
  e = (pb.p == 2.0) ? launch_sweep<kPow2>(a, stream) : launch_sweep<kPowGeneral>(a, stream);
  if (e != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev->stop, stream)) != cudaSuccess) return e;

  combine_f32_kernel<<<static_cast<unsigned>((pb.m + 255) / 256), 256, 0, stream>>>(
      partial, pb.m, plan.data_tiles, plan.units, plan.grid, kTinySumPerPoint * double(pb.n),
      pb.out, pb.s0_out, pb.hit_out, ctrl, list);
  slow_path_kernel<float, float><<<2 * sm_count, kSlowThreads, 0, stream>>>(
      pb.data, pb.n, pb.queries, pb.p, ctrl, list, pb.out, pb.s0_out, pb.hit_out);
  return cudaGetLastError();
}

}  // namespace idw
