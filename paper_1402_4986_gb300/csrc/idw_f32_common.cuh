// Pieces shared by the FP32 forward and adjoint translation units: the
// per-problem instance table passed by value to the kernels, the coordinate
// range scan, the power-of-two prescaling and the staging of data tiles.
#pragma once

#include <cfloat>
#include <cmath>

#include "idw_device.cuh"
#include "idw_internal.h"

namespace idw {
namespace {

constexpr int kTB32 = kRecordsF32;
constexpr uint32_t kTileBytes32 = static_cast<uint32_t>(kTileBytesF32);

// Staging layouts of a data tile (the layout ablation; 0 is the default):
//   0  duplicated pair records: kTB32 x (x,x,y,y) then kTB32 x (z,z), 24 B/point;
//   1  aligned AoS (the paper's AoaS record): kTB32 x (x,y,z,pad), 16 B/point;
//   2  SoA: kTB32 x x, then kTB32 x y, then kTB32 x z, 12 B/point.
template <int LAYOUT>
__host__ __device__ constexpr uint32_t tile_bytes_of() {
  return LAYOUT == 0 ? 24u * kTB32 : (LAYOUT == 1 ? 16u * kTB32 : 12u * kTB32);
}
static_assert(tile_bytes_of<0>() == kTileBytes32, "default layout");
static_assert(tile_bytes_of<1>() % 16 == 0 && tile_bytes_of<2>() % 16 == 0, "bulk copy sizes");

// Padding records of the p = 2 form sit at (2^63, 2^63): for any query with
// |coordinate| <= 2^10, d^2 = 2^127, whose reciprocal is subnormal and
// flushes to 0, and the shared product overflows to +inf, whose reciprocal
// is 0.  The general form pads at +inf (its log2 is clamped).
constexpr float kPadPow2 = 9.223372036854775808e18f;  // 2^63

struct Instance {
  const float* data;     // n x 3 rows (caller)
  const float* queries;  // m x 2 rows (caller)
  float* out;
  double* s0_out;
  int32_t* hit_out;
  unsigned char* tiles;  // this problem's staged tiles (workspace)
  int64_t unit_base;     // first global work unit
  int64_t record_base;   // first global staged record
  int32_t n, m;
  int32_t data_tiles;
  int32_t qtile_base;    // first global query tile
};
static_assert(sizeof(Instance) == 80, "instance record layout");

template <int CAP>
struct Table {
  int32_t count;
  int32_t pad;
  Instance inst[CAP];
};


// Largest instance index whose `field` <= v (fields ascend with the index).
template <int CAP>
__device__ __forceinline__ int find_unit(const Table<CAP>& t, int64_t v) {
  int lo = 0, hi = t.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.inst[mid].unit_base <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}
template <int CAP>
__device__ __forceinline__ int find_record(const Table<CAP>& t, int64_t v) {
  int lo = 0, hi = t.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.inst[mid].record_base <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}
template <int CAP>
__device__ __forceinline__ int find_qtile(const Table<CAP>& t, int64_t v) {
  int lo = 0, hi = t.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.inst[mid].qtile_base <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Power of two that maps the largest finite |coordinate| into [2^9, 2^10).
__device__ __forceinline__ float scale_from_max(unsigned bits) {
  const float mx = __uint_as_float(bits);
  if (!(mx > 0.f)) return 1.f;
  int e = 0;
  frexpf(mx, &e);  // mx = f 2^e, f in [0.5, 1)
  const int k = max(-100, min(100, 10 - e));
  return ldexpf(1.f, k);
}

__device__ __forceinline__ float mul_ftz(float a, float b) {
  float r;
  asm("mul.rn.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// Largest finite |x|, |y| over each problem's data and queries.
template <int CAP>
__global__ void __launch_bounds__(256) range_kernel(const __grid_constant__ Table<CAP> t,
                                                    unsigned* __restrict__ maxbits) {
  __shared__ float red[8];
  pdl_trigger();
  pdl_wait();
  const Instance& I = t.inst[blockIdx.y];
  float mx = 0.f;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int64_t first = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  for (int64_t i = first; i < I.n; i += stride) {
    const float a = fabsf(I.data[3 * i]), b = fabsf(I.data[3 * i + 1]);
    if (a <= FLT_MAX) mx = fmaxf(mx, a);
    if (b <= FLT_MAX) mx = fmaxf(mx, b);
  }
  for (int64_t i = first; i < I.m; i += stride) {
    const float a = fabsf(I.queries[2 * i]), b = fabsf(I.queries[2 * i + 1]);
    if (a <= FLT_MAX) mx = fmaxf(mx, a);
    if (b <= FLT_MAX) mx = fmaxf(mx, b);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[w]);
    atomicMax(&maxbits[blockIdx.y], __float_as_uint(mx));  // order-preserving for x >= 0
  }
}

// Stages each problem's n x 3 rows into tiles of kTB32 records: kTB32 x (x,x,y,y)
// then kTB32 x (z,z), coordinates scaled by the problem's power of two.
template <int CAP, int MODE, int LAYOUT = 0>
__global__ void __launch_bounds__(256)
    stage_kernel(const __grid_constant__ Table<CAP> t, int64_t total_records,
                 const unsigned* __restrict__ maxbits, float* __restrict__ scales) {
  pdl_trigger();
  pdl_wait();
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= total_records) return;
  const int k = find_record(t, r);
  const Instance& I = t.inst[k];
  const int64_t lr = r - I.record_base;
  const float s = scale_from_max(maxbits[k]);
  if (lr == 0) scales[k] = s;
  const float pad = MODE == kPow2 ? kPadPow2 : INFINITY;
  float x = pad, y = pad, z = 0.f;
  if (lr < I.n) {
    x = I.data[3 * lr] * s;
    y = I.data[3 * lr + 1] * s;
    z = I.data[3 * lr + 2];
  }
  unsigned char* base = I.tiles + (lr / kTB32) * tile_bytes_of<LAYOUT>();
  const int slot = static_cast<int>(lr % kTB32);
  if (LAYOUT == 0) {
    reinterpret_cast<float4*>(base)[slot] = make_float4(x, x, y, y);
    reinterpret_cast<float2*>(base + kTB32 * 16)[slot] = make_float2(z, z);
  } else if (LAYOUT == 1) {
    reinterpret_cast<float4*>(base)[slot] = make_float4(x, y, z, 0.f);
  } else {
    float* f = reinterpret_cast<float*>(base);
    f[slot] = x;
    f[kTB32 + slot] = y;
    f[2 * kTB32 + slot] = z;
  }
}


}  // namespace
}  // namespace idw
