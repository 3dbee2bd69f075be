// Slow path for the queries that the fast combine flags: an exact hit
// (d = 0, where Eq. 1 is undefined) or a weight sum outside the fast form's
// range.  One CTA per flagged query, FP64 throughout, on the caller's
// original (unscaled) data.
#pragma once

#include <climits>
#include <cmath>

#include "idw_device.cuh"
#include "idw_internal.h"

namespace idw {

constexpr int kSlowThreads = 256;

template <typename T>
__device__ __forceinline__ T block_reduce(T v, T* scratch, bool is_min) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T other = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_min ? (other < v ? other : v) : v + other;
  }
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (kSlowThreads / 32) ? scratch[lane] : (is_min ? scratch[0] : T(0));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T other = __shfl_xor_sync(0xffffffffu, v, o);
      v = is_min ? (other < v ? other : v) : v + other;
    }
    if (lane == 0) scratch[0] = v;
  }
  __syncthreads();
  const T r = scratch[0];
  __syncthreads();
  return r;
}

// One flagged query j, by the whole CTA:
//  1. the lowest data index i with (x_i, y_i) == (qx, qy) gives Z = z_i;
//  2. otherwise Eq. 1 in FP64 with weights scaled by d2_min^(p/2) (the
//     common factor cancels in the ratio and keeps every weight in (0, 1]).
template <typename T, typename OutT>
__device__ void slow_one_query(const T* __restrict__ data, int64_t n, T qx, T qy, double p,
                               OutT* out_j, double* s0_j, int32_t* hit_j) {
  __shared__ double red_d[kSlowThreads / 32];
  __shared__ long long red_i[kSlowThreads / 32];

  long long best = LLONG_MAX;
  for (int64_t i = threadIdx.x; i < n; i += kSlowThreads) {
    if (data[3 * i] == qx && data[3 * i + 1] == qy) {
      best = i;
      break;
    }
  }
  best = block_reduce<long long>(best, red_i, true);
  if (best != LLONG_MAX) {
    if (threadIdx.x == 0) {
      *out_j = static_cast<OutT>(data[3 * best + 2]);
      if (s0_j) *s0_j = INFINITY;
      if (hit_j) *hit_j = static_cast<int32_t>(best);
    }
    return;
  }

  const double dqx = qx, dqy = qy;
  double dmin = INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += kSlowThreads) {
    const double dx = dqx - double(data[3 * i]), dy = dqy - double(data[3 * i + 1]);
    const double d2 = dx * dx + dy * dy;
    dmin = d2 < dmin ? d2 : dmin;
  }
  dmin = block_reduce<double>(dmin, red_d, true);

  const bool pow2 = (p == 2.0);
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kSlowThreads) {
    const double dx = dqx - double(data[3 * i]), dy = dqy - double(data[3 * i + 1]);
    const double r = dmin / (dx * dx + dy * dy);
    const double w = pow2 ? r : pow(r, 0.5 * p);
    s0 += w;
    s1 += w * double(data[3 * i + 2]);
  }
  s0 = block_reduce<double>(s0, red_d, false);
  s1 = block_reduce<double>(s1, red_d, false);
  if (threadIdx.x == 0) {
    *out_j = static_cast<OutT>(s1 / s0);
    if (s0_j) *s0_j = s0 * pow(dmin, -0.5 * p);
    if (hit_j) *hit_j = kRecomputedF64;
  }
}

// Single problem: list holds query indices.
template <typename T, typename OutT>
__global__ void __launch_bounds__(kSlowThreads)
    slow_path_kernel(const T* __restrict__ data, int64_t n, const T* __restrict__ queries,
                     double p, const Control* __restrict__ ctrl, const int32_t* __restrict__ list,
                     OutT* __restrict__ out, double* __restrict__ s0_out,
                     int32_t* __restrict__ hit_out) {
  const unsigned count = ctrl->flagged;
  for (unsigned f = blockIdx.x; f < count; f += gridDim.x) {
    const int64_t j = list[f];
    slow_one_query<T, OutT>(data, n, queries[2 * j], queries[2 * j + 1], p, &out[j],
                            s0_out ? &s0_out[j] : nullptr, hit_out ? &hit_out[j] : nullptr);
  }
}

}  // namespace idw
