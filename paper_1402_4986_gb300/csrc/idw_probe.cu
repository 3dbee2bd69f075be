// Pipe-rate probe: issue rate of the arithmetic the forward pass uses
// (FFMA, packed FFMA2, MUFU rcp / lg2 / ex2, DFMA), in operations per SM
// per clock.  Each CTA times its own loop with the SM's clock counter and
// reports its SM id; the host sums operations per SM and divides by the
// span of that SM's clock readings, so the result does not depend on the
// clock speed.  These rates are the denominators of the pipe roofline.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <vector>

#include "idw_device.cuh"
#include "idw_internal.h"

namespace idw {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kProbeIters = 8192;  // long enough that launch skew is noise
constexpr int kChains = 8;
constexpr int kRounds = 16;        // rounds per loop trip: loop overhead ~2%

enum ProbeOp : int { kOpFfma = 0, kOpFfma2, kOpRcp, kOpLg2, kOpEx2, kOpDfma, kNumOps };

struct ProbeOut {
  unsigned long long start, stop;
  unsigned smid;
  unsigned pad;
};

__device__ __forceinline__ unsigned smid() {
  unsigned s;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
  return s;
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) probe_kernel(float seed, ProbeOut* out,
                                                              float* sink) {
  float v[kChains];
  double dv[kChains];
  u64 pv[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    v[c] = seed + 0.01f * (threadIdx.x + c);
    dv[c] = v[c];
    pv[c] = pk(v[c], v[c] + 1.f);
  }
  const u64 a2 = pk(0.999f, 0.998f), b2 = pk(0.001f, 0.002f);
  __syncthreads();
  const unsigned long long t0 = clock64();
#pragma unroll 1
  for (int it = 0; it < kProbeIters; it += kRounds) {
#pragma unroll
    for (int c = 0; c < kRounds * kChains; ++c) {
      const int k = c % kChains;
      if (OP == kOpFfma) v[k] = fmaf(v[k], 0.999f, 0.001f);
      if (OP == kOpFfma2) pv[k] = fma2(pv[k], a2, b2);
      if (OP == kOpRcp) v[k] = rcp_approx(v[k]) + 0.5f;  // fixed point 1.28
      if (OP == kOpLg2) v[k] = lg2_approx(v[k]) + 2.f;   // fixed point 4
      if (OP == kOpEx2) v[k] = ex2_approx(v[k]) * -0.5f; // bounded orbit
      if (OP == kOpDfma) dv[k] = fma(dv[k], 0.999, 0.001);
    }
  }
  __syncthreads();
  const unsigned long long t1 = clock64();
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    float lo, hi;
    upk(pv[c], lo, hi);
    acc += v[c] + float(dv[c]) + lo + hi;
  }
  if (acc == 12345.678f) sink[threadIdx.x] = acc;  // keeps the loops live
  if (threadIdx.x == 0) {
    out[blockIdx.x].start = t0;
    out[blockIdx.x].stop = t1;
    out[blockIdx.x].smid = smid();
  }
}

template <int OP>
cudaError_t run_probe(int sm_count, int blocks_per_sm, double* rate) {
  const int grid = sm_count * blocks_per_sm;
  ProbeOut* d_out = nullptr;
  float* d_sink = nullptr;
  cudaError_t e = cudaMalloc(&d_out, sizeof(ProbeOut) * grid);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&d_sink, sizeof(float) * kProbeThreads);
  if (e != cudaSuccess) {
    cudaFree(d_out);
    return e;
  }
  probe_kernel<OP><<<grid, kProbeThreads>>>(0.5f, d_out, d_sink);  // warm-up
  probe_kernel<OP><<<grid, kProbeThreads>>>(0.5f, d_out, d_sink);
  e = cudaDeviceSynchronize();
  std::vector<ProbeOut> h(grid);
  if (e == cudaSuccess)
    e = cudaMemcpy(h.data(), d_out, sizeof(ProbeOut) * grid, cudaMemcpyDeviceToHost);
  cudaFree(d_out);
  cudaFree(d_sink);
  if (e != cudaSuccess) return e;
  // Per SM: operations of all its CTAs over the span of its clock readings.
  std::vector<unsigned long long> lo(1024, ~0ull), hi(1024, 0);
  std::vector<int> ctas(1024, 0);
  for (const ProbeOut& o : h) {
    if (o.smid >= 1024) continue;
    lo[o.smid] = o.start < lo[o.smid] ? o.start : lo[o.smid];
    hi[o.smid] = o.stop > hi[o.smid] ? o.stop : hi[o.smid];
    ctas[o.smid]++;
  }
  const double per_cta = double(kProbeThreads) * kProbeIters * kChains * (OP == kOpFfma2 ? 2 : 1);
  double sum = 0.0;
  int used = 0;
  for (int s = 0; s < 1024; ++s) {
    if (!ctas[s] || hi[s] <= lo[s]) continue;
    sum += per_cta * ctas[s] / double(hi[s] - lo[s]);
    ++used;
  }
  *rate = used ? sum / used : 0.0;
  return cudaSuccess;
}

// ------------------------------------------------ MUFU accuracy, exhaustive
// Every fp32 input of a range is evaluated; errors are measured against the
// FP64 functions (exact for the reciprocal: r x needs 48 bits).
//   op 0: max |rcp.approx.ftz(x) x - 1| over normal x with 1/x normal;
//   op 1: lg2.approx.ftz(x) - log2(x): the largest absolute error over
//         x in [1/2, 2] (slot 1) and the largest error relative to |log2 x|
//         over every other normal x (slot 3);
//   op 2: max |ex2.approx.ftz(t) / 2^t - 1| over t in [-126, 127) where 2^t
//         is a normal float.
// A non-negative double's bit pattern orders like the double, so the maxima
// are reduced with 64-bit integer atomics.
constexpr int kErrThreads = 256;

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* dst, double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(dst, static_cast<unsigned long long>(__double_as_longlong(v)));
}

__global__ void __launch_bounds__(kErrThreads)
    mufu_error_kernel(int op, uint32_t first_bits, uint64_t count, unsigned long long* out) {
  double worst = 0.0, outer = 0.0;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += stride) {
    const float x = __uint_as_float(first_bits + static_cast<uint32_t>(i));
    double e = 0.0;
    if (op == 0) {
      const float r = rcp_approx(x);
      if (fabsf(r) >= FLT_MIN && fabsf(r) <= FLT_MAX) e = fabs(double(r) * double(x) - 1.0);
    } else if (op == 1) {
      const double ref = log2(double(x));
      e = fabs(double(lg2_approx(x)) - ref);
      if (fabs(ref) > 1.0) {
        outer = fmax(outer, e / fabs(ref));
        e = 0.0;
      }
    } else {
      const double ref = exp2(double(x));
      if (ref >= double(FLT_MIN) && ref <= double(FLT_MAX))
        e = fabs(double(ex2_approx(x)) / ref - 1.0);
    }
    worst = fmax(worst, e);
  }
  atomic_max_nonneg(out + op, worst);
  if (op == 1) atomic_max_nonneg(out + 3, outer);
}

}  // namespace

cudaError_t measure_mufu_errors(int sm_count, double errs[4]) {
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 4 * sizeof(unsigned long long));
  if (e != cudaSuccess) return e;
  e = cudaMemset(d, 0, 4 * sizeof(unsigned long long));
  // Positive inputs only: the three functions are odd or defined for x > 0,
  // and the sign of x does not enter the MUFU's mantissa arithmetic.
  const uint32_t min_normal = 0x00800000u, inf_bits = 0x7f800000u;
  struct Range { int op; uint32_t first; uint64_t count; };
  const uint32_t t_lo = __builtin_bit_cast(uint32_t, 0x1p-30f), t_hi = __builtin_bit_cast(uint32_t, 127.0f);
  const Range ranges[] = {
      {0, min_normal, uint64_t(inf_bits - min_normal)},
      {1, min_normal, uint64_t(inf_bits - min_normal)},
      {2, t_lo, uint64_t(t_hi - t_lo)},                           // t in [2^-30, 127)
      {2, t_lo | 0x80000000u, uint64_t(__builtin_bit_cast(uint32_t, 126.0f) - t_lo)},  // -t
  };
  const unsigned grid = static_cast<unsigned>(sm_count) * 8u;
  for (const Range& r : ranges) {
    if (e != cudaSuccess) break;
    mufu_error_kernel<<<grid, kErrThreads>>>(r.op, r.first, r.count, d);
    e = cudaGetLastError();
  }
  unsigned long long h[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < 4; ++k) errs[k] = __builtin_bit_cast(double, h[k]);
  return cudaSuccess;
}

cudaError_t measure_pipe_rates(int sm_count, double rates[6]) {
  cudaError_t e;
  if ((e = run_probe<kOpFfma>(sm_count, 2, &rates[0])) != cudaSuccess) return e;
  if ((e = run_probe<kOpFfma2>(sm_count, 2, &rates[1])) != cudaSuccess) return e;
  if ((e = run_probe<kOpRcp>(sm_count, 2, &rates[2])) != cudaSuccess) return e;
  if ((e = run_probe<kOpLg2>(sm_count, 2, &rates[3])) != cudaSuccess) return e;
  if ((e = run_probe<kOpEx2>(sm_count, 2, &rates[4])) != cudaSuccess) return e;
  if ((e = run_probe<kOpDfma>(sm_count, 2, &rates[5])) != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace idw
