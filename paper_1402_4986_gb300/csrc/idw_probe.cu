// Pipe-rate probe: issue rate of the arithmetic the forward pass uses
// (FFMA, packed FFMA2, MUFU rcp / lg2 / ex2, DFMA), in operations per SM
// per clock.  Each CTA times its own loop with the SM's clock counter and
// reports its SM id; the host sums operations per SM and divides by the
// span of that SM's clock readings, so the result does not depend on the
// clock speed.  These rates are the denominators of the pipe roofline.
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

}  // namespace

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
