// Device helpers for the sm_103a IDW kernels: packed fp32x2 arithmetic,
// MUFU approximations, mbarrier + 1-D bulk TMA with bounded waits, and the
// stream-K work split shared by the persistent kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace idw {

typedef unsigned long long u64;

// Error bits written to the handle's device error word.
enum : unsigned { kErrWaitTimeout = 1u };

// A bounded wait gives up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// ------------------------------------------------------------ fp32x2 ops
// One instruction computes two independent fp32 lanes; the pair lives in an
// aligned 64-bit register pair (low half = first element).

__device__ __forceinline__ u64 pk(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk(u64 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// Rounded to nearest, subnormal results flushed: the pair arithmetic.
__device__ __forceinline__ u64 sub2f(u64 a, u64 b) {
  u64 r;
  asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 mul2f(u64 a, u64 b) {
  u64 r;
  asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 fma2f(u64 a, u64 b, u64 c) {
  u64 r;
  asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// Rounded to nearest with subnormals kept: the accumulation and the
// error-free transformations, which must be exact down to the subnormals.
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// Knuth's TwoSum on both lanes: s + e == a + b exactly (no overflow).
// Folds a chunk sum c into the running (hi, lo) pair.
__device__ __forceinline__ void two_sum_acc(u64& hi, u64& lo, u64 c) {
  const u64 s = add2(hi, c);
  const u64 bv = sub2(s, hi);
  const u64 av = sub2(s, bv);
  const u64 ea = sub2(hi, av);
  const u64 eb = sub2(c, bv);
  lo = add2(lo, add2(ea, eb));
  hi = s;
}

// Scalar TwoSum fold: hi + lo gains exactly c up to the rounding of lo + e.
__device__ __forceinline__ void two_sum_acc_f32(float& hi, float& lo, float c) {
  const float s = __fadd_rn(hi, c);
  const float bv = __fsub_rn(s, hi);
  const float av = __fsub_rn(s, bv);
  lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, av), __fsub_rn(c, bv)));
  hi = s;
}

// Renormalises a (hi, lo) pair with TwoSum: afterwards hi = fl(hi + lo) and
// lo is its exact remainder, so |lo| <= ulp(hi) / 2.  Keeping lo that small
// keeps the rounding of later `lo += e` steps second order in u.
__device__ __forceinline__ void two_sum_renorm(u64& hi, u64& lo) {
  const u64 s = add2(hi, lo);
  const u64 bv = sub2(s, hi);
  const u64 av = sub2(s, bv);
  lo = add2(sub2(hi, av), sub2(lo, bv));
  hi = s;
}

// Balanced pairwise summation of 2^LEVELS packed terms fed one at a time.
// Term i (a compile-time constant once the caller's loop is unrolled) enters
// at level 0; P[l] holds the sum of the last finished block of 2^l terms
// still waiting for its right-hand partner.  Every addition joins two blocks
// of equal size, so each term passes through exactly LEVELS roundings.  The
// sum of all 2^LEVELS terms lands in `total` with the last term.
template <int LEVELS>
__device__ __forceinline__ void tree_push(u64 (&P)[LEVELS], u64 v, int i, u64& total) {
#pragma unroll
  for (int l = 0; l < LEVELS; ++l) {
    if (!((i >> l) & 1)) {
      P[l] = v;
      return;
    }
    v = add2(P[l], v);
  }
  total = v;
}

// ------------------------------------------- programmatic dependent launch
// A kernel launched with programmatic stream serialization may start before
// the kernel ahead of it in the stream has finished.  pdl_wait() blocks
// until every grid it depends on has completed and its memory is visible,
// so a kernel calls it before it reads or writes anything those grids may
// touch; without that launch attribute it returns at once.  pdl_trigger()
// lets the next such kernel launch as soon as every CTA of this grid has
// started (it still waits for this grid's completion in its pdl_wait()).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------------- MUFU ops
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ------------------------------------------------- mbarrier + bulk TMA
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Producer side: announce `bytes` of transaction, then start one 1-D bulk
// copy global -> shared that completes those bytes on the barrier.
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the phase with the given parity to complete.  Gives up after
// kWaitLimitNs (or 2^30 polls), sets kErrWaitTimeout in *err and returns
// false; never spins without limit.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, unsigned* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (uint32_t it = 1; it < (1u << 30); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 0 && global_ns() - t0 > kWaitLimitNs) break;
  }
  atomicOr(err, kErrWaitTimeout);
  return false;
}

// ------------------------------------------------------ tile ring
// A ring of ST shared-memory stages fed by one 1-D bulk copy per work unit.
// Thread 0 produces; every thread consumes.  `src(u)` gives the global
// address of work unit u's tile.  Units are numbered locally from 0 (the
// CTA's first unit) to `total`.
template <int ST, class Src>
struct TileRing {
  unsigned char* smem;
  unsigned long long* bars;
  uint32_t bytes;
  unsigned* err;
  int64_t total;
  Src src;
  int64_t issued;  // meaningful in thread 0 only

  __device__ void start() {
    issued = 0;
    if (threadIdx.x == 0) {
      for (int s = 0; s < ST; ++s) mbar_init(smem_u32(&bars[s]), 1);
      fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (; issued < ST && issued < total; ++issued) issue(issued);
  }
  __device__ void issue(int64_t local) {
    const int s = static_cast<int>(local % ST);
    bulk_load(smem_u32(smem + size_t(s) * bytes), src(local), bytes, smem_u32(&bars[s]));
  }
  // Waits (bounded) for unit `local`; returns its stage, sets ok.
  __device__ const unsigned char* wait(int64_t local, bool& ok) {
    const int s = static_cast<int>(local % ST);
    ok = mbar_wait_bounded(smem_u32(&bars[s]), static_cast<uint32_t>((local / ST) & 1), err);
    return smem + size_t(s) * bytes;
  }
  // All threads are done with unit `local`'s stage: refill it, unless some
  // thread's wait gave up (then every thread returns false).
  __device__ bool release(bool ok) {
    if (__syncthreads_or(!ok)) return false;
    if (threadIdx.x == 0 && issued < total) {
      issue(issued);
      ++issued;
    }
    return true;
  }
  // After an abort at unit `from`: let copies still in flight land.
  __device__ void drain(int64_t from) {
    if (threadIdx.x != 0) return;
    for (int64_t k = from; k < issued; ++k)
      mbar_wait_bounded(smem_u32(&bars[k % ST]), static_cast<uint32_t>((k / ST) & 1), err);
  }
};

// ------------------------------------------------------ stream-K split
// Work units (query tile, data tile) are numbered query-tile-major; CTA g of
// G sweeps units [floor(g U / G), floor((g + 1) U / G)).
__host__ __device__ __forceinline__ int64_t unit_begin(int64_t g, int64_t units, int64_t grid) {
  return g * units / grid;
}
// The CTA whose run contains unit u.
__host__ __device__ __forceinline__ int64_t cta_of_unit(int64_t u, int64_t units, int64_t grid) {
  return ((u + 1) * grid - 1) / units;
}

// ------------------------------------------------------------ reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_min_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

}  // namespace idw
