// FP32-compensated forward pass of global Shepard IDW (Sec. 2.1, Eq. 1),
// for one problem or a batch of independent problems in one launch.
//
// Pipeline (one call): coordinate range scan -> staging -> persistent
// all-pairs sweep -> combine (FP64 division) with the FP64 slow path of
// flagged queries.
//
// The sweep is the paper's tiled kernel (Sec. 4.2: the data are read once
// per block of prediction points, tile by tile) rebuilt for sm_103a:
//   * each thread holds 2*kQueryPairsF32 queries in registers as pairs, so
//     every FP32 operation is a packed fp32x2 instruction over two queries;
//   * data tiles stream global -> shared by 1-D bulk TMA into a ring of
//     stages guarded by mbarriers (bounded waits); every warp reads the same
//     record (a broadcast shared load);
//   * the record is staged pre-duplicated as (x,x,y,y)+(z,z) so it feeds the
//     packed instructions with no register moves (the paper's aligned AoS
//     record, Sec. 3.3, widened for pair arithmetic);
//   * w = d^-p without a square root.  p = 2: one MUFU reciprocal of d^2,
//     except that for one of the query pairs the two pairs share one
//     reciprocal, 1/(da db), and recover 1/da = db/(da db) with two FMULs;
//     this moves work from the MUFU pipe (the binding one) to the FMA pipe.
//     General p: 2^(-(p/2) log2 d^2) with the product's rounding error
//     recovered by an FMA and applied to first order;
//   * sums run in chunks of 64 (p = 2) or 32 points: S0 as a balanced
//     binary tree, S1 as FMA chains of products joined by a tree; each chunk
//     sum is folded into a (hi, lo) pair by Knuth's TwoSum (the pairs live in
//     shared memory, one slot per thread and query pair) and the pair is
//     renormalised once per work unit, so the worst-case error is a fixed
//     number of roundings per term, independent of n;
//   * the (problem, query tile, data tile) work units are split evenly over
//     a grid of co-resident CTAs (stream-K).  Pieces of a query tile are
//     summed as compensated FP32 pairs by the combine, which converts each
//     query's sums to FP64 once for the division; it plays the role of the
//     paper's in-block reduction of the improved CDP kernel (Sec. 3.1).
//   * coordinates are multiplied by a power of two per problem (exact in
//     FP32) so the largest magnitude lies in [2^9, 2^10): Eq. 1 depends only
//     on distance ratios, so Z is unchanged, and products of squared
//     distances cannot overflow.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <utility>

#include "idw_device.cuh"
#include "idw_internal.h"
#include "idw_f32_common.cuh"
#include "idw_slowpath.cuh"

namespace idw {
namespace {

constexpr int TB = kRecordsF32;
constexpr int ST = kStagesF32;
constexpr uint32_t kTileBytes = static_cast<uint32_t>(kTileBytesF32);
static_assert(kTileBytes % 16 == 0, "bulk copies move multiples of 16 bytes");
constexpr bool chunk_shape_ok(ChunkShape c) {
  return TB % c.points == 0 && c.points == (1 << c.tree_levels) &&
         c.points == c.chain << c.chain_levels;
}
static_assert(chunk_shape_ok(kChunkPow2) && chunk_shape_ok(kChunkGeneral), "chunk trees");

// Compiled sweep variants (the autotuner picks one per size class):
// threads per CTA, query pairs per thread, and how many of those pairs share
// one reciprocal per data point at p = 2.  Each keeps 128 registers/thread
// and 16 resident warps per SM (variant 4: all 16 in one CTA, which keeps
// them in step at every tile barrier).
// KSH pairs share on every data point; pair KALT (if >= 0) also shares on
// every other data point, so a fraction (KSH + 0.5 [KALT >= 0]) / KP of the
// pairs share.
// TBV is the number of data points per work unit: 256 (one staging tile),
// or 64 for the fine-grained variant 5, which splits small problems into
// four times as many units; it needs the record-contiguous aligned-AoS
// staging (p = 2).
template <int V> struct Var;
template <> struct Var<0> { static constexpr int NT = 256, KP = 4, KSH = 1, KALT = -1, TBV = 256; };
template <> struct Var<1> { static constexpr int NT = 256, KP = 4, KSH = 0, KALT = -1, TBV = 256; };
template <> struct Var<2> { static constexpr int NT = 256, KP = 4, KSH = 1, KALT = 1, TBV = 256; };
template <> struct Var<3> { static constexpr int NT = 128, KP = 4, KSH = 1, KALT = -1, TBV = 256; };
template <> struct Var<4> { static constexpr int NT = 512, KP = 4, KSH = 1, KALT = 1, TBV = 256; };
template <> struct Var<5> { static constexpr int NT = 256, KP = 4, KSH = 1, KALT = -1, TBV = 64; };
template <int V> __host__ __device__ constexpr int qt_of() { return Var<V>::NT * 2 * Var<V>::KP; }
static_assert(kNumSweepVariants == 6, "variant table");
static_assert(qt_of<0>() == kQueriesPerCtaF32, "default variant is the documented tiling");

struct SweepArgs {
  int64_t units;
  int grid;
  float half_p, neg_half_p;
  float4* partial;  // partial_slots x QT records (S0 hi, S0 lo, S1 hi, S1 lo)
  const float* scales;
  unsigned* err;
};

// log2 on the FMA pipe, for both lanes: x = 2^k m, m in [1/sqrt 2, sqrt 2),
// log2 x = k + s P(s), s = m - 1 (exact), P the degree-8 minimax fit of
// log2(1 + s)/s for the relative error (Remez exchange, fit_log2.py),
// rounded to fp32 and evaluated by Horner's rule with packed FMAs.  Zero or
// subnormal x gives -inf and an infinite or NaN x gives 2^20, as the MUFU
// path with its clamp does.  Error: at most 1.5u absolute for x in
// [1/2, 2] and 1.5u relative to |log2 x| elsewhere (checked exhaustively
// on the CPU).
__constant__ float kLog2Poly[] = {
    1.4426950216293335f,  -0.7213473320007324f, 0.48091062903404236f,
    -0.3607036769390106f, 0.28791624307632446f, -0.23894482851028442f,
    0.21571560204029083f, -0.20726972818374634f, 0.12583701312541962f,
};
constexpr int kLog2PolyDegree = 8;

__device__ __forceinline__ u64 log2_fma_pair(u64 x2) {
  float xa, xb;
  upk(x2, xa, xb);
  const int ua = __float_as_int(xa), ub = __float_as_int(xb);
  const int ka = (ua - 0x3F3504F3) >> 23, kb = (ub - 0x3F3504F3) >> 23;  // m >= 1/sqrt 2
  const u64 m = pk(__int_as_float(ua - (ka << 23)), __int_as_float(ub - (kb << 23)));
  // float(k) exactly: k sits in the low mantissa bits of 1.5 2^23.
  const u64 kf = pk(__int_as_float(0x4B400000 + ka) - 12582912.f,
                    __int_as_float(0x4B400000 + kb) - 12582912.f);
  const u64 sv = sub2(m, pk(1.f, 1.f));
  u64 poly = pk(kLog2Poly[kLog2PolyDegree], kLog2Poly[kLog2PolyDegree]);
#pragma unroll
  for (int i = kLog2PolyDegree - 1; i >= 0; --i) poly = fma2(poly, sv, pk(kLog2Poly[i], kLog2Poly[i]));
  float la, lb;
  upk(fma2(sv, poly, kf), la, lb);
  const int ea = (ua >> 23) & 0xff, eb = (ub >> 23) & 0xff;
  la = ea == 0 ? -INFINITY : (ea == 0xff ? 1048576.f : la);
  lb = eb == 0 ? -INFINITY : (eb == 0xff ? 1048576.f : lb);
  return pk(la, lb);
}

template <int MODE>
__device__ __forceinline__ u64 weight_pair(u64 d2, bool shared_rcp, u64 half_p2,
                                           u64 neg_half_p2, bool fma_log2 = false) {
  float a, b;
  upk(d2, a, b);
  if (MODE == kPow2) {
    if (shared_rcp) {
      const float r = rcp_approx(mul_ftz(a, b));  // 1 / (da db)
      return pk(mul_ftz(b, r), mul_ftz(a, r));
    }
    return pk(rcp_approx(a), rcp_approx(b));
  } else {
    // L = log2 d^2, clamped so that +inf (padding) stays finite below; on
    // the MUFU pipe, or for a fixed fraction of the pairs on the FMA pipe.
    const u64 L = fma_log2 ? log2_fma_pair(d2)
                           : pk(fminf(lg2_approx(a), 1048576.f), fminf(lg2_approx(b), 1048576.f));
    const u64 th = mul2(L, neg_half_p2);  // t_hi = fl(t), t = -(p/2) L
    // (p/2) L + t_hi = -(t - t_hi): the product's rounding error, exact.
    const u64 ntl = fma2(L, half_p2, th);
    float ta, tb;
    upk(th, ta, tb);
    const u64 e = pk(ex2_approx(ta), ex2_approx(tb));
    const u64 c = mul2(ntl, pk(-0.6931471805599453f, -0.6931471805599453f));  // t_lo ln 2
    return fma2(e, c, e);  // 2^(t_hi + t_lo) to first order in t_lo
  }
}

// General power with the FMA-pipe log2 (IDW_OPT_FMA_LOG2): query pair 0
// takes log2 d^2 on the FMA pipe for the data points r with
// r % kLog2FmaPeriod == 0, 1 pair in 16.  The MUFU pipe (lg2 at 16 and ex2
// at 32 per SM per clock) binds the general sweep while the FMA pipe is 73 %
// busy, yet every fraction measured (1/16 to 1/4) was slower: the polynomial
// and its exponent handling cost more issue slots than the lg2 they replace.
// It is kept as an option, off by default.
constexpr int kLog2FmaPeriod = 4;

// The record of data point c + r of a staged tile as three register pairs
// (x,x), (y,y), (z,z), for each staging layout.
template <int LAYOUT>
__device__ __forceinline__ void load_record(const unsigned char* tile, int i, u64& xx, u64& yy,
                                            u64& zz) {
  if (LAYOUT == 0) {
    const ulonglong2 xy = reinterpret_cast<const ulonglong2*>(tile)[i];
    xx = xy.x;
    yy = xy.y;
    zz = reinterpret_cast<const u64*>(tile + TB * 16)[i];
  } else if (LAYOUT == 1) {
    const float4 v = reinterpret_cast<const float4*>(tile)[i];
    xx = pk(v.x, v.x);
    yy = pk(v.y, v.y);
    zz = pk(v.z, v.z);
  } else {
    const float* f = reinterpret_cast<const float*>(tile);
    const float x = f[i], y = f[TB + i], z = f[2 * TB + i];
    xx = pk(x, x);
    yy = pk(y, y);
    zz = pk(z, z);
  }
}

// The running (hi, lo) pairs of a thread: slot 2k holds (S0 hi, S0 lo) of
// query pair k and slot 2k + 1 (S1 hi, S1 lo), each a pair of packed lanes;
// in registers, or in shared memory at [s NT + tid] after the tile ring.
constexpr bool kSumsInShared = true;

template <int KP, int NT, bool SMEM>
struct SumSlots;
template <int KP, int NT>
struct SumSlots<KP, NT, false> {
  ulonglong2 r[2 * KP];
  __device__ __forceinline__ void bind(unsigned char*, int) {}
  __device__ __forceinline__ ulonglong2 get(int s) const { return r[s]; }
  __device__ __forceinline__ void set(int s, ulonglong2 v) { r[s] = v; }
};
template <int KP, int NT>
struct SumSlots<KP, NT, true> {
  ulonglong2* base;  // this thread's slot 0
  __device__ __forceinline__ void bind(unsigned char* p, int tid) {
    base = reinterpret_cast<ulonglong2*>(p) + tid;
  }
  __device__ __forceinline__ ulonglong2 get(int s) const { return base[s * NT]; }
  __device__ __forceinline__ void set(int s, ulonglong2 v) { base[s * NT] = v; }
};

// Shared memory of one sweep CTA: the tile ring, then the sum slots.
template <int V, int LAYOUT>
__host__ __device__ constexpr size_t ring_bytes_of() {
  return size_t(ST) * (Var<V>::TBV == TB ? tile_bytes_of<LAYOUT>() : Var<V>::TBV * 16u);
}
template <int V>
__host__ __device__ constexpr size_t hl_bytes_of() {
  return kSumsInShared ? size_t(2) * Var<V>::KP * Var<V>::NT * sizeof(ulonglong2) : 0;
}
template <int V, int LAYOUT>
__host__ __device__ constexpr size_t sweep_smem_of() {
  return ring_bytes_of<V, LAYOUT>() + hl_bytes_of<V>();
}

template <int MODE, int CAP, int V, int LAYOUT = 0, bool FMA_LOG2 = false>
__global__ void __launch_bounds__(Var<V>::NT, 512 / Var<V>::NT)
    sweep_kernel(const SweepArgs a, const __grid_constant__ Table<CAP> t) {
  constexpr int NT = Var<V>::NT, KP = Var<V>::KP, KSHARED = Var<V>::KSH, QT = qt_of<V>();
  constexpr int KALT = Var<V>::KALT;
  constexpr ChunkShape SH = MODE == kPow2 ? kChunkPow2 : kChunkGeneral;
  constexpr int CH = SH.points;
  constexpr int TBU = Var<V>::TBV;
  static_assert(TBU == TB || LAYOUT == 1, "sub-tile units need record-contiguous staging");
  static_assert(TBU % CH == 0, "chunks tile a work unit");
  // Bytes of one work unit's data: a whole staging tile, or a slice of the
  // record-contiguous aligned-AoS array.
  constexpr uint32_t kTileBytes = TBU == TB ? tile_bytes_of<LAYOUT>() : TBU * 16u;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long full_bar[ST];
  SumSlots<KP, NT, kSumsInShared> HL;
  HL.bind(smem + ring_bytes_of<V, LAYOUT>(), threadIdx.x);

  const int tid = threadIdx.x;
  const int64_t g = blockIdx.x;
  const int64_t u0 = unit_begin(g, a.units, a.grid);
  const int64_t total = unit_begin(g + 1, a.units, a.grid) - u0;
  if (total <= 0) return;

  if (tid == 0) {
    for (int s = 0; s < ST; ++s) mbar_init(smem_u32(&full_bar[s]), 1);
    fence_barrier_init();
  }
  pdl_trigger();
  pdl_wait();  // the staged tiles and scales come from the kernels before
  __syncthreads();

  // Producer (thread 0): one bulk copy per unit, STAGES units ahead.
  int64_t issued = 0;
  int pk_inst = find_unit(t, u0);
  auto issue = [&](int64_t local) {
    const int64_t u = u0 + local;
    while (pk_inst + 1 < t.count && t.inst[pk_inst + 1].unit_base <= u) ++pk_inst;
    const Instance& I = t.inst[pk_inst];
    const int64_t dt = (u - I.unit_base) % I.data_tiles;
    const int s = static_cast<int>(local % ST);
    bulk_load(smem_u32(smem + s * kTileBytes), I.tiles + dt * kTileBytes, kTileBytes,
              smem_u32(&full_bar[s]));
  };
  if (tid == 0) {
    for (; issued < ST && issued < total; ++issued) issue(issued);
  }

  const u64 hp2 = pk(a.half_p, a.half_p);
  const u64 nhp2 = pk(a.neg_half_p, a.neg_half_p);
  int ci = find_unit(t, u0);
  int64_t i = 0;
  bool aborted = false;
  while (i < total) {
    const int64_t u = u0 + i;
    while (ci + 1 < t.count && t.inst[ci + 1].unit_base <= u) ++ci;
    const Instance& I = t.inst[ci];
    const int64_t qt = (u - I.unit_base) / I.data_tiles;
    const int64_t seg_end = min(total, I.unit_base + (qt + 1) * I.data_tiles - u0);
    const float sc = a.scales[ci];

    u64 QX[KP], QY[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const int64_t ja = qt * QT + (2 * k) * NT + tid;
      const int64_t jb = ja + NT;
      const float xa = ja < I.m ? I.queries[2 * ja] * sc : 0.f;
      const float ya = ja < I.m ? I.queries[2 * ja + 1] * sc : 0.f;
      const float xb = jb < I.m ? I.queries[2 * jb] * sc : 0.f;
      const float yb = jb < I.m ? I.queries[2 * jb + 1] * sc : 0.f;
      QX[k] = pk(xa, xb);
      QY[k] = pk(ya, yb);
      HL.set(2 * k, make_ulonglong2(0ull, 0ull));
      HL.set(2 * k + 1, make_ulonglong2(0ull, 0ull));
    }

    for (; i < seg_end; ++i) {
      const int s = static_cast<int>(i % ST);
      const uint32_t parity = static_cast<uint32_t>((i / ST) & 1);
      const bool ok = mbar_wait_bounded(smem_u32(&full_bar[s]), parity, a.err);
      if (ok) {
        const unsigned char* tile = smem + s * kTileBytes;
#pragma unroll 1
        for (int c = 0; c < TBU; c += CH) {
          // S0: tree over the chunk's weights.  S1: chains of SH.chain
          // products w z (one MUL, then FMAs), chains joined by a tree.
          u64 P0[KP][SH.tree_levels], P1[KP][SH.chain_levels], T1[KP], C0[KP], C1[KP];
#pragma unroll
          for (int r = 0; r < CH; ++r) {
            u64 xx, yy, zz;
            load_record<LAYOUT>(tile, c + r, xx, yy, zz);
#pragma unroll
            for (int k = 0; k < KP; ++k) {
              // d^2 rounded to nearest with subnormals kept: a d^2 that is
              // itself subnormal is flushed by the weight's MUFU input and
              // sends the query to the FP64 path through a non-finite sum.
              const u64 dx = sub2(QX[k], xx);
              const u64 dy = sub2(QY[k], yy);
              const u64 d2 = fma2(dy, dy, mul2(dx, dx));
              const bool shared = k < KSHARED || (k == KALT && (r & 1));
              const bool fma_log2 = FMA_LOG2 && k == 0 && r % kLog2FmaPeriod == 0;
              const u64 w = weight_pair<MODE>(d2, shared, hp2, nhp2, fma_log2);
              tree_push<SH.tree_levels>(P0[k], w, r, C0[k]);
              if (r % SH.chain == 0) {
                T1[k] = mul2(w, zz);
              } else {
                T1[k] = fma2(w, zz, T1[k]);
              }
              if (r % SH.chain == SH.chain - 1)
                tree_push<SH.chain_levels>(P1[k], T1[k], r / SH.chain, C1[k]);
            }
          }
          // Error-free folds of the chunk sums into the (hi, lo) slots; the
          // last chunk of a work unit also renormalises each pair.
          const bool last = c + CH == TBU;
#pragma unroll
          for (int k = 0; k < KP; ++k) {
            ulonglong2 s0 = HL.get(2 * k);
            ulonglong2 s1 = HL.get(2 * k + 1);
            two_sum_acc(s0.x, s0.y, C0[k]);
            two_sum_acc(s1.x, s1.y, C1[k]);
            if (last) {
              two_sum_renorm(s0.x, s0.y);
              two_sum_renorm(s1.x, s1.y);
            }
            HL.set(2 * k, s0);
            HL.set(2 * k + 1, s1);
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

    float4* P = a.partial + (I.qtile_base + qt + g) * QT;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const ulonglong2 s0 = HL.get(2 * k);
      const ulonglong2 s1 = HL.get(2 * k + 1);
      float h0a, h0b, l0a, l0b, h1a, h1b, l1a, l1b;
      upk(s0.x, h0a, h0b);
      upk(s0.y, l0a, l0b);
      upk(s1.x, h1a, h1b);
      upk(s1.y, l1a, l1b);
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

// FP64 combine of the pieces of each query: Z = S1 / S0, or, for a query
// outside the fast form (exact hit or FP32 range exceeded), the FP64 slow
// path run by the same CTA.  One CTA covers 32 consecutive query slots
// (lanes x) and splits each query's pieces over 8 warps (lanes y, strided);
// every warp's loads are coalesced across its 32 queries, and the 8 partial
// sums are added in a fixed order, so the result is deterministic.  The
// CTA's flagged queries are then redone one after another by all 256
// threads (a query's slow path reads all n points).  Block 0 finally clears
// the per-problem range words the range scan and staging of this call used,
// so the next call (or graph replay) starts from zero without a memset.
constexpr int kCombineQueries = 32;
constexpr int kCombineLanes = 8;
static_assert(kCombineQueries * kCombineLanes == kSlowThreads, "the combine CTA runs the slow path");

template <int CAP, int QT>
__global__ void __launch_bounds__(kCombineQueries * kCombineLanes)
    combine_kernel(const __grid_constant__ Table<CAP> t, const float4* __restrict__ partial,
                   int64_t total_slots, int64_t units, int grid, const float* __restrict__ scales,
                   double p, Control* __restrict__ ctrl) {
  __shared__ float4 red[kCombineLanes][kCombineQueries];
  __shared__ int2 flagged[kCombineQueries];
  __shared__ int nflagged;
  pdl_trigger();
  pdl_wait();
  const int lx = threadIdx.x % kCombineQueries, ly = threadIdx.x / kCombineQueries;
  const int64_t idx = int64_t(blockIdx.x) * kCombineQueries + lx;
  bool valid = idx < total_slots;
  const int64_t qtg = idx / QT, lq = idx % QT;
  const int k = valid ? find_qtile(t, qtg) : 0;
  const Instance& I = t.inst[k];
  const int64_t qt = qtg - I.qtile_base;
  const int64_t j = qt * QT + lq;
  valid = valid && j < I.m;
  // Each piece is an (S0 hi, S0 lo, S1 hi, S1 lo) record with |lo| at most
  // half an ulp of hi.  Pieces are added as FP32 (hi, lo) pairs, the hi parts
  // by TwoSum and the lo parts and the TwoSum errors plainly (the loss is of
  // order P^2 u^2 for P pieces): the FP32 pipe runs this at 64 times the FP64
  // pipe's rate.  The sums go to FP64 once, for the division.
  float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
  if (valid) {
    const int64_t g0 = cta_of_unit(I.unit_base + qt * I.data_tiles, units, grid);
    const int64_t g1 = cta_of_unit(I.unit_base + (qt + 1) * I.data_tiles - 1, units, grid);
#pragma unroll 4
    for (int64_t g = g0 + ly; g <= g1; g += kCombineLanes) {
      const float4 v = partial[(qtg + g) * QT + lq];
      two_sum_acc_f32(h0, l0, v.x);
      l0 += v.y;
      two_sum_acc_f32(h1, l1, v.z);
      l1 += v.w;
    }
  }
  red[ly][lx] = make_float4(h0, l0, h1, l1);
  if (threadIdx.x == 0) nflagged = 0;
  __syncthreads();
  if (ly == 0 && valid) {
#pragma unroll
    for (int y = 1; y < kCombineLanes; ++y) {
      const float4 r = red[y][lx];
      two_sum_acc_f32(h0, l0, r.x);
      l0 += r.y;
      two_sum_acc_f32(h1, l1, r.z);
      l1 += r.w;
    }
    const double s0 = double(h0) + double(l0), s1 = double(h1) + double(l1);
    if (!(s0 > kTinySumPerPoint * double(I.n)) || !isfinite(s0) || !isfinite(s1) ||
        (p >= 2.0 && s0 > kHugeSumPow2Up)) {
      flagged[atomicAdd(&nflagged, 1)] = make_int2(k, static_cast<int>(j));
    } else {
      I.out[j] = static_cast<float>(s1 / s0);
      // Weights were computed on coordinates scaled by s: w = s^-p w_true.
      if (I.s0_out) I.s0_out[j] = s0 * pow(double(scales[k]), p);
      if (I.hit_out) I.hit_out[j] = kNoHit;
    }
  }
  __syncthreads();
  const int nf = nflagged;
  for (int f = 0; f < nf; ++f) {  // uniform across the CTA
    const int2 e = flagged[f];
    const Instance& F = t.inst[e.x];
    const int64_t jf = e.y;
    slow_one_query<float, float>(F.data, F.n, F.queries[2 * jf], F.queries[2 * jf + 1], p,
                                 &F.out[jf], F.s0_out ? &F.s0_out[jf] : nullptr,
                                 F.hit_out ? &F.hit_out[jf] : nullptr);
  }
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c < t.count; c += blockDim.x) ctrl->maxbits[c] = 0u;
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

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Launches `kernel` allowed to start before the kernel ahead of it in the
// stream completes (programmatic dependent launch); the kernel itself waits
// in pdl_wait() before touching memory, so results are as with a plain
// launch and only launch latency overlaps.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t stream, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Raises a kernel's dynamic shared memory limit to `bytes` (needed above
// 48 KB), once per kernel and device (one flag word per instantiation).
template <auto KERNEL>
cudaError_t allow_dynamic_smem(size_t bytes) {
  static unsigned long long done = 0;  // one bit per device ordinal < 64
  if (bytes <= 48u * 1024u) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (__atomic_load_n(&done, __ATOMIC_ACQUIRE) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(bytes));
  if (e == cudaSuccess && bit) __atomic_fetch_or(&done, bit, __ATOMIC_ACQ_REL);
  return e;
}

template <int CAP, int V, int MODE, int LAYOUT, bool FMA_LOG2 = false>
cudaError_t launch_impl(const F32Problem* probs, const BatchPlan& plan, double p,
                        unsigned char* ws, Control* ctrl, int sm_count, const SweepEvents* ev,
                        cudaStream_t stream) {
  Table<CAP> t;
  t.count = plan.count;
  t.pad = 0;
  unsigned char* tiles = ws;
  float4* partial = reinterpret_cast<float4*>(ws + plan.staged_bytes);
  float* scales = reinterpret_cast<float*>(ws + plan.staged_bytes + plan.partial_bytes);
  unsigned* maxbits = ctrl->maxbits;  // zero on entry: cleared by the previous call's combine
  int64_t longest = 1;
  for (int k = 0; k < plan.count; ++k) {
    Instance& I = t.inst[k];
    I.data = probs[k].data;
    I.queries = probs[k].queries;
    I.out = probs[k].out;
    I.s0_out = probs[k].s0_out;
    I.hit_out = probs[k].hit_out;
    I.tiles = tiles + size_t(plan.tile_offset[k]) * tile_bytes_of<LAYOUT>();
    I.unit_base = plan.unit_base[k];
    I.record_base = plan.tile_offset[k] * TB;
    I.n = static_cast<int32_t>(probs[k].n);
    I.m = static_cast<int32_t>(probs[k].m);
    I.data_tiles = static_cast<int32_t>(plan.data_tiles[k]);
    I.qtile_base = static_cast<int32_t>(plan.qtile_base[k]);
    longest = std::max<int64_t>(longest, std::max(probs[k].n, probs[k].m));
  }
  cudaError_t e;

  const unsigned gx = static_cast<unsigned>(std::min<int64_t>(1024, (longest + 255) / 256));
  if ((e = launch_pdl(range_kernel<CAP>, dim3(gx, plan.count), dim3(256), 0, stream, t,
                      maxbits)) != cudaSuccess)
    return e;
  const int64_t records = plan.total_stage_tiles * TB;
  const unsigned sgrid = static_cast<unsigned>((records + 255) / 256);
  if ((e = launch_pdl(stage_kernel<CAP, MODE, LAYOUT>, dim3(sgrid), dim3(256), 0, stream, t,
                      records, static_cast<const unsigned*>(maxbits), scales)) != cudaSuccess)
    return e;

  SweepArgs a;
  a.units = plan.units;
  a.grid = plan.grid;
  a.half_p = static_cast<float>(0.5 * p);
  a.neg_half_p = -a.half_p;
  a.partial = partial;
  a.scales = scales;
  a.err = &ctrl->error;
  constexpr size_t smem = sweep_smem_of<V, LAYOUT>();
  if ((e = allow_dynamic_smem<sweep_kernel<MODE, CAP, V, LAYOUT, FMA_LOG2>>(smem)) != cudaSuccess)
    return e;
  if (ev && (e = cudaEventRecord(ev->start, stream)) != cudaSuccess) return e;
  constexpr int NT = Var<V>::NT, QT = qt_of<V>();
  // With profiling events the sweep is launched plainly, so that the events
  // around it bracket it alone.
  if (ev)
    sweep_kernel<MODE, CAP, V, LAYOUT, FMA_LOG2><<<plan.grid, NT, smem, stream>>>(a, t);
  else if ((e = launch_pdl(sweep_kernel<MODE, CAP, V, LAYOUT, FMA_LOG2>, dim3(plan.grid),
                           dim3(NT), smem, stream, a, t)) != cudaSuccess)
    return e;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev && (e = cudaEventRecord(ev->stop, stream)) != cudaSuccess) return e;

  const int64_t slots = plan.total_query_tiles * QT;
  return launch_pdl(combine_kernel<CAP, QT>,
                    dim3(static_cast<unsigned>((slots + kCombineQueries - 1) / kCombineQueries)),
                    dim3(kCombineQueries * kCombineLanes), 0, stream, t,
                    static_cast<const float4*>(partial), slots, plan.units, plan.grid,
                    static_cast<const float*>(scales), p, ctrl);
}

}  // namespace

int sweep_variant_queries_per_cta(int variant) {
  switch (variant) {
    case 1: return qt_of<1>();
    case 2: return qt_of<2>();
    case 3: return qt_of<3>();
    case 4: return qt_of<4>();
    case 5: return qt_of<5>();
    default: return qt_of<0>();
  }
}

int sweep_variant_points_per_unit(int variant) {
  switch (variant) {
    case 5: return Var<5>::TBV;
    default: return TB;
  }
}

int default_sweep_variant(const F32Problem* probs, int count, bool general_form, int sm_count) {
  const int64_t q4 = qt_of<4>(), q0 = qt_of<0>();
  double pad4 = 0, pad0 = 0, units0 = 0;
  for (int k = 0; k < count; ++k) {
    pad4 += double((probs[k].m + q4 - 1) / q4 * q4);
    pad0 += double((probs[k].m + q0 - 1) / q0 * q0);
    units0 += double((probs[k].m + q0 - 1) / q0) * double((probs[k].n + TB - 1) / TB);
  }
  if (!general_form && units0 < 4.0 * sm_count * 2) return 5;
  return pad4 <= 1.01 * pad0 ? 4 : 0;
}

int resolve_sweep_variant(int variant, bool general_form) {
  if (variant < 0 || variant >= kNumSweepVariants) return 0;
  // Sub-tile work units need the aligned-AoS staging of the p = 2 form.
  if (general_form && sweep_variant_points_per_unit(variant) != TB) return 0;
  return variant;
}

void plan_batch_f32(const F32Problem* probs, int count, int sm_count, int ctas_per_sm,
                    int variant, BatchPlan* bp) {
  const int QT = sweep_variant_queries_per_cta(variant);
  const int TBU = sweep_variant_points_per_unit(variant);
  bp->variant = variant;
  bp->count = count;
  bp->data_tiles.assign(count, 0);
  bp->query_tiles.assign(count, 0);
  bp->unit_base.assign(count, 0);
  bp->qtile_base.assign(count, 0);
  bp->tile_offset.assign(count, 0);
  int64_t units = 0, qtiles = 0, tiles = 0, queries = 0;
  for (int k = 0; k < count; ++k) {
    const int64_t dt = (probs[k].n + TBU - 1) / TBU;  // work units along the data
    const int64_t st = (probs[k].n + TB - 1) / TB;    // staging tiles
    const int64_t qt = (probs[k].m + QT - 1) / QT;
    bp->data_tiles[k] = dt;
    bp->query_tiles[k] = qt;
    bp->unit_base[k] = units;
    bp->qtile_base[k] = qtiles;
    bp->tile_offset[k] = tiles;
    units += dt * qt;
    qtiles += qt;
    tiles += st;
    queries += probs[k].m;
  }
  bp->units = units;
  bp->total_query_tiles = qtiles;
  bp->total_stage_tiles = tiles;
  const int64_t resident = int64_t(sm_count) * (ctas_per_sm > 0 ? ctas_per_sm : 1);
  bp->grid = static_cast<int>(std::max<int64_t>(1, std::min(units, resident)));
  bp->partial_slots = qtiles + bp->grid - 1;
  bp->staged_bytes = round_up(size_t(tiles) * kTileBytes, 256);  // the widest layout
  bp->partial_bytes = round_up(size_t(bp->partial_slots) * QT * sizeof(float4), 256);
  bp->list_bytes = 0;  // flagged queries are listed in the combine CTA's shared memory
  bp->scale_bytes = round_up(size_t(count) * sizeof(float), 256);
  bp->workspace_bytes = bp->staged_bytes + bp->partial_bytes + bp->list_bytes + bp->scale_bytes;
}

cudaError_t launch_batch_f32(const F32Problem* probs, const BatchPlan& plan, double p,
                             void* workspace, Control* ctrl, int sm_count,
                             const SweepEvents* ev, cudaStream_t stream) {
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  if (plan.count < 1 || plan.count > kBatchCap) return cudaErrorInvalidValue;
  const bool one = plan.count == 1;
  const bool pow2 = (p == 2.0) && !plan.force_general;
  // Default staging layout per weight form (measured fastest on GB300): the
  // aligned AoS record at p = 2, whose one shared load per point leaves the
  // special-function queue to the reciprocals; duplicated pair records for
  // general p, which need no register moves.  The other layouts are built
  // for the single-problem sweep of variant 0 (the layout ablation).
  const int layout = plan.layout >= 0 ? plan.layout : (pow2 ? 1 : 0);
  if (one && plan.variant == 4 && !pow2 && plan.fma_log2)
    return launch_impl<1, 4, kPowGeneral, 0, true>(probs, plan, p, ws, ctrl, sm_count, ev, stream);
  if (one && plan.variant == 0) {
    if (pow2 && layout == 0) return launch_impl<1, 0, kPow2, 0>(probs, plan, p, ws, ctrl, sm_count, ev, stream);
    if (pow2 && layout == 2) return launch_impl<1, 0, kPow2, 2>(probs, plan, p, ws, ctrl, sm_count, ev, stream);
    if (!pow2 && layout == 1) return launch_impl<1, 0, kPowGeneral, 1>(probs, plan, p, ws, ctrl, sm_count, ev, stream);
    if (!pow2 && layout == 2) return launch_impl<1, 0, kPowGeneral, 2>(probs, plan, p, ws, ctrl, sm_count, ev, stream);
  }
#define IDW_LAUNCH(V)                                                                        \
  if (pow2)                                                                                  \
    return one ? launch_impl<1, V, kPow2, 1>(probs, plan, p, ws, ctrl, sm_count, ev, stream) \
               : launch_impl<kBatchCap, V, kPow2, 1>(probs, plan, p, ws, ctrl, sm_count, ev,  \
                                                      stream);                               \
  return one ? launch_impl<1, V, kPowGeneral, 0>(probs, plan, p, ws, ctrl, sm_count, ev, stream) \
             : launch_impl<kBatchCap, V, kPowGeneral, 0>(probs, plan, p, ws, ctrl, sm_count, ev, \
                                                         stream)
  switch (plan.variant) {
    case 1: IDW_LAUNCH(1);
    case 2: IDW_LAUNCH(2);
    case 3: IDW_LAUNCH(3);
    case 4: IDW_LAUNCH(4);
    case 5:
      if (pow2)
        return one ? launch_impl<1, 5, kPow2, 1>(probs, plan, p, ws, ctrl, sm_count, ev, stream)
                   : launch_impl<kBatchCap, 5, kPow2, 1>(probs, plan, p, ws, ctrl, sm_count, ev,
                                                         stream);
      return cudaErrorInvalidValue;  // resolve_sweep_variant maps it away for general p
    default: IDW_LAUNCH(0);
  }
#undef IDW_LAUNCH
}

namespace {
template <int V>
int occupancy_variant(bool general_p) {
  int blocks = 0;
  if constexpr (Var<V>::TBV == TB) {
    if (general_p) {
      constexpr size_t smem = sweep_smem_of<V, 0>();
      allow_dynamic_smem<sweep_kernel<kPowGeneral, kBatchCap, V, 0>>(smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &blocks, sweep_kernel<kPowGeneral, kBatchCap, V, 0>, Var<V>::NT, smem);
      return blocks > 0 ? blocks : 1;
    }
  }
  constexpr size_t smem = sweep_smem_of<V, 1>();
  allow_dynamic_smem<sweep_kernel<kPow2, kBatchCap, V, 1>>(smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, sweep_kernel<kPow2, kBatchCap, V, 1>,
                                                Var<V>::NT, smem);
  return blocks > 0 ? blocks : 1;
}
}  // namespace

int occupancy_forward_f32(bool general_p, int variant) {
  switch (variant) {
    case 1: return occupancy_variant<1>(general_p);
    case 2: return occupancy_variant<2>(general_p);
    case 3: return occupancy_variant<3>(general_p);
    case 4: return occupancy_variant<4>(general_p);
    case 5: return general_p ? occupancy_variant<0>(true) : occupancy_variant<5>(false);
    default: return occupancy_variant<0>(general_p);
  }
}

cudaError_t launch_bounded_wait_selftest(Control* ctrl, cudaStream_t stream) {
  bounded_wait_selftest_kernel<<<1, 32, 0, stream>>>(&ctrl->error);
  return cudaGetLastError();
}

}  // namespace idw
