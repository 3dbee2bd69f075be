// Adjoint of global Shepard IDW (Sec. 2.1, Eq. 1) for L = sum_j g_j Z(q_j).
//
// With w_ij = (d_ij^2)^(-p/2), S0_j = sum_i w_ij and Z_j = S1_j / S0_j
// (chain rule on Eq. 1; the paper gives no gradient):
//   dL/dq_j = -g_j (p / S0_j) sum_i (z_i - Z_j) w_ij (q_j - x_i) / d_ij^2
//   dL/dp   = -sum_j g_j / (2 S0_j) sum_i (z_i - Z_j) w_ij ln d_ij^2
//   dL/dz_i =  sum_j g_j w_ij / S0_j
//   dL/dx_i =  sum_j g_j (p / S0_j) (z_i - Z_j) w_ij (q_j - x_i) / d_ij^2
//
// Two all-pairs sweeps recompute the weights tile by tile (nothing of size
// n x m is stored):
//   * the query sweep holds queries in registers and streams the staged data
//     tiles of the forward pass (three sums per query);
//   * the data sweep is its transpose: data points in registers, staged
//     query records (q, g/S0, Z) streamed (three sums per data point).
// Both use the forward pass's machinery: packed fp32x2 arithmetic, 1-D bulk
// TMA tiles, chunked sums folded by TwoSum, stream-K pieces summed in FP64.
// Queries that the forward pass routed to its slow path (an exact hit, or
// FP32 range exceeded) are padded out of both sweeps and handled in FP64.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "idw_device.cuh"
#include "idw_f32_common.cuh"
#include "idw_internal.h"
#include "idw_slowpath.cuh"

namespace idw {
namespace {

constexpr int NTA = 512;             // threads per CTA (one CTA per SM keeps 16 warps in step)
constexpr int KPA = 2;               // register pairs per thread
constexpr int RT = NTA * 2 * KPA;    // register-side points per CTA tile (2048)
constexpr int CHA = 64;              // chunk length between TwoSum folds
constexpr int STA = 3;               // ring stages
constexpr int TQ = 256;              // query records per streamed query tile
constexpr uint32_t kQTileBytes = TQ * 16;  // (qx, qy, c, Z): one shared load per query
static_assert(kTB32 % CHA == 0 && TQ % CHA == 0, "chunks tile the streamed tiles");

struct AdjArgs {
  int64_t units;
  int grid;
  int64_t stream_tiles;  // streamed tiles per register tile
  const unsigned char* tiles;
  int64_t nreg;          // register-side points (m for the query sweep, n for the data sweep)
  int64_t nstream;       // streamed points (n, or m)
  const float* reg_xy;   // register-side coordinates
  int reg_stride;        // floats between consecutive points (2 queries, 3 data)
  const float* reg_val;  // Z_j (query sweep, stride 1) or z_i (data sweep, stride 3)
  int val_stride;
  const float* scales;
  float neg_half_p, neg_half_p1;  // -p/2, -(p/2 + 1)
  float2* partial;       // slots x 3 x RT (hi, lo)
  unsigned* err;
};

// w = (d^2)^(-p/2) and v = w / d^2 on both lanes; L = log2 d^2 when asked.
// No clamp on log2: the query sweep masks its padding records, and the data
// sweep's padding queries sit at a finite far point (weights underflow to 0).
template <bool POW2, bool WANT_L>
__device__ __forceinline__ void weights(u64 d2, u64 nhp2, u64 nhp12, u64& w, u64& v, u64& L) {
  float da, db;
  upk(d2, da, db);
  if (POW2) {
    w = pk(rcp_approx(da), rcp_approx(db));
    v = mul2(w, w);
    if (WANT_L) L = pk(lg2_approx(da), lg2_approx(db));
  } else {
    L = pk(lg2_approx(da), lg2_approx(db));
    float ta, tb, ua, ub;
    upk(mul2(L, nhp2), ta, tb);   // -(p/2) L
    upk(mul2(L, nhp12), ua, ub);  // -(p/2 + 1) L
    w = pk(ex2_approx(ta), ex2_approx(tb));
    v = pk(ex2_approx(ua), ex2_approx(ub));
  }
}

__device__ __forceinline__ void write_piece(float2* P, int comp, int idx, u64 hi, u64 lo) {
  float ha, hb, la, lb;
  upk(hi, ha, hb);
  upk(lo, la, lb);
  P[comp * RT + idx] = make_float2(ha, la);
  P[comp * RT + idx + NTA] = make_float2(hb, lb);
}

// One staged data tile for the query sweep.  MASKED (the last tile of a
// sweep only) skips the padding records; full tiles run straight-line code.
template <bool POW2, bool NEED_P, bool MASKED>
__device__ __forceinline__ void query_tile(const unsigned char* st, int valid, u64 NHP2, u64 NHP12,
                                           u64 SHIFT, const u64* QX, const u64* QY,
                                           const u64* ZQ, u64* XH, u64* XL, u64* YH, u64* YL,
                                           u64* PH, u64* PL) {
  const ulonglong2* XY = reinterpret_cast<const ulonglong2*>(st);
  const u64* ZZ = reinterpret_cast<const u64*>(st + kTB32 * 16);
#pragma unroll 1
  for (int c = 0; c < valid; c += CHA) {
    u64 CX[KPA], CY[KPA], CP[KPA];
#pragma unroll
    for (int k = 0; k < KPA; ++k) CX[k] = CY[k] = CP[k] = 0ull;
#pragma unroll
    for (int r = 0; r < CHA; ++r) {
      if (!MASKED || c + r < valid) {  // uniform across the CTA
        const ulonglong2 xy = XY[c + r];
        const u64 zz = ZZ[c + r];
#pragma unroll
        for (int k = 0; k < KPA; ++k) {
          const u64 dx = sub2f(QX[k], xy.x);
          const u64 dy = sub2f(QY[k], xy.y);
          const u64 d2 = fma2f(dy, dy, mul2f(dx, dx));
          u64 w, v, L = 0ull;
          weights<POW2, NEED_P>(d2, NHP2, NHP12, w, v, L);
          const u64 e = sub2(zz, ZQ[k]);  // z_i - Z_j
          const u64 ev = mul2(e, v);
          CX[k] = fma2(ev, dx, CX[k]);
          CY[k] = fma2(ev, dy, CY[k]);
          if (NEED_P) CP[k] = fma2(mul2(e, w), add2(L, SHIFT), CP[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < KPA; ++k) {
      two_sum_acc(XH[k], XL[k], CX[k]);
      two_sum_acc(YH[k], YL[k], CY[k]);
      if (NEED_P) two_sum_acc(PH[k], PL[k], CP[k]);
    }
  }
}

// Query sweep: sums over data points of (z - Z) w (q - x) / d^2 (x and y)
// and of (z - Z) w log2 d^2, per query, in scaled coordinates.
template <bool POW2, bool NEED_P>
__global__ void __launch_bounds__(NTA, 1) query_adj_kernel(const AdjArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long bars[STA];
  const int tid = threadIdx.x;
  const int64_t g = blockIdx.x;
  const int64_t u0 = unit_begin(g, a.units, a.grid);
  const int64_t total = unit_begin(g + 1, a.units, a.grid) - u0;
  if (total <= 0) return;
  auto src = [&](int64_t local) {
    return static_cast<const void*>(a.tiles + ((u0 + local) % a.stream_tiles) * kTileBytes32);
  };
  TileRing<STA, decltype(src)> ring{smem, bars, kTileBytes32, a.err, total, src, 0};
  ring.start();

  const float s = a.scales[0];
  const u64 NHP2 = pk(a.neg_half_p, a.neg_half_p), NHP12 = pk(a.neg_half_p1, a.neg_half_p1);
  // log2 of the unscaled d^2 = log2 of the scaled one - 2 log2 s (exact).
  const float shift = -2.f * static_cast<float>(ilogbf(s));
  const u64 SHIFT = pk(shift, shift);
  const int64_t last_valid = a.nstream - (a.stream_tiles - 1) * kTB32;  // records in last tile

  int64_t i = 0;
  bool aborted = false;
  while (i < total) {
    const int64_t rt = (u0 + i) / a.stream_tiles;
    const int64_t seg_end = min(total, (rt + 1) * a.stream_tiles - u0);
    u64 QX[KPA], QY[KPA], ZQ[KPA], XH[KPA], XL[KPA], YH[KPA], YL[KPA], PH[KPA], PL[KPA];
#pragma unroll
    for (int k = 0; k < KPA; ++k) {
      const int64_t ja = rt * RT + (2 * k) * NTA + tid, jb = ja + NTA;
      const bool va = ja < a.nreg, vb = jb < a.nreg;
      QX[k] = pk(va ? a.reg_xy[a.reg_stride * ja] * s : 0.f,
                 vb ? a.reg_xy[a.reg_stride * jb] * s : 0.f);
      QY[k] = pk(va ? a.reg_xy[a.reg_stride * ja + 1] * s : 0.f,
                 vb ? a.reg_xy[a.reg_stride * jb + 1] * s : 0.f);
      ZQ[k] = pk(va ? a.reg_val[a.val_stride * ja] : 0.f, vb ? a.reg_val[a.val_stride * jb] : 0.f);
      XH[k] = XL[k] = YH[k] = YL[k] = PH[k] = PL[k] = 0ull;
    }
    for (; i < seg_end; ++i) {
      bool ok;
      const unsigned char* st = ring.wait(i, ok);
      if (ok) {
        const bool last = ((u0 + i) % a.stream_tiles) == a.stream_tiles - 1;
        if (last && last_valid < kTB32)
          query_tile<POW2, NEED_P, true>(st, static_cast<int>(last_valid), NHP2, NHP12, SHIFT, QX,
                                         QY, ZQ, XH, XL, YH, YL, PH, PL);
        else
          query_tile<POW2, NEED_P, false>(st, kTB32, NHP2, NHP12, SHIFT, QX, QY, ZQ, XH, XL, YH,
                                          YL, PH, PL);
      }
      if (!ring.release(ok)) {
        aborted = true;
        break;
      }
    }
    if (aborted) break;
    float2* P = a.partial + (rt + g) * 3 * RT;
#pragma unroll
    for (int k = 0; k < KPA; ++k) {
      write_piece(P, 0, 2 * k * NTA + tid, XH[k], XL[k]);
      write_piece(P, 1, 2 * k * NTA + tid, YH[k], YL[k]);
      write_piece(P, 2, 2 * k * NTA + tid, PH[k], PL[k]);
    }
  }
  if (aborted) ring.drain(i);
}

// Data sweep: sums over queries of c w, c (z - Z) w (q - x) / d^2 (x and y)
// per data point, with c_j = g_j / S0_j (scaled), in scaled coordinates.
// Padding and excluded queries carry c = 0 at a finite far point.
template <bool POW2>
__global__ void __launch_bounds__(NTA, 1) data_adj_kernel(const AdjArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long bars[STA];
  const int tid = threadIdx.x;
  const int64_t g = blockIdx.x;
  const int64_t u0 = unit_begin(g, a.units, a.grid);
  const int64_t total = unit_begin(g + 1, a.units, a.grid) - u0;
  if (total <= 0) return;
  auto src = [&](int64_t local) {
    return static_cast<const void*>(a.tiles + ((u0 + local) % a.stream_tiles) * kQTileBytes);
  };
  TileRing<STA, decltype(src)> ring{smem, bars, kQTileBytes, a.err, total, src, 0};
  ring.start();
  const float s = a.scales[0];
  const u64 NHP2 = pk(a.neg_half_p, a.neg_half_p), NHP12 = pk(a.neg_half_p1, a.neg_half_p1);

  int64_t i = 0;
  bool aborted = false;
  while (i < total) {
    const int64_t rt = (u0 + i) / a.stream_tiles;
    const int64_t seg_end = min(total, (rt + 1) * a.stream_tiles - u0);
    u64 XD[KPA], YD[KPA], ZD[KPA], GZH[KPA], GZL[KPA], GXH[KPA], GXL[KPA], GYH[KPA], GYL[KPA];
#pragma unroll
    for (int k = 0; k < KPA; ++k) {
      const int64_t ia = rt * RT + (2 * k) * NTA + tid, ib = ia + NTA;
      const bool va = ia < a.nreg, vb = ib < a.nreg;
      XD[k] = pk(va ? a.reg_xy[a.reg_stride * ia] * s : 0.f,
                 vb ? a.reg_xy[a.reg_stride * ib] * s : 0.f);
      YD[k] = pk(va ? a.reg_xy[a.reg_stride * ia + 1] * s : 0.f,
                 vb ? a.reg_xy[a.reg_stride * ib + 1] * s : 0.f);
      ZD[k] = pk(va ? a.reg_val[a.val_stride * ia] : 0.f, vb ? a.reg_val[a.val_stride * ib] : 0.f);
      GZH[k] = GZL[k] = GXH[k] = GXL[k] = GYH[k] = GYL[k] = 0ull;
    }
    for (; i < seg_end; ++i) {
      bool ok;
      const unsigned char* st = ring.wait(i, ok);
      if (ok) {
        const float4* QR = reinterpret_cast<const float4*>(st);  // (qx, qy, c, Z)
#pragma unroll 1
        for (int c = 0; c < TQ; c += CHA) {
          u64 CGZ[KPA], CGX[KPA], CGY[KPA];
#pragma unroll
          for (int k = 0; k < KPA; ++k) CGZ[k] = CGX[k] = CGY[k] = 0ull;
#pragma unroll
          for (int r = 0; r < CHA; ++r) {
            const float4 qr = QR[c + r];
            const u64 qxx = pk(qr.x, qr.x), qyy = pk(qr.y, qr.y);
            const u64 cc = pk(qr.z, qr.z), zq = pk(qr.w, qr.w);
#pragma unroll
            for (int k = 0; k < KPA; ++k) {
              const u64 dx = sub2f(qxx, XD[k]);  // q_j - x_i
              const u64 dy = sub2f(qyy, YD[k]);
              const u64 d2 = fma2f(dy, dy, mul2f(dx, dx));
              u64 w, v, L;
              weights<POW2, false>(d2, NHP2, NHP12, w, v, L);
              const u64 cw = mul2(cc, w);
              CGZ[k] = add2(CGZ[k], cw);
              const u64 b = mul2(mul2(cc, sub2(ZD[k], zq)), v);  // c (z_i - Z_j) w / d^2
              CGX[k] = fma2(b, dx, CGX[k]);
              CGY[k] = fma2(b, dy, CGY[k]);
            }
          }
#pragma unroll
          for (int k = 0; k < KPA; ++k) {
            two_sum_acc(GZH[k], GZL[k], CGZ[k]);
            two_sum_acc(GXH[k], GXL[k], CGX[k]);
            two_sum_acc(GYH[k], GYL[k], CGY[k]);
          }
        }
      }
      if (!ring.release(ok)) {
        aborted = true;
        break;
      }
    }
    if (aborted) break;
    float2* P = a.partial + (rt + g) * 3 * RT;
#pragma unroll
    for (int k = 0; k < KPA; ++k) {
      write_piece(P, 0, 2 * k * NTA + tid, GZH[k], GZL[k]);
      write_piece(P, 1, 2 * k * NTA + tid, GXH[k], GXL[k]);
      write_piece(P, 2, 2 * k * NTA + tid, GYH[k], GYL[k]);
    }
  }
  if (aborted) ring.drain(i);
}

// Streamed query records of the data sweep: (s qx, s qy, c, Z) with
// c = g / S0_scaled (tiles of TQ records are consecutive).  Excluded and padding queries sit at a
// far finite point with c = 0.
__global__ void __launch_bounds__(256)
    stage_queries_kernel(const float* __restrict__ queries, int64_t m, int64_t records,
                         const float* __restrict__ Z, const double* __restrict__ s0,
                         const int32_t* __restrict__ hit, const float* __restrict__ g,
                         const float* __restrict__ scales, double p,
                         unsigned char* __restrict__ tiles) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= records) return;
  const float s = scales[0];
  float qx = kPadPow2, qy = kPadPow2, c = 0.f, z = 0.f;
  if (j < m && hit[j] == kNoHit) {
    qx = queries[2 * j] * s;
    qy = queries[2 * j + 1] * s;
    // S0 of the scaled coordinates is S0 s^-p.
    c = static_cast<float>(double(g[j]) * pow(double(s), p) / s0[j]);
    z = Z[j];
  }
  reinterpret_cast<float4*>(tiles)[j] = make_float4(qx, qy, c, z);
}

__device__ __forceinline__ void piece_range(int64_t rt, int64_t stream_tiles, int64_t units,
                                            int grid, int64_t& g0, int64_t& g1) {
  g0 = cta_of_unit(rt * stream_tiles, units, grid);
  g1 = cta_of_unit((rt + 1) * stream_tiles - 1, units, grid);
}

__global__ void __launch_bounds__(256)
    query_combine_kernel(const float2* __restrict__ partial, int64_t m, int64_t stream_tiles,
                         int64_t units, int grid, const float* __restrict__ g,
                         const double* __restrict__ s0, const int32_t* __restrict__ hit,
                         const float* __restrict__ scales, double p,
                         float* __restrict__ grad_q, double* __restrict__ gp,
                         Control* __restrict__ ctrl, int32_t* __restrict__ list) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= m) return;
  if (hit[j] != kNoHit) {  // exact hits: 0; FP64 queries: written by the fix-up
    if (grad_q) grad_q[2 * j] = grad_q[2 * j + 1] = 0.f;
    gp[j] = 0.0;
    return;
  }
  const int64_t rt = j / RT, lq = j % RT;
  int64_t g0, g1;
  piece_range(rt, stream_tiles, units, grid, g0, g1);
  double ax = 0.0, ay = 0.0, ap = 0.0;
  for (int64_t q = g0; q <= g1; ++q) {
    const float2* P = partial + (rt + q) * 3 * RT;
    ax += double(P[lq].x) + double(P[lq].y);
    ay += double(P[RT + lq].x) + double(P[RT + lq].y);
    ap += double(P[2 * RT + lq].x) + double(P[2 * RT + lq].y);
  }
  if (!isfinite(ax) || !isfinite(ay) || !isfinite(ap)) {
    // A pair too close for FP32's range of w / d^2: redo this query's
    // query-side sums in FP64 (its data-side terms are fine).
    list[atomicAdd(&ctrl->flagged, 1u)] = static_cast<int32_t>(-(j + 1));
    return;
  }
  const double sc = scales[0];
  const double s0s = s0[j] * pow(sc, -p);  // S0 of the scaled coordinates
  const double gj = g[j];
  if (grad_q) {
    // d/dq of the unscaled problem = s x d/dq of the scaled one.
    grad_q[2 * j] = static_cast<float>(-gj * p * sc * ax / s0s);
    grad_q[2 * j + 1] = static_cast<float>(-gj * p * sc * ay / s0s);
  }
  gp[j] = -gj * 0.6931471805599453 * ap / (2.0 * s0s);
}

__global__ void __launch_bounds__(256)
    data_combine_kernel(const float2* __restrict__ partial, int64_t n, int64_t stream_tiles,
                        int64_t units, int grid, const float* __restrict__ scales, double p,
                        float* __restrict__ grad_z, float* __restrict__ grad_xy,
                        unsigned* __restrict__ dcount, int32_t* __restrict__ dlist) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t rt = i / RT, li = i % RT;
  int64_t g0, g1;
  piece_range(rt, stream_tiles, units, grid, g0, g1);
  double gz = 0.0, gx = 0.0, gy = 0.0;
  for (int64_t q = g0; q <= g1; ++q) {
    const float2* P = partial + (rt + q) * 3 * RT;
    gz += double(P[li].x) + double(P[li].y);
    gx += double(P[RT + li].x) + double(P[RT + li].y);
    gy += double(P[2 * RT + li].x) + double(P[2 * RT + li].y);
  }
  if (!isfinite(gz) || !isfinite(gx) || !isfinite(gy)) {
    dlist[atomicAdd(dcount, 1u)] = static_cast<int32_t>(i);  // recomputed in FP64
    return;
  }
  const double sc = scales[0];
  if (grad_z) grad_z[i] = static_cast<float>(gz);
  if (grad_xy) {
    grad_xy[2 * i] = static_cast<float>(p * sc * gx);
    grad_xy[2 * i + 1] = static_cast<float>(p * sc * gy);
  }
}

// Queries the forward pass did not take the fast path for: exact hits add
// g_j to dL/dz_k; FP64-recomputed queries are listed for the FP64 kernel.
__global__ void __launch_bounds__(256)
    fixup_scan_kernel(int64_t m, const int32_t* __restrict__ hit, const float* __restrict__ g,
                      float* __restrict__ grad_z, Control* __restrict__ ctrl,
                      int32_t* __restrict__ list) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int32_t h = hit[j];
  if (h >= 0) {
    if (grad_z) atomicAdd(&grad_z[h], g[j]);
  } else if (h == kRecomputedF64) {
    list[atomicAdd(&ctrl->flagged, 1u)] = static_cast<int32_t>(j);
  }
}

// Gradient contribution of one listed query in FP64 (unscaled data,
// weights scaled by d2_min^(p/2), which cancels in every ratio).
__global__ void __launch_bounds__(kSlowThreads)
    slow_grad_kernel(const float* __restrict__ data, int64_t n, const float* __restrict__ queries,
                     double p, const float* __restrict__ g, const Control* __restrict__ ctrl,
                     const int32_t* __restrict__ list, float* __restrict__ grad_z,
                     float* __restrict__ grad_xy, float* __restrict__ grad_q,
                     double* __restrict__ gp) {
  __shared__ double red[kSlowThreads / 32];
  const unsigned count = ctrl->flagged;
  for (unsigned f = blockIdx.x; f < count; f += gridDim.x) {
    // e >= 0: query excluded from the data sweep (all its terms here);
    // e < 0: query -e-1 whose query-side sums left FP32's range.
    const int64_t e_ = list[f];
    const bool full = e_ >= 0;
    const int64_t j = full ? e_ : -e_ - 1;
    const double qx = queries[2 * j], qy = queries[2 * j + 1], gj = g[j];
    double dmin = INFINITY;
    for (int64_t i = threadIdx.x; i < n; i += kSlowThreads) {
      const double dx = qx - data[3 * i], dy = qy - data[3 * i + 1];
      dmin = fmin(dmin, dx * dx + dy * dy);
    }
    dmin = block_reduce<double>(dmin, red, true);
    double s0 = 0.0, s1 = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kSlowThreads) {
      const double dx = qx - data[3 * i], dy = qy - data[3 * i + 1];
      const double w = pow(dmin / (dx * dx + dy * dy), 0.5 * p);
      s0 += w;
      s1 += w * data[3 * i + 2];
    }
    s0 = block_reduce<double>(s0, red, false);
    s1 = block_reduce<double>(s1, red, false);
    const double Z = s1 / s0;
    double ax = 0.0, ay = 0.0, ap = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kSlowThreads) {
      const double dx = qx - data[3 * i], dy = qy - data[3 * i + 1];
      const double d2 = dx * dx + dy * dy;
      const double w = pow(dmin / d2, 0.5 * p);
      const double e = (data[3 * i + 2] - Z) * w;
      ax += e * dx / d2;
      ay += e * dy / d2;
      ap += e * log(d2);
      if (full && grad_z) atomicAdd(&grad_z[i], static_cast<float>(gj * w / s0));
      if (full && grad_xy) {
        const double b = gj * p * e / (s0 * d2);
        atomicAdd(&grad_xy[2 * i], static_cast<float>(b * dx));
        atomicAdd(&grad_xy[2 * i + 1], static_cast<float>(b * dy));
      }
    }
    ax = block_reduce<double>(ax, red, false);
    ay = block_reduce<double>(ay, red, false);
    ap = block_reduce<double>(ap, red, false);
    if (threadIdx.x == 0) {
      if (grad_q) {
        grad_q[2 * j] = static_cast<float>(-gj * p * ax / s0);
        grad_q[2 * j + 1] = static_cast<float>(-gj * p * ay / s0);
      }
      gp[j] = -gj * ap / (2.0 * s0);
    }
  }
}

// Data points whose FP32 sums left FP32's range: their sums over the queries
// of the data sweep, in FP64 with the saved S0 and Z.
__global__ void __launch_bounds__(kSlowThreads)
    slow_data_kernel(const float* __restrict__ data, const float* __restrict__ queries,
                     int64_t m, double p, const float* __restrict__ Z,
                     const double* __restrict__ s0, const int32_t* __restrict__ hit,
                     const float* __restrict__ g, const unsigned* __restrict__ dcount,
                     const int32_t* __restrict__ dlist, float* __restrict__ grad_z,
                     float* __restrict__ grad_xy) {
  __shared__ double red[kSlowThreads / 32];
  const unsigned count = *dcount;
  for (unsigned f = blockIdx.x; f < count; f += gridDim.x) {
    const int64_t i = dlist[f];
    const double x = data[3 * i], y = data[3 * i + 1], z = data[3 * i + 2];
    double gz = 0.0, gx = 0.0, gy = 0.0;
    for (int64_t j = threadIdx.x; j < m; j += kSlowThreads) {
      if (hit[j] != kNoHit) continue;
      const double dx = double(queries[2 * j]) - x, dy = double(queries[2 * j + 1]) - y;
      const double d2 = dx * dx + dy * dy;
      const double w = pow(d2, -0.5 * p);
      const double c = double(g[j]) / s0[j];
      gz += c * w;
      const double b = c * p * (z - double(Z[j])) * w / d2;
      gx += b * dx;
      gy += b * dy;
    }
    gz = block_reduce<double>(gz, red, false);
    gx = block_reduce<double>(gx, red, false);
    gy = block_reduce<double>(gy, red, false);
    if (threadIdx.x == 0) {
      if (grad_z) grad_z[i] = static_cast<float>(gz);
      if (grad_xy) {
        grad_xy[2 * i] = static_cast<float>(gx);
        grad_xy[2 * i + 1] = static_cast<float>(gy);
      }
    }
  }
}

// dL/dp = sum_j gp[j], in a fixed order (one CTA).
__global__ void __launch_bounds__(1024)
    reduce_p_kernel(const double* __restrict__ gp, int64_t m, double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) acc += gp[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) *out = acc;
  }
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

template <class K>
int occupancy_of(K kernel, size_t smem) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, NTA, smem);
  return b > 0 ? b : 1;
}

}  // namespace

void plan_backward_f32(int64_t n, int64_t m, int sm_count, int ctas_per_sm, BwdPlan* bp) {
  bp->data_tiles = (n + kTB32 - 1) / kTB32;
  bp->query_records_tiles = (m + TQ - 1) / TQ;
  bp->query_reg_tiles = (m + RT - 1) / RT;
  bp->data_reg_tiles = (n + RT - 1) / RT;
  bp->units_q = bp->query_reg_tiles * bp->data_tiles;
  bp->units_d = bp->data_reg_tiles * bp->query_records_tiles;
  const int64_t resident = int64_t(sm_count) * std::max(1, ctas_per_sm);
  bp->grid_q = static_cast<int>(std::max<int64_t>(1, std::min(bp->units_q, resident)));
  bp->grid_d = static_cast<int>(std::max<int64_t>(1, std::min(bp->units_d, resident)));
  bp->staged_bytes = round_up(size_t(bp->data_tiles) * kTileBytes32, 256);
  bp->qtiles_bytes = round_up(size_t(bp->query_records_tiles) * kQTileBytes, 256);
  const size_t slots = size_t(std::max(bp->query_reg_tiles + bp->grid_q - 1,
                                       bp->data_reg_tiles + bp->grid_d - 1));
  bp->partial_bytes = round_up(slots * 3 * RT * sizeof(float2), 256);
  bp->gp_bytes = round_up(size_t(m) * sizeof(double), 256);
  bp->list_bytes = round_up(size_t(m) * sizeof(int32_t), 256);
  bp->dlist_bytes = round_up(size_t(n) * sizeof(int32_t), 256);
  bp->scale_bytes = 256;
  bp->workspace_bytes = bp->staged_bytes + bp->qtiles_bytes + bp->partial_bytes + bp->gp_bytes +
                        bp->list_bytes + bp->dlist_bytes + bp->scale_bytes;
}

int occupancy_backward_f32() {
  return std::min(occupancy_of(query_adj_kernel<false, true>, size_t(STA) * kTileBytes32),
                  occupancy_of(data_adj_kernel<false>, size_t(STA) * kQTileBytes));
}

cudaError_t launch_backward_f32(const BwdProblem& pb, const BwdPlan& bp, void* workspace,
                                Control* ctrl, int sm_count, cudaStream_t stream) {
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  unsigned char* dtiles = ws;
  unsigned char* qtiles = ws + bp.staged_bytes;
  float2* partial = reinterpret_cast<float2*>(qtiles + bp.qtiles_bytes);
  double* gp = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(partial) +
                                         bp.partial_bytes);
  int32_t* list = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(gp) + bp.gp_bytes);
  int32_t* dlist =
      reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(list) + bp.list_bytes);
  unsigned* maxbits = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(dlist) +
                                                  bp.dlist_bytes);
  float* scales = reinterpret_cast<float*>(maxbits + 1);
  unsigned* dcount = maxbits + 2;
  const bool pow2 = pb.p == 2.0;
  const bool need_q = pb.grad_q || pb.grad_p;
  const bool need_d = pb.grad_z || pb.grad_xy;

  Table<1> t;
  t.count = 1;
  t.pad = 0;
  Instance& I = t.inst[0];
  I.data = pb.data;
  I.queries = pb.queries;
  I.out = nullptr;
  I.s0_out = nullptr;
  I.hit_out = nullptr;
  I.tiles = dtiles;
  I.unit_base = 0;
  I.record_base = 0;
  I.n = static_cast<int32_t>(pb.n);
  I.m = static_cast<int32_t>(pb.m);
  I.data_tiles = static_cast<int32_t>(bp.data_tiles);
  I.qtile_base = 0;

  cudaError_t e = cudaMemsetAsync(maxbits, 0, 3 * sizeof(unsigned), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(&ctrl->flagged, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  const int64_t longest = std::max(pb.n, pb.m);
  const unsigned gx = static_cast<unsigned>(std::min<int64_t>(1024, (longest + 255) / 256));
  range_kernel<1><<<dim3(gx, 1), 256, 0, stream>>>(t, maxbits);
  // Data tiles with finite far padding (both weight forms); the query sweep
  // masks the padding of its last tile, and products with it stay finite.
  const int64_t records = bp.data_tiles * kTB32;
  stage_kernel<1, kPow2><<<static_cast<unsigned>((records + 255) / 256), 256, 0, stream>>>(
      t, records, maxbits, scales);

  AdjArgs a;
  a.scales = scales;
  a.neg_half_p = static_cast<float>(-0.5 * pb.p);
  a.neg_half_p1 = static_cast<float>(-0.5 * pb.p - 1.0);
  a.partial = partial;
  a.err = &ctrl->error;

  if (need_q) {
    a.units = bp.units_q;
    a.grid = bp.grid_q;
    a.stream_tiles = bp.data_tiles;
    a.tiles = dtiles;
    a.nreg = pb.m;
    a.nstream = pb.n;
    a.reg_xy = pb.queries;
    a.reg_stride = 2;
    a.reg_val = pb.Z;
    a.val_stride = 1;
    const size_t smem = size_t(STA) * kTileBytes32;
    if (pow2) {
      if (pb.grad_p)
        query_adj_kernel<true, true><<<bp.grid_q, NTA, smem, stream>>>(a);
      else
        query_adj_kernel<true, false><<<bp.grid_q, NTA, smem, stream>>>(a);
    } else {
      query_adj_kernel<false, true><<<bp.grid_q, NTA, smem, stream>>>(a);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    query_combine_kernel<<<static_cast<unsigned>((pb.m + 255) / 256), 256, 0, stream>>>(
        partial, pb.m, bp.data_tiles, bp.units_q, bp.grid_q, pb.g, pb.s0, pb.hit, scales, pb.p,
        pb.grad_q, gp, ctrl, list);
  }
  if (need_d) {
    const int64_t qrec = bp.query_records_tiles * TQ;
    stage_queries_kernel<<<static_cast<unsigned>((qrec + 255) / 256), 256, 0, stream>>>(
        pb.queries, pb.m, qrec, pb.Z, pb.s0, pb.hit, pb.g, scales, pb.p, qtiles);
    a.units = bp.units_d;
    a.grid = bp.grid_d;
    a.stream_tiles = bp.query_records_tiles;
    a.tiles = qtiles;
    a.nreg = pb.n;
    a.nstream = pb.m;
    a.reg_xy = pb.data;
    a.reg_stride = 3;
    a.reg_val = pb.data + 2;
    a.val_stride = 3;
    const size_t smem = size_t(STA) * kQTileBytes;
    if (pow2)
      data_adj_kernel<true><<<bp.grid_d, NTA, smem, stream>>>(a);
    else
      data_adj_kernel<false><<<bp.grid_d, NTA, smem, stream>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    data_combine_kernel<<<static_cast<unsigned>((pb.n + 255) / 256), 256, 0, stream>>>(
        partial, pb.n, bp.query_records_tiles, bp.units_d, bp.grid_d, scales, pb.p, pb.grad_z,
        pb.grad_xy, dcount, dlist);
    slow_data_kernel<<<2 * sm_count, kSlowThreads, 0, stream>>>(
        pb.data, pb.queries, pb.m, pb.p, pb.Z, pb.s0, pb.hit, pb.g, dcount, dlist, pb.grad_z,
        pb.grad_xy);
  }
  fixup_scan_kernel<<<static_cast<unsigned>((pb.m + 255) / 256), 256, 0, stream>>>(
      pb.m, pb.hit, pb.g, pb.grad_z, ctrl, list);
  slow_grad_kernel<<<2 * sm_count, kSlowThreads, 0, stream>>>(
      pb.data, pb.n, pb.queries, pb.p, pb.g, ctrl, list, pb.grad_z, pb.grad_xy, pb.grad_q, gp);
  if (pb.grad_p) reduce_p_kernel<<<1, 1024, 0, stream>>>(gp, pb.m, pb.grad_p);
  return cudaGetLastError();
}

}  // namespace idw
