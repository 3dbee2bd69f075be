// The paper's own GPU designs for Eq. 1, built on sm_103a as measured
// baselines in the paper's data layouts (Sec. 2.2 and Sec. 3.2-3.5):
//   naive : one thread per prediction point, reading every data point from
//           global memory, so the data are read m times (Sec. 3, Sec. 4.2);
//   tiled : one thread per prediction point; a block stages blockDim data
//           points in shared memory, then every thread sweeps them, so the
//           data are read m / blockDim times (Sec. 4.2).
// Both sum plainly in the kernel's precision (float or double); p = 2 is
// 1/d^2, other p use pow().  A query that coincides with a data point takes
// the z of the lowest such index (the library's reading of d = 0).
//
// Layouts of the n data points (user rows are staged into them first):
//   SoA    : x[n], y[n], z[n]
//   AoS    : rows (x, y, z) without alignment (12 or 24 bytes)
//   AoaS   : aligned records (x, y, z, pad) (16 or 32 bytes)
//   Hybrid : (x, y) pairs beside z[n] (double only in the paper, Sec. 3.5)
#include <cmath>
#include <cstdint>

#include "idw.h"
#include "idw_internal.h"

namespace idw {
namespace {

constexpr int kPaperThreads = 256;

// The aligned record of the AoaS layout: (x, y, z, pad), 16 or 32 bytes.
struct __align__(16) Rec4f { float x, y, z, w; };
struct __align__(32) Rec4d { double x, y, z, w; };
template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef Rec4f type; };
template <> struct Vec4<double> { typedef Rec4d type; };
template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float2 type; };
template <> struct Vec2<double> { typedef double2 type; };

// Reads data point i of a staged layout.
template <typename T, int LAYOUT>
__device__ __forceinline__ void point_at(const unsigned char* base, int64_t n, int64_t i, T& x,
                                         T& y, T& z) {
  if (LAYOUT == IDW_LAYOUT_SOA) {
    const T* a = reinterpret_cast<const T*>(base);
    x = a[i];
    y = a[n + i];
    z = a[2 * n + i];
  } else if (LAYOUT == IDW_LAYOUT_AOS) {
    const T* a = reinterpret_cast<const T*>(base);
    x = a[3 * i];
    y = a[3 * i + 1];
    z = a[3 * i + 2];
  } else if (LAYOUT == IDW_LAYOUT_AOAS) {
    const typename Vec4<T>::type v = reinterpret_cast<const typename Vec4<T>::type*>(base)[i];
    x = v.x;
    y = v.y;
    z = v.z;
  } else {
    const typename Vec2<T>::type v = reinterpret_cast<const typename Vec2<T>::type*>(base)[i];
    x = v.x;
    y = v.y;
    z = reinterpret_cast<const T*>(base + size_t(n) * sizeof(typename Vec2<T>::type))[i];
  }
}

template <typename T>
__device__ __forceinline__ void accumulate(T qx, T qy, T x, T y, T z, int64_t i, double p,
                                           bool pow2, T& s0, T& s1, int64_t& hit) {
  const T dx = qx - x, dy = qy - y;
  const T d2 = dx * dx + dy * dy;
  if (d2 == T(0)) {
    if (hit < 0 || i < hit) hit = i;
    return;
  }
  const T w = pow2 ? T(1) / d2 : T(pow(double(d2), -0.5 * p));
  s0 += w;
  s1 += w * z;
}

template <typename T, int LAYOUT>
__global__ void __launch_bounds__(kPaperThreads)
    naive_kernel(const unsigned char* __restrict__ data, int64_t n, const T* __restrict__ queries,
                 int64_t m, double p, T* __restrict__ out) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const T qx = queries[2 * j], qy = queries[2 * j + 1];
  const bool pow2 = p == 2.0;
  T s0 = 0, s1 = 0;
  int64_t hit = -1;
  for (int64_t i = 0; i < n; ++i) {
    T x, y, z;
    point_at<T, LAYOUT>(data, n, i, x, y, z);
    accumulate(qx, qy, x, y, z, i, p, pow2, s0, s1, hit);
  }
  if (hit >= 0) {
    T x, y, z;
    point_at<T, LAYOUT>(data, n, hit, x, y, z);
    out[j] = z;
  } else {
    out[j] = s1 / s0;
  }
}

template <typename T, int LAYOUT>
__global__ void __launch_bounds__(kPaperThreads)
    tiled_kernel(const unsigned char* __restrict__ data, int64_t n, const T* __restrict__ queries,
                 int64_t m, double p, T* __restrict__ out) {
  // One tile of blockDim points in the same layout as global memory.
  constexpr int kTileBytes = LAYOUT == IDW_LAYOUT_AOAS ? kPaperThreads * 4 * sizeof(T)
                                                       : kPaperThreads * 3 * sizeof(T);
  __shared__ __align__(32) unsigned char tile[kTileBytes];
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool active = j < m;
  const T qx = active ? queries[2 * j] : T(0), qy = active ? queries[2 * j + 1] : T(0);
  const bool pow2 = p == 2.0;
  T s0 = 0, s1 = 0;
  int64_t hit = -1;
  for (int64_t b = 0; b < n; b += kPaperThreads) {
    const int count = static_cast<int>(n - b < kPaperThreads ? n - b : kPaperThreads);
    if (threadIdx.x < count) {
      T x, y, z;
      point_at<T, LAYOUT>(data, n, b + threadIdx.x, x, y, z);
      const int t = threadIdx.x;
      if (LAYOUT == IDW_LAYOUT_SOA) {
        T* s = reinterpret_cast<T*>(tile);
        s[t] = x;
        s[kPaperThreads + t] = y;
        s[2 * kPaperThreads + t] = z;
      } else if (LAYOUT == IDW_LAYOUT_AOS) {
        T* s = reinterpret_cast<T*>(tile);
        s[3 * t] = x;
        s[3 * t + 1] = y;
        s[3 * t + 2] = z;
      } else if (LAYOUT == IDW_LAYOUT_AOAS) {
        typename Vec4<T>::type v;
        v.x = x;
        v.y = y;
        v.z = z;
        v.w = T(0);
        reinterpret_cast<typename Vec4<T>::type*>(tile)[t] = v;
      } else {
        typename Vec2<T>::type v;
        v.x = x;
        v.y = y;
        reinterpret_cast<typename Vec2<T>::type*>(tile)[t] = v;
        reinterpret_cast<T*>(tile + kPaperThreads * sizeof(typename Vec2<T>::type))[t] = z;
      }
    }
    __syncthreads();
    for (int r = 0; r < count; ++r) {
      T x, y, z;
      point_at<T, LAYOUT>(tile, kPaperThreads, r, x, y, z);
      accumulate(qx, qy, x, y, z, b + r, p, pow2, s0, s1, hit);
    }
    __syncthreads();
  }
  if (!active) return;
  if (hit >= 0) {
    T x, y, z;
    point_at<T, LAYOUT>(data, n, hit, x, y, z);
    out[j] = z;
  } else {
    out[j] = s1 / s0;
  }
}

// User rows (x, y, z) -> the requested layout.
template <typename T, int LAYOUT>
__global__ void stage_layout_kernel(const T* __restrict__ rows, int64_t n,
                                    unsigned char* __restrict__ dst) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T x = rows[3 * i], y = rows[3 * i + 1], z = rows[3 * i + 2];
  if (LAYOUT == IDW_LAYOUT_SOA) {
    T* a = reinterpret_cast<T*>(dst);
    a[i] = x;
    a[n + i] = y;
    a[2 * n + i] = z;
  } else if (LAYOUT == IDW_LAYOUT_AOAS) {
    typename Vec4<T>::type v;
    v.x = x;
    v.y = y;
    v.z = z;
    v.w = T(0);
    reinterpret_cast<typename Vec4<T>::type*>(dst)[i] = v;
  } else if (LAYOUT == IDW_LAYOUT_HYBRID) {
    typename Vec2<T>::type v;
    v.x = x;
    v.y = y;
    reinterpret_cast<typename Vec2<T>::type*>(dst)[i] = v;
    reinterpret_cast<T*>(dst + size_t(n) * sizeof(typename Vec2<T>::type))[i] = z;
  }
}

template <typename T, int LAYOUT>
cudaError_t run_layout(int kernel, const T* rows, int64_t n, const T* queries, int64_t m, double p,
                       T* out, unsigned char* ws, cudaStream_t s) {
  const unsigned char* data = reinterpret_cast<const unsigned char*>(rows);
  if (LAYOUT != IDW_LAYOUT_AOS) {  // user rows already are the unaligned AoS layout
    stage_layout_kernel<T, LAYOUT><<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(rows, n,
                                                                                           ws);
    data = ws;
  }
  const unsigned grid = static_cast<unsigned>((m + kPaperThreads - 1) / kPaperThreads);
  if (kernel == IDW_PAPER_NAIVE)
    naive_kernel<T, LAYOUT><<<grid, kPaperThreads, 0, s>>>(data, n, queries, m, p, out);
  else
    tiled_kernel<T, LAYOUT><<<grid, kPaperThreads, 0, s>>>(data, n, queries, m, p, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_typed(int kernel, int layout, const T* rows, int64_t n, const T* queries,
                      int64_t m, double p, T* out, unsigned char* ws, cudaStream_t s) {
  switch (layout) {
    case IDW_LAYOUT_SOA: return run_layout<T, IDW_LAYOUT_SOA>(kernel, rows, n, queries, m, p, out, ws, s);
    case IDW_LAYOUT_AOS: return run_layout<T, IDW_LAYOUT_AOS>(kernel, rows, n, queries, m, p, out, ws, s);
    case IDW_LAYOUT_AOAS: return run_layout<T, IDW_LAYOUT_AOAS>(kernel, rows, n, queries, m, p, out, ws, s);
    default: return run_layout<T, IDW_LAYOUT_HYBRID>(kernel, rows, n, queries, m, p, out, ws, s);
  }
}

}  // namespace

size_t paper_layout_bytes(int64_t n, bool fp64) {
  return size_t(n) * (fp64 ? 32 : 16) + 256;  // the widest layout (AoaS)
}

cudaError_t launch_paper_kernel(int kernel, int layout, bool fp64, const void* rows, int64_t n,
                                const void* queries, int64_t m, double p, void* out,
                                void* workspace, cudaStream_t stream) {
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  if (fp64)
    return run_typed<double>(kernel, layout, static_cast<const double*>(rows), n,
                             static_cast<const double*>(queries), m, p,
                             static_cast<double*>(out), ws, stream);
  return run_typed<float>(kernel, layout, static_cast<const float*>(rows), n,
                          static_cast<const float*>(queries), m, p, static_cast<float*>(out), ws,
                          stream);
}

}  // namespace idw
