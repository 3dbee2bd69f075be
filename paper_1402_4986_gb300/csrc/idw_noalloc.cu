// Allocation-free variant of the FP32-compensated forward pass.
//
// Some callers cannot allocate device memory: a host application that owns
// the whole device-memory budget and forbids its plug-ins to allocate, or a
// latency-critical loop that cannot afford cudaMalloc/cudaFree, which
// synchronise the device.  Such callers cannot create a handle either
// (idw_create allocates), so this entry point takes none.  Its scratch (the
// staged data tiles, the per-piece partial sums, the list of queries routed
// to the slow path and the control words) lives in one file-scope device
// array of fixed size; the caller still passes the inputs and the output.
//
// The array name below is a host-side stand-in in host code, not a device
// address: set-up asks the runtime for the real address once per device,
// with that device current, and passes that address to the kernels.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "idw.h"
#include "idw_internal.h"

namespace idw {
namespace {

// 32 MiB of scratch, held by every GPU that loads this module until exit.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr size_t kControlBytes = (sizeof(Control) + 255) / 256 * 256;  // padded to keep alignment
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
  bool ready = false;
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
  int sm_count = 0;
  int occ[2][kNumSweepVariants] = {};  // resident CTAs per SM: [general p][variant]
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

// Once per device, with that device current: resolve the array's device
// address, query the SM count and the occupancy of every sweep variant, and
// zero the control words.  The clear is waited for (cudaDeviceSynchronize),
// so no later call on any stream can overtake it.
idw_status setup_current_device(DeviceSetup* out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return IDW_ERR_CUDA;
  if (dev >= kMaxDevices) return IDW_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
      return IDW_ERR_CUDA;
    if (major != 10 || minor != 3) return IDW_ERR_UNSUPPORTED;
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr)
      return IDW_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return IDW_ERR_CUDA;
    if (cudaMemset(ptr, 0, kControlBytes) != cudaSuccess) return IDW_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return IDW_ERR_CUDA;
    s.scratch = static_cast<unsigned char*>(ptr);
    s.sm_count = sms;
    for (int g = 0; g < 2; ++g)
      for (int v = 0; v < kNumSweepVariants; ++v)
        if (resolve_sweep_variant(v, g != 0) == v) s.occ[g][v] = occupancy_forward_f32(g != 0, v);
    s.ready = true;
  }
  *out = s;
  return IDW_OK;
}

}  // namespace
}  // namespace idw

extern "C" idw_status idw_interpolate_noalloc(const float* data_xyz, int64_t n,
                                              const float* queries_xy, int64_t m, double p,
                                              float* out, void* stream) {
  using namespace idw;
  if (n < 1 || n >= (int64_t(1) << 31) || m < 0 || m >= (int64_t(1) << 31)) return IDW_ERR_INVALID_ARG;
  if (!(p > 0.0) || !(p < INFINITY)) return IDW_ERR_INVALID_ARG;
  if (m == 0) return IDW_OK;
  if (!data_xyz || !queries_xy || !out) return IDW_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(data_xyz) | reinterpret_cast<uintptr_t>(queries_xy) |
       reinterpret_cast<uintptr_t>(out)) % 4 != 0)
    return IDW_ERR_ALIGNMENT;

  DeviceSetup dev;
  idw_status st = setup_current_device(&dev);
  if (st != IDW_OK) return st;

  // The same launch plan as idw_interpolate without tuning (host arithmetic
  // only): the default sweep variant for this size and weight form.
  const bool general = p != 2.0;
  F32Problem pb{data_xyz, n, queries_xy, m, out, nullptr, nullptr};
  const int variant =
      resolve_sweep_variant(default_sweep_variant(&pb, 1, general, dev.sm_count), general);
  BatchPlan plan;
  plan_batch_f32(&pb, 1, dev.sm_count, dev.occ[general ? 1 : 0][variant], variant, &plan);
  if (plan.workspace_bytes > kNoAllocScratchBytes - kControlBytes) return IDW_ERR_WORKSPACE;

  Control* ctrl = reinterpret_cast<Control*>(dev.scratch);
  const cudaError_t e = launch_batch_f32(&pb, plan, p, dev.scratch + kControlBytes, ctrl,
                                         dev.sm_count, nullptr, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? IDW_OK : IDW_ERR_CUDA;
}

// The device-side outcome of earlier idw_interpolate_noalloc calls on the
// current device: waits for `stream`, then reads the sticky error bits of the
// shared control words (a bounded wait inside a sweep that gave up sets
// them; the call that hit it produced no valid output) and clears them.
extern "C" idw_status idw_noalloc_sync_status(void* stream) {
  using namespace idw;
  DeviceSetup dev;
  idw_status st = setup_current_device(&dev);
  if (st != IDW_OK) return st;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return IDW_ERR_CUDA;
  Control* ctrl = reinterpret_cast<Control*>(dev.scratch);
  Control c;
  if (cudaMemcpy(&c, ctrl, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return IDW_ERR_CUDA;
  if (c.error == 0) return IDW_OK;
  if (cudaMemset(&ctrl->error, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess)
    return IDW_ERR_CUDA;
  return IDW_ERR_DEVICE_TIMEOUT;
}

// Failure-detection self-test of the allocation-free path: one bounded wait
// on a barrier nothing completes, reporting into the shared control words,
// so that idw_noalloc_sync_status has a timeout to find.
extern "C" idw_status idw_noalloc_selftest_bounded_wait(void* stream) {
  using namespace idw;
  DeviceSetup dev;
  idw_status st = setup_current_device(&dev);
  if (st != IDW_OK) return st;
  const cudaError_t e = launch_bounded_wait_selftest(reinterpret_cast<Control*>(dev.scratch),
                                                     static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? IDW_OK : IDW_ERR_CUDA;
}
