// C ABI of the IDW library (declared in include/idw.h): argument checks,
// launch planning, workspace ownership and the host-buffer path.  Every
// step of the computation runs in the kernels of the other translation
// units; this file only validates, plans and enqueues.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <cstdlib>
#include <fstream>
#include <initializer_list>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "idw.h"
#include "idw_device.cuh"
#include "idw_internal.h"
#include "idw_f64_layout.h"
#include "idw_local.h"

struct idw_handle_s {
  int device = 0;
  int sm_count = 0;
  void* ws = nullptr;  // device workspace (staged tiles, partials, flag list)
  size_t ws_bytes = 0;
  void* io = nullptr;  // device buffers of the host-pointer entry point
  size_t io_bytes = 0;
  idw::Control* ctrl = nullptr;  // device control words
  int occ_f64 = 0, occ_bwd = 0;
  int occ_f64_layout[3] = {};  // plain FP64 form per staging layout
  int occ_f32[2][idw::kNumSweepVariants] = {};  // [general p][variant]
  // Options (idw_set_option).
  int opt_autotune = 0, opt_variant = -1, opt_force_general = 0, opt_layout = -1;
  int opt_validate = 0;         // scan inputs for NaN / inf before computing
  int opt_query_order = 0;      // local forms: 1 keeps the caller's query order
  bool opt_deterministic = false;  // k-NN gradients summed in a fixed order
  bool opt_fma_log2 = false;       // general p: part of log2 on the FMA pipe
  int opt_knn_search = 0;          // k-NN search: 0 one thread per query, 1 warp-cooperative
  unsigned* vflag = nullptr;    // device word the scan sets
  int last_variant = -1;
  std::map<std::string, int> tuned;  // size class -> sweep variant
  std::string tune_path;             // JSON cache file ("" = memory only)
  char last_cuda[256] = "no error";
  bool profiling = false;
  std::vector<idw::SweepEvents> events;  // recorded sweep launches, oldest first
  size_t events_used = 0;
};

// A prepared index of the local forms (idw_local_index_create).
struct idw_local_index_s {
  int device = 0;
  double radius = 0.0;  // > 0: a radius index built for this radius
  int k = 0;            // > 0: a k-NN index built for k neighbours
  idw::IndexLayout X;
  void* mem = nullptr;  // device buffer laid out by X
};

namespace {

using idw::Plan;

constexpr int64_t kMaxCount = int64_t(1) << 31;

inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// An NVTX range around one entry point (visible in Nsight timelines; a
// no-op unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// Makes the handle's device current for the lifetime of the guard.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

idw_status cuda_fail(idw_handle_t h, cudaError_t e) {
  if (h) {
    std::snprintf(h->last_cuda, sizeof(h->last_cuda), "%s: %s", cudaGetErrorName(e),
                  cudaGetErrorString(e));
  }
  return IDW_ERR_CUDA;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Launch plan of the single-problem forward pass (host arithmetic only).
void make_plan(int sm_count, int ctas_per_sm, int64_t n, int64_t m, idw_precision prec,
               Plan* pl) {
  const bool f32 = prec == IDW_PREC_F32_COMP;
  pl->threads = f32 ? idw::kThreadsF32 : idw::kThreadsF64;
  pl->queries_per_cta = f32 ? idw::kQueriesPerCtaF32 : idw::kQueriesPerCtaF64;
  pl->records_per_tile = f32 ? idw::kRecordsF32 : idw::kRecordsF64;
  pl->query_tiles = (m + pl->queries_per_cta - 1) / pl->queries_per_cta;
  pl->data_tiles = (n + pl->records_per_tile - 1) / pl->records_per_tile;
  pl->units = pl->query_tiles * pl->data_tiles;
  const int64_t resident = int64_t(sm_count) * (ctas_per_sm > 0 ? ctas_per_sm : 1);
  pl->grid = static_cast<int>(pl->units < resident ? (pl->units > 0 ? pl->units : 1) : resident);
  pl->partial_slots = pl->query_tiles + pl->grid - 1;
  // Upper bound on CTAs sharing one query tile; exact value by idw_plan_forward.
  pl->max_pieces = static_cast<int>(
      pl->units > 0 ? ((pl->data_tiles - 1) * pl->grid) / pl->units + 2 : 0);
  const size_t tile_bytes = f32 ? idw::kTileBytesF32 : idw::kTileBytesF64;
  pl->staged_bytes = round_up(size_t(pl->data_tiles) * tile_bytes, 256);
  pl->partial_bytes = round_up(size_t(pl->partial_slots) * pl->queries_per_cta * 16, 256);
  pl->list_bytes = round_up(size_t(m > 0 ? m : 1) * sizeof(int32_t), 256);
  pl->workspace_bytes = pl->staged_bytes + pl->partial_bytes + pl->list_bytes;
}

idw_status ensure_buffer(idw_handle_t h, void** buf, size_t* have, size_t need) {
  if (need <= *have) return IDW_OK;
  if (*buf) {
    cudaError_t e = cudaFree(*buf);  // synchronises: earlier work may still use it
    *buf = nullptr;
    *have = 0;
    if (e != cudaSuccess) return cuda_fail(h, e);
  }
  const size_t bytes = round_up(need + need / 4, size_t(1) << 20);
  cudaError_t e = cudaMalloc(buf, bytes);
  if (e != cudaSuccess) {
    *buf = nullptr;
    cuda_fail(h, e);
    return IDW_ERR_WORKSPACE;
  }
  *have = bytes;
  return IDW_OK;
}

// Event pair for the next sweep launch, or nullptr when timing is off.
const idw::SweepEvents* next_events(idw_handle_t h) {
  if (!h->profiling) return nullptr;
  if (h->events_used == h->events.size()) {
    idw::SweepEvents ev;
    if (cudaEventCreate(&ev.start) != cudaSuccess) return nullptr;
    if (cudaEventCreate(&ev.stop) != cudaSuccess) {
      cudaEventDestroy(ev.start);
      return nullptr;
    }
    h->events.push_back(ev);
  }
  return &h->events[h->events_used++];
}

void destroy_events(idw_handle_t h) {
  for (auto& ev : h->events) {
    cudaEventDestroy(ev.start);
    cudaEventDestroy(ev.stop);
  }
  h->events.clear();
  h->events_used = 0;
}

bool uses_general_power(idw_handle_t h, double p) { return p != 2.0 || h->opt_force_general; }

int ctas_per_sm(idw_handle_t h, idw_precision prec, double p, int variant = 0) {
  if (prec == IDW_PREC_F64_PLAIN) {
    if (!h->occ_f64) h->occ_f64 = idw::occupancy_forward_f64();
    return h->occ_f64;
  }
  const int gen = uses_general_power(h, p) ? 1 : 0;
  int& occ = h->occ_f32[gen][variant];
  if (!occ) occ = idw::occupancy_forward_f32(gen != 0, variant);
  return occ;
}

// ------------------------------------------------------------- autotuner
// Size class of a batch: weight form, and log2 of the mean data and query
// counts and of the total number of pairs.
std::string size_class(idw_handle_t h, const idw::F32Problem* probs, int count, double p) {
  double n = 0, m = 0, pairs = 0;
  for (int k = 0; k < count; ++k) {
    n += double(probs[k].n);
    m += double(probs[k].m);
    pairs += double(probs[k].n) * double(probs[k].m);
  }
  std::ostringstream o;
  o << "sm" << h->sm_count << (uses_general_power(h, p) ? "_gen" : "_pow2") << "_n"
    << int(std::lround(std::log2(n / count))) << "_m" << int(std::lround(std::log2(m / count)))
    << "_pairs" << int(std::lround(std::log2(pairs)));
  return o.str();
}

void load_tuning(idw_handle_t h) {
  if (h->tune_path.empty()) return;
  std::ifstream f(h->tune_path);
  std::string line;
  while (std::getline(f, line)) {
    const size_t a = line.find('"'), b = line.find('"', a + 1), c = line.find(':', b + 1);
    if (a == std::string::npos || b == std::string::npos || c == std::string::npos) continue;
    const int v = std::atoi(line.c_str() + c + 1);
    if (v >= 0 && v < idw::kNumSweepVariants) h->tuned[line.substr(a + 1, b - a - 1)] = v;
  }
}

void save_tuning(idw_handle_t h) {
  if (h->tune_path.empty()) return;
  const std::string tmp = h->tune_path + ".tmp";
  {
    std::ofstream f(tmp);
    f << "{\n";
    size_t k = 0;
    for (const auto& kv : h->tuned)
      f << "  \"" << kv.first << "\": " << kv.second << (++k < h->tuned.size() ? ",\n" : "\n");
    f << "}\n";
  }
  std::rename(tmp.c_str(), h->tune_path.c_str());
}

// Sweep variant for a batch: forced, tuned (timed once per size class with
// CUDA events, never while the stream is being captured), or the default
// rule of idw::default_sweep_variant.
int default_variant(idw_handle_t h, const idw::F32Problem* probs, int count, double p) {
  return idw::default_sweep_variant(probs, count, uses_general_power(h, p), h->sm_count);
}

int choose_variant_unresolved(idw_handle_t h, const idw::F32Problem* probs, int count, double p,
                              cudaStream_t s);

// The sweep variant for a batch, resolved for the weight form.
int choose_variant(idw_handle_t h, const idw::F32Problem* probs, int count, double p,
                   cudaStream_t s) {
  return idw::resolve_sweep_variant(choose_variant_unresolved(h, probs, count, p, s),
                                    uses_general_power(h, p));
}

int choose_variant_unresolved(idw_handle_t h, const idw::F32Problem* probs, int count, double p,
                              cudaStream_t s) {
  if (h->opt_variant >= 0) return h->opt_variant;
  if (!h->opt_autotune) return default_variant(h, probs, count, p);
  const std::string key = size_class(h, probs, count, p);
  auto it = h->tuned.find(key);
  if (it != h->tuned.end()) return it->second;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return default_variant(h, probs, count, p);
  std::vector<idw::BatchPlan> plans(idw::kNumSweepVariants);
  size_t need = 0;
  const bool general = uses_general_power(h, p);
  for (int v = 0; v < idw::kNumSweepVariants; ++v) {
    if (idw::resolve_sweep_variant(v, general) != v) continue;
    idw::plan_batch_f32(probs, count, h->sm_count, ctas_per_sm(h, IDW_PREC_F32_COMP, p, v), v,
                        &plans[v]);
    plans[v].force_general = h->opt_force_general != 0;
    need = std::max(need, plans[v].workspace_bytes);
  }
  if (ensure_buffer(h, &h->ws, &h->ws_bytes, need) != IDW_OK) return 0;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return 0;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return 0;
  }
  int best = 0;
  float best_ms = 0.f;
  for (int v = 0; v < idw::kNumSweepVariants; ++v) {
    if (idw::resolve_sweep_variant(v, general) != v) continue;
    float ms = 0.f;
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep) {  // the first run loads the module
      ok = cudaEventRecord(a, s) == cudaSuccess &&
           idw::launch_batch_f32(probs, plans[v], p, h->ws, h->ctrl, h->sm_count, nullptr, s) ==
               cudaSuccess &&
           cudaEventRecord(b, s) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
           cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
    }
    if (ok && (v == 0 || ms < best_ms)) {
      best = v;
      best_ms = ms;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  h->tuned[key] = best;
  save_tuning(h);
  return best;
}

// Sets *flag when any of the count values is NaN or infinite.
template <typename T>
__global__ void __launch_bounds__(256)
    nonfinite_scan_kernel(const T* __restrict__ a, int64_t count, unsigned* __restrict__ flag) {
  bool bad = false;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
       i += int64_t(gridDim.x) * blockDim.x)
    bad |= !isfinite(a[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

struct Span {
  const void* ptr;
  int64_t count;  // values
  bool fp64;
};

// With IDW_OPT_VALIDATE_INPUTS set: scans every span and returns
// IDW_ERR_NOT_FINITE_INPUT if any value is NaN or infinite.  Reads the
// verdict back, so it synchronises the stream and refuses a capture.
idw_status validate_inputs(idw_handle_t h, std::initializer_list<Span> spans, cudaStream_t s) {
  if (!h->opt_validate) return IDW_OK;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return cuda_fail(h, e);
  if (cap != cudaStreamCaptureStatusNone) return IDW_ERR_UNSUPPORTED;
  if (!h->vflag && (e = cudaMalloc(&h->vflag, sizeof(unsigned))) != cudaSuccess) {
    h->vflag = nullptr;
    return cuda_fail(h, e);
  }
  if ((e = cudaMemsetAsync(h->vflag, 0, sizeof(unsigned), s)) != cudaSuccess)
    return cuda_fail(h, e);
  for (const Span& sp : spans) {
    if (!sp.ptr || sp.count <= 0) continue;
    const unsigned grid = static_cast<unsigned>(
        std::max<int64_t>(1, std::min<int64_t>(int64_t(h->sm_count) * 4, (sp.count + 255) / 256)));
    if (sp.fp64)
      nonfinite_scan_kernel<double><<<grid, 256, 0, s>>>(static_cast<const double*>(sp.ptr),
                                                          sp.count, h->vflag);
    else
      nonfinite_scan_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float*>(sp.ptr),
                                                         sp.count, h->vflag);
  }
  unsigned flag = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, h->vflag, sizeof(flag), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e);
  return flag ? IDW_ERR_NOT_FINITE_INPUT : IDW_OK;
}

idw_status check_common(idw_handle_t h, const void* data, int64_t n, const void* queries,
                        int64_t m, double p, idw_precision prec, const void* out) {
  if (!h) return IDW_ERR_INVALID_ARG;
  if (prec != IDW_PREC_F32_COMP && prec != IDW_PREC_F64_PLAIN) return IDW_ERR_INVALID_ARG;
  if (n < 1 || n >= kMaxCount || m < 0 || m >= kMaxCount) return IDW_ERR_INVALID_ARG;
  if (!(p > 0.0) || !std::isfinite(p)) return IDW_ERR_INVALID_ARG;
  if (m == 0) return IDW_OK;
  if (!data || !queries || !out) return IDW_ERR_INVALID_ARG;
  const size_t es = prec == IDW_PREC_F32_COMP ? 4 : 8;
  if (!aligned(data, es) || !aligned(queries, es) || !aligned(out, es)) return IDW_ERR_ALIGNMENT;
  return IDW_OK;
}

// One query call on a radius index, plain or modified Shepard weights.
idw_status index_radius_call(idw_handle_t h, idw_local_index_t ix,
                              const float* queries, int64_t m, double p, double radius,
                              float* out, int32_t* count_out, void* stream, bool modified) {
  if (!h || !ix || ix->radius <= 0.0 || h->device != ix->device) return IDW_ERR_INVALID_ARG;
  if (m < 0 || m >= kMaxCount || !(p > 0.0) || !std::isfinite(p)) return IDW_ERR_INVALID_ARG;
  if (!(radius > 0.0 && radius <= ix->radius)) return IDW_ERR_INVALID_ARG;
  if (m == 0) return IDW_OK;
  if (!queries || !out) return IDW_ERR_INVALID_ARG;
  if (!aligned(queries, 4) || !aligned(out, 4) || (count_out && !aligned(count_out, 4)))
    return IDW_ERR_ALIGNMENT;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  idw_status st = validate_inputs(h, {{queries, 2 * m, false}}, s);
  if (st != IDW_OK) return st;
  const idw::QueryLayout Q = idw::query_layout(m, ix->X.max_cells);
  st = ensure_buffer(h, &h->ws, &h->ws_bytes, Q.bytes);
  if (st != IDW_OK) return st;
  const cudaError_t e = idw::launch_index_local(ix->mem, ix->X, queries, m, p, radius, out,
                                                count_out, h->ws, Q, h->sm_count, s,
                                                h->opt_query_order == 0, modified);
  return e == cudaSuccess ? IDW_OK : cuda_fail(h, e);
}


// The radius form's gradients, plain or modified Shepard weights.
idw_status radius_backward_call(idw_handle_t h, const float* data, int64_t n,
                                const float* queries,
                              int64_t m, double p, double radius, const float* grad_out,
                              float* grad_z, float* grad_data_xy, float* grad_query_xy,
                              double* grad_p, void* stream, bool modified) {
  idw_status st = check_common(h, data, n, queries, m, p, IDW_PREC_F32_COMP, grad_out);
  if (st != IDW_OK) return st;
  if (!(radius > 0.0)) return IDW_ERR_INVALID_ARG;
  if ((grad_z && !aligned(grad_z, 4)) || (grad_data_xy && !aligned(grad_data_xy, 4)) ||
      (grad_query_xy && !aligned(grad_query_xy, 4)) || (grad_p && !aligned(grad_p, 8)))
    return IDW_ERR_ALIGNMENT;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (m == 0) {  // no query: every gradient is zero
    if (grad_z) e = cudaMemsetAsync(grad_z, 0, size_t(n) * 4, s);
    if (e == cudaSuccess && grad_data_xy) e = cudaMemsetAsync(grad_data_xy, 0, size_t(n) * 8, s);
    if (e == cudaSuccess && grad_p) e = cudaMemsetAsync(grad_p, 0, sizeof(double), s);
    return e == cudaSuccess ? IDW_OK : cuda_fail(h, e);
  }
  st = validate_inputs(h, {{data, 3 * n, false}, {queries, 2 * m, false}, {grad_out, m, false}}, s);
  if (st != IDW_OK) return st;
  const idw::LocalLayout L = idw::local_layout(n, m, idw::local_max_cells(n));
  st = ensure_buffer(h, &h->ws, &h->ws_bytes, L.bytes + idw::local_grad_record_bytes(m));
  if (st != IDW_OK) return st;
  e = idw::launch_local_backward(data, n, queries, m, p, radius, grad_out, grad_z, grad_data_xy,
                                 grad_query_xy, grad_p, h->ws, L, h->sm_count, s, modified);
  return e == cudaSuccess ? IDW_OK : cuda_fail(h, e);
}


}  // namespace

extern "C" {

const char* idw_status_string(idw_status s) {
  switch (s) {
    case IDW_OK: return "IDW_OK";
    case IDW_ERR_INVALID_ARG: return "IDW_ERR_INVALID_ARG";
    case IDW_ERR_ALIGNMENT: return "IDW_ERR_ALIGNMENT";
    case IDW_ERR_CUDA: return "IDW_ERR_CUDA";
    case IDW_ERR_NOT_FINITE_INPUT: return "IDW_ERR_NOT_FINITE_INPUT";
    case IDW_ERR_WORKSPACE: return "IDW_ERR_WORKSPACE";
    case IDW_ERR_UNSUPPORTED: return "IDW_ERR_UNSUPPORTED";
    case IDW_ERR_DEVICE_TIMEOUT: return "IDW_ERR_DEVICE_TIMEOUT";
  }
  return "IDW_ERR_UNKNOWN";
}

idw_status idw_create(idw_handle_t* out, int device) {
  if (!out) return IDW_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return IDW_ERR_INVALID_ARG;
  DeviceGuard guard(device);
  if (!guard.ok) return IDW_ERR_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return IDW_ERR_CUDA;
  if (prop.major != 10 || prop.minor != 3) return IDW_ERR_UNSUPPORTED;
  idw_handle_t h = new idw_handle_s();
  h->device = device;
  h->sm_count = prop.multiProcessorCount;
  cudaError_t e = cudaMalloc(&h->ctrl, sizeof(idw::Control));
  if (e == cudaSuccess) e = cudaMemset(h->ctrl, 0, sizeof(idw::Control));
  if (e != cudaSuccess) {
    if (h->ctrl) cudaFree(h->ctrl);
    delete h;
    return IDW_ERR_CUDA;
  }
  if (const char* path = std::getenv("IDW_AUTOTUNE_CACHE")) {
    h->tune_path = path;
    load_tuning(h);
  }
  *out = h;
  return IDW_OK;
}

idw_status idw_create_ex(idw_handle_t* out, int device, const char* autotune_cache) {
  idw_status st = idw_create(out, device);
  if (st != IDW_OK || !autotune_cache) return st;
  (*out)->tune_path = autotune_cache;  // overrides IDW_AUTOTUNE_CACHE
  (*out)->tuned.clear();
  load_tuning(*out);
  return IDW_OK;
}

idw_status idw_destroy(idw_handle_t h) {
  if (!h) return IDW_ERR_INVALID_ARG;
  DeviceGuard guard(h->device);
  cudaDeviceSynchronize();
  if (h->ws) cudaFree(h->ws);
  if (h->io) cudaFree(h->io);
  if (h->ctrl) cudaFree(h->ctrl);
  if (h->vflag) cudaFree(h->vflag);
  destroy_events(h);
  delete h;
  return IDW_OK;
}

const char* idw_last_cuda_error(idw_handle_t h) { return h ? h->last_cuda : "null handle"; }

idw_status idw_interpolate_saved(idw_handle_t h, const void* data, int64_t n, const void* queries,
                                 int64_t m, double p, idw_precision prec, void* out,
                                 double* s0_out, int32_t* hit_out, void* stream) {
  NvtxRange nvtx("idw_interpolate_saved");
  idw_status st = check_common(h, data, n, queries, m, p, prec, out);
  if (st != IDW_OK || m == 0) return st;
  if (!aligned(s0_out, 8) || !aligned(hit_out, 4)) return IDW_ERR_ALIGNMENT;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool f64 = prec == IDW_PREC_F64_PLAIN;
  st = validate_inputs(h, {{data, 3 * n, f64}, {queries, 2 * m, f64}}, s);
  if (st != IDW_OK) return st;
  cudaError_t e;
  if (prec == IDW_PREC_F32_COMP) {
    idw::F32Problem pb{static_cast<const float*>(data), n, static_cast<const float*>(queries), m,
                       static_cast<float*>(out), s0_out, hit_out};
    const bool fma_log2 = h->opt_fma_log2 && uses_general_power(h, p);
    const int v = fma_log2 ? 4 : choose_variant(h, &pb, 1, p, s);
    idw::BatchPlan bp;
    idw::plan_batch_f32(&pb, 1, h->sm_count, ctas_per_sm(h, prec, p, v), v, &bp);
    bp.force_general = h->opt_force_general != 0;
    bp.layout = v == 0 ? h->opt_layout : -1;
    bp.fma_log2 = fma_log2;
    st = ensure_buffer(h, &h->ws, &h->ws_bytes, bp.workspace_bytes);
    if (st != IDW_OK) return st;
    h->last_variant = v;
    e = idw::launch_batch_f32(&pb, bp, p, h->ws, h->ctrl, h->sm_count, next_events(h), s);
  } else {
    // Staging layout of the FP64 form: 1 = AoaS, 2 = SoA, otherwise Hybrid.
    const int layout = h->opt_layout >= 1 ? h->opt_layout : idw::kF64Hybrid;
    int& occ = h->occ_f64_layout[layout];
    if (!occ) occ = idw::occupancy_forward_f64_layout(layout);
    Plan plan;
    make_plan(h->sm_count, occ, n, m, prec, &plan);
    // make_plan sizes Hybrid tiles; the AoaS records are wider.
    plan.workspace_bytes -= plan.staged_bytes;
    plan.staged_bytes = round_up(size_t(plan.data_tiles) * idw::f64_tile_bytes(layout), 256);
    plan.workspace_bytes += plan.staged_bytes;
    st = ensure_buffer(h, &h->ws, &h->ws_bytes, plan.workspace_bytes);
    if (st != IDW_OK) return st;
    idw::F64Problem pb{static_cast<const double*>(data), n, static_cast<const double*>(queries), m,
                       p, static_cast<double*>(out), s0_out, hit_out};
    e = idw::launch_forward_f64_layout(pb, plan, layout, h->ws, h->ctrl, h->sm_count,
                                       next_events(h), s);
  }
  if (e != cudaSuccess) return cuda_fail(h, e);
  return IDW_OK;
}

idw_status idw_interpolate(idw_handle_t h, const void* data, int64_t n, const void* queries,
                           int64_t m, double p, idw_precision prec, void* out, void* stream) {
  return idw_interpolate_saved(h, data, n, queries, m, p, prec, out, nullptr, nullptr, stream);
}

idw_status idw_interpolate_host(idw_handle_t h, const void* data, int64_t n, const void* queries,
                                int64_t m, double p, idw_precision prec, void* out, void* stream) {
  NvtxRange nvtx("idw_interpolate_host");
  idw_status st = check_common(h, data, n, queries, m, p, prec, out);
  if (st != IDW_OK || m == 0) return st;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  const size_t es = prec == IDW_PREC_F32_COMP ? 4 : 8;
  const size_t db = round_up(size_t(n) * 3 * es, 256), qb = round_up(size_t(m) * 2 * es, 256);
  const size_t ob = round_up(size_t(m) * es, 256);
  st = ensure_buffer(h, &h->io, &h->io_bytes, db + qb + ob);
  if (st != IDW_OK) return st;
  unsigned char* io = static_cast<unsigned char*>(h->io);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(io, data, size_t(n) * 3 * es, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(io + db, queries, size_t(m) * 2 * es, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(h, e);
  st = idw_interpolate_saved(h, io, n, io + db, m, p, prec, io + db + qb, nullptr, nullptr, stream);
  if (st != IDW_OK) return st;
  e = cudaMemcpyAsync(out, io + db + qb, size_t(m) * es, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e);
  return IDW_OK;
}

idw_status idw_interpolate_batched(idw_handle_t h, int32_t count, const void* const* data,
                                   const int64_t* n, const void* const* queries, const int64_t* m,
                                   double p, idw_precision prec, void* const* out, void* stream) {
  NvtxRange nvtx("idw_interpolate_batched");
  if (!h || count < 0 || (count > 0 && (!data || !n || !queries || !m || !out)))
    return IDW_ERR_INVALID_ARG;
  for (int32_t k = 0; k < count; ++k) {
    idw_status st = check_common(h, data[k], n[k], queries[k], m[k], p, prec, out[k]);
    if (st != IDW_OK) return st;
  }
  if (prec == IDW_PREC_F64_PLAIN) {
    // The comparison form: one stream-ordered single-problem call each
    // (consecutive problems reuse the workspace in stream order).
    for (int32_t k = 0; k < count; ++k) {
      const idw_status st = idw_interpolate_saved(h, data[k], n[k], queries[k], m[k], p, prec,
                                                  out[k], nullptr, nullptr, stream);
      if (st != IDW_OK) return st;
    }
    return IDW_OK;
  }
  // Problems with m = 0 have nothing to compute; the rest go in chunks of
  // up to kBatchCap problems, one persistent launch per chunk.
  std::vector<idw::F32Problem> probs;
  probs.reserve(count);
  for (int32_t k = 0; k < count; ++k) {
    if (m[k] == 0) continue;
    probs.push_back(idw::F32Problem{static_cast<const float*>(data[k]), n[k],
                                    static_cast<const float*>(queries[k]), m[k],
                                    static_cast<float*>(out[k]), nullptr, nullptr});
  }
  if (probs.empty()) return IDW_OK;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (const idw::F32Problem& pb : probs) {
    const idw_status vs = validate_inputs(h, {{pb.data, 3 * pb.n, false}, {pb.queries, 2 * pb.m, false}}, s);
    if (vs != IDW_OK) return vs;
  }
  std::vector<idw::BatchPlan> plans;
  size_t need = 0;
  for (size_t b = 0; b < probs.size(); b += idw::kBatchCap) {
    const int c = static_cast<int>(std::min<size_t>(idw::kBatchCap, probs.size() - b));
    const int v = choose_variant(h, &probs[b], c, p, s);
    plans.emplace_back();
    idw::plan_batch_f32(&probs[b], c, h->sm_count, ctas_per_sm(h, prec, p, v), v, &plans.back());
    plans.back().force_general = h->opt_force_general != 0;
    need = std::max(need, plans.back().workspace_bytes);
    h->last_variant = v;
  }
  idw_status st = ensure_buffer(h, &h->ws, &h->ws_bytes, need);
  if (st != IDW_OK) return st;
  for (size_t c = 0; c < plans.size(); ++c) {
    cudaError_t e = idw::launch_batch_f32(&probs[c * idw::kBatchCap], plans[c], p, h->ws, h->ctrl,
                                          h->sm_count, next_events(h), s);
    if (e != cudaSuccess) return cuda_fail(h, e);
  }
  return IDW_OK;
}

idw_status idw_backward(idw_handle_t h, const float* data, int64_t n, const float* queries,
                        int64_t m, double p, const float* Z, const double* s0, const int32_t* hit,
                        const float* grad_out, float* grad_z, float* grad_data_xy,
                        float* grad_query_xy, double* grad_p, void* stream) {
  NvtxRange nvtx("idw_backward");
  idw_status st = check_common(h, data, n, queries, m, p, IDW_PREC_F32_COMP, Z);
  if (st != IDW_OK) return st;
  if (m == 0) {
    // No query contributes: every requested gradient is zero.
    DeviceGuard guard(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (grad_z) e = cudaMemsetAsync(grad_z, 0, size_t(n) * sizeof(float), s);
    if (e == cudaSuccess && grad_data_xy)
      e = cudaMemsetAsync(grad_data_xy, 0, size_t(n) * 2 * sizeof(float), s);
    if (e == cudaSuccess && grad_p) e = cudaMemsetAsync(grad_p, 0, sizeof(double), s);
    return e == cudaSuccess ? IDW_OK : cuda_fail(h, e);
  }
  if (!s0 || !hit || !grad_out) return IDW_ERR_INVALID_ARG;
  if (!aligned(s0, 8) || !aligned(hit, 4) || !aligned(grad_out, 4) || !aligned(grad_z, 4) ||
      !aligned(grad_data_xy, 4) || !aligned(grad_query_xy, 4) || !aligned(grad_p, 8))
    return IDW_ERR_ALIGNMENT;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  st = validate_inputs(h, {{data, 3 * n, false}, {queries, 2 * m, false}, {grad_out, m, false}},
                       static_cast<cudaStream_t>(stream));
  if (st != IDW_OK) return st;
  if (!h->occ_bwd) h->occ_bwd = idw::occupancy_backward_f32();
  idw::BwdPlan bp;
  idw::plan_backward_f32(n, m, h->sm_count, h->occ_bwd, &bp);
  st = ensure_buffer(h, &h->ws, &h->ws_bytes, bp.workspace_bytes);
  if (st != IDW_OK) return st;
  idw::BwdProblem pb{static_cast<const float*>(data), n, static_cast<const float*>(queries), m, p,
                     Z, s0, hit, grad_out, grad_z, grad_data_xy, grad_query_xy, grad_p};
  cudaError_t e = idw::launch_backward_f32(pb, bp, h->ws, h->ctrl, h->sm_count,
                                           static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? IDW_OK : cuda_fail(h, e);
}

idw_status idw_paper_interpolate(idw_handle_t h, idw_paper_kernel kernel, idw_paper_layout layout,
                                 const void* data, int64_t n, const void* queries, int64_t m,
                                 double p, idw_precision prec, void* out, void* stream) {
  NvtxRange nvtx("idw_paper_interpolate");
  idw_status st = check_common(h, data, n, queries, m, p, prec, out);
  if (st != IDW_OK || m == 0) return st;
  if (kernel != IDW_PAPER_NAIVE && kernel != IDW_PAPER_TILED) return IDW_ERR_INVALID_ARG;
  if (layout < IDW_LAYOUT_SOA || layout > IDW_LAYOUT_HYBRID) return IDW_ERR_INVALID_ARG;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  const bool fp64 = prec == IDW_PREC_F64_PLAIN;
  st = validate_inputs(h, {{data, 3 * n, fp64}, {queries, 2 * m, fp64}},
                       static_cast<cudaStream_t>(stream));
  if (st != IDW_OK) return st;
  st = ensure_buffer(h, &h->ws, &h->ws_bytes, idw::paper_layout_bytes(n, fp64));
  if (st != IDW_OK) return st;
  const cudaError_t e = idw::launch_paper_kernel(kernel, layout, fp64, data, n, queries, m, p, out,
                                                 h->ws, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? IDW_OK : cuda_fail(h, e);
}

idw_status idw_interpolate_local(idw_handle_t h, const float* data, int64_t n,
                                 const float* queries, int64_t m, double p, double radius,
                                 float* out, int32_t* count_out, void* stream) {
  NvtxRange nvtx("idw_interpolate_local");
  idw_status st = check_common(h, data, n, queries, m, p, IDW_PREC_F32_COMP, out);
  if (st != IDW_OK) return st;
  if (!(radius > 0.0)) return IDW_ERR_INVALID_ARG;
  if (m == 0) return IDW_OK;
  if (count_out && !aligned(count_out, 4)) return IDW_ERR_ALIGNMENT;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  st = validate_inputs(h, {{data, 3 * n, false}, {queries, 2 * m, false}},
                       static_cast<cudaStream_t>(stream));
  if (st != IDW_OK) return st;
  const int64_t max_cells = idw::local_max_cells(n);
  const idw::LocalLayout L = idw::local_layout(n, m, max_cells);
  st = ensure_buffer(h, &h->ws, &h->ws_bytes, L.bytes);
  if (st != IDW_OK) return st;
  const cudaError_t e = idw::launch_local(data, n, queries, m, p, radius, out, count_out, h->ws, L,
                                          h->sm_count, static_cast<cudaStream_t>(stream),
                                          h->opt_query_order == 0);
  return e == cudaSuccess ? IDW_OK : cuda_fail(h, e);
}

idw_status idw_interpolate_modified(idw_handle_t h, const float* data, int64_t n,
                                    const float* queries, int64_t m, double p, double radius,
                                    float* out, int32_t* count_out, void* stream) {
  NvtxRange nvtx("idw_interpolate_modified");
  idw_status st = check_common(h, data, n, queries, m, p, IDW_PREC_F32_COMP, out);
  if (st != IDW_OK) return st;
  if (!(radius > 0.0)) return IDW_ERR_INVALID_ARG;
  if (m == 0) return IDW_OK;
  if (count_out && !aligned(count_out, 4)) return IDW_ERR_ALIGNMENT;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  st = validate_inputs(h, {{data, 3 * n, false}, {queries, 2 * m, false}},
                       static_cast<cudaStream_t>(stream));
  if (st != IDW_OK) return st;
  const idw::LocalLayout L = idw::local_layout(n, m, idw::local_max_cells(n));
  st = ensure_buffer(h, &h->ws, &h->ws_bytes, L.bytes);
  if (st != IDW_OK) return st;
  const cudaError_t e = idw::launch_local(data, n, queries, m, p, radius, out, count_out, h->ws, L,
                                          h->sm_count, static_cast<cudaStream_t>(stream),
                                          h->opt_query_order == 0, true);
  return e == cudaSuccess ? IDW_OK : cuda_fail(h, e);
}

idw_status idw_interpolate_knn(idw_handle_t h, const float* data, int64_t n, const float* queries,
                               int64_t m, double p, int32_t k, float* out, int32_t* nbr_out,
                               float* kd2_out, void* stream) {
  NvtxRange nvtx("idw_interpolate_knn");
  idw_status st = check_common(h, data, n, queries, m, p, IDW_PREC_F32_COMP, out);
  if (st != IDW_OK) return st;
  if (k < 1 || k > idw::kKnnMax) return IDW_ERR_INVALID_ARG;
  if (m == 0) return IDW_OK;
  if ((nbr_out && !aligned(nbr_out, 4)) || (kd2_out && !aligned(kd2_out, 4)))
    return IDW_ERR_ALIGNMENT;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  st = validate_inputs(h, {{data, 3 * n, false}, {queries, 2 * m, false}},
                       static_cast<cudaStream_t>(stream));
  if (st != IDW_OK) return st;
  const idw::LocalLayout L = idw::local_layout(n, m, idw::local_max_cells(n));
  st = ensure_buffer(h, &h->ws, &h->ws_bytes, L.bytes);
  if (st != IDW_OK) return st;
  const cudaError_t e = idw::launch_knn(data, n, queries, m, p, k, out, nbr_out, kd2_out, h->ws, L,
                                        h->sm_count, static_cast<cudaStream_t>(stream), nullptr,
                                        h->opt_query_order == 0, true, h->opt_knn_search == 1);
  return e == cudaSuccess ? IDW_OK : cuda_fail(h, e);
}

idw_status idw_local_backward(idw_handle_t h, const float* data, int64_t n, const float* queries,
                              int64_t m, double p, double radius, const float* grad_out,
                              float* grad_z, float* grad_data_xy, float* grad_query_xy,
                              double* grad_p, void* stream) {
  NvtxRange nvtx("idw_local_backward");
  return radius_backward_call(h, data, n, queries, m, p, radius, grad_out, grad_z, grad_data_xy,
                              grad_query_xy, grad_p, stream, false);
}

idw_status idw_modified_backward(idw_handle_t h, const float* data, int64_t n,
                                 const float* queries, int64_t m, double p, double radius,
                                 const float* grad_out, float* grad_z, float* grad_data_xy,
                                 float* grad_query_xy, double* grad_p, void* stream) {
  NvtxRange nvtx("idw_modified_backward");
  return radius_backward_call(h, data, n, queries, m, p, radius, grad_out, grad_z, grad_data_xy,
                              grad_query_xy, grad_p, stream, true);
}

idw_status idw_knn_backward(idw_handle_t h, const float* data, int64_t n, const float* queries,
                            int64_t m, double p, int32_t k, const float* grad_out, float* grad_z,
                            float* grad_data_xy, float* grad_query_xy, double* grad_p,
                            void* stream) {
  NvtxRange nvtx("idw_knn_backward");
  idw_status st = check_common(h, data, n, queries, m, p, IDW_PREC_F32_COMP, grad_out);
  if (st != IDW_OK) return st;
  if (k < 1 || k > idw::kKnnMax) return IDW_ERR_INVALID_ARG;
  if ((grad_z && !aligned(grad_z, 4)) || (grad_data_xy && !aligned(grad_data_xy, 8)) ||
      (grad_query_xy && !aligned(grad_query_xy, 4)) || (grad_p && !aligned(grad_p, 8)))
    return IDW_ERR_ALIGNMENT;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (m == 0) {  // no query: every gradient is zero
    if (grad_z) e = cudaMemsetAsync(grad_z, 0, size_t(n) * 4, s);
    if (e == cudaSuccess && grad_data_xy) e = cudaMemsetAsync(grad_data_xy, 0, size_t(n) * 8, s);
    if (e == cudaSuccess && grad_p) e = cudaMemsetAsync(grad_p, 0, sizeof(double), s);
    return e == cudaSuccess ? IDW_OK : cuda_fail(h, e);
  }
  st = validate_inputs(h, {{data, 3 * n, false}, {queries, 2 * m, false}, {grad_out, m, false}}, s);
  if (st != IDW_OK) return st;
  const bool det = h->opt_deterministic;
  if (det && m * int64_t(k) >= (int64_t(1) << 31)) return IDW_ERR_UNSUPPORTED;
  const idw::LocalLayout L = idw::local_layout(n, m, idw::local_max_cells(n));
  st = ensure_buffer(h, &h->ws, &h->ws_bytes, L.bytes + idw::knn_grad_scratch_bytes(n, m, k, det));
  if (st != IDW_OK) return st;
  e = idw::launch_knn_backward(data, n, queries, m, p, k, grad_out, grad_z, grad_data_xy,
                               grad_query_xy, grad_p, h->ws, L, h->sm_count, s,
                               h->opt_query_order == 0, det, h->opt_knn_search == 1);
  return e == cudaSuccess ? IDW_OK : cuda_fail(h, e);
}

idw_status idw_local_index_create(idw_handle_t h, const float* data, int64_t n, double radius,
                                  int32_t k, idw_local_index_t* index, void* stream) {
  NvtxRange nvtx("idw_local_index_create");
  if (!h || !index || !data) return IDW_ERR_INVALID_ARG;
  *index = nullptr;
  if (n < 1 || n >= kMaxCount) return IDW_ERR_INVALID_ARG;
  const bool knn = radius == 0.0 && k >= 1 && k <= idw::kKnnMax;
  const bool rad = radius > 0.0 && k == 0;  // NaN fails both
  if (!knn && !rad) return IDW_ERR_INVALID_ARG;
  if (!aligned(data, 4)) return IDW_ERR_ALIGNMENT;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  idw_status st = validate_inputs(h, {{data, 3 * n, false}}, s);
  if (st != IDW_OK) return st;
  idw_local_index_t ix = new idw_local_index_s();
  ix->device = h->device;
  ix->radius = rad ? radius : 0.0;
  ix->k = knn ? k : 0;
  ix->X = idw::index_layout(n, knn);
  cudaError_t e = cudaMalloc(&ix->mem, ix->X.bytes);
  if (e != cudaSuccess) {
    cuda_fail(h, e);
    delete ix;
    return IDW_ERR_WORKSPACE;
  }
  e = idw::launch_index_build(data, n, rad ? radius : 0.0, ix->k, ix->mem, ix->X, h->sm_count, s);
  if (e != cudaSuccess) {
    cudaFree(ix->mem);
    delete ix;
    return cuda_fail(h, e);
  }
  *index = ix;
  return IDW_OK;
}


idw_status idw_local_index_interpolate(idw_handle_t h, idw_local_index_t ix,
                                       const float* queries, int64_t m, double p, double radius,
                                       float* out, int32_t* count_out, void* stream) {
  NvtxRange nvtx("idw_local_index_interpolate");
  return index_radius_call(h, ix, queries, m, p, radius, out, count_out, stream, false);
}

idw_status idw_local_index_modified(idw_handle_t h, idw_local_index_t ix, const float* queries,
                                    int64_t m, double p, double radius, float* out,
                                    int32_t* count_out, void* stream) {
  NvtxRange nvtx("idw_local_index_modified");
  return index_radius_call(h, ix, queries, m, p, radius, out, count_out, stream, true);
}

idw_status idw_local_index_knn(idw_handle_t h, idw_local_index_t ix, const float* queries,
                               int64_t m, double p, int32_t k, float* out, int32_t* nbr_out,
                               float* kd2_out, void* stream) {
  NvtxRange nvtx("idw_local_index_knn");
  if (!h || !ix || ix->k <= 0 || h->device != ix->device) return IDW_ERR_INVALID_ARG;
  if (m < 0 || m >= kMaxCount || !(p > 0.0) || !std::isfinite(p)) return IDW_ERR_INVALID_ARG;
  if (k < 1 || k > idw::kKnnMax) return IDW_ERR_INVALID_ARG;
  if (m == 0) return IDW_OK;
  if (!queries || !out) return IDW_ERR_INVALID_ARG;
  if (!aligned(queries, 4) || !aligned(out, 4) || (nbr_out && !aligned(nbr_out, 4)) ||
      (kd2_out && !aligned(kd2_out, 4)))
    return IDW_ERR_ALIGNMENT;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  idw_status st = validate_inputs(h, {{queries, 2 * m, false}}, s);
  if (st != IDW_OK) return st;
  const idw::QueryLayout Q = idw::query_layout(m, ix->X.max_cells);
  st = ensure_buffer(h, &h->ws, &h->ws_bytes, Q.bytes);
  if (st != IDW_OK) return st;
  const cudaError_t e = idw::launch_index_knn(ix->mem, ix->X, queries, m, p, k, out, nbr_out,
                                              kd2_out, h->ws, Q, h->sm_count, s,
                                              h->opt_query_order == 0);
  return e == cudaSuccess ? IDW_OK : cuda_fail(h, e);
}

idw_status idw_local_index_destroy(idw_local_index_t ix) {
  if (!ix) return IDW_ERR_INVALID_ARG;
  DeviceGuard guard(ix->device);
  cudaDeviceSynchronize();
  if (ix->mem) cudaFree(ix->mem);
  delete ix;
  return IDW_OK;
}

idw_status idw_sync_status(idw_handle_t h, void* stream) {
  if (!h) return IDW_ERR_INVALID_ARG;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e);
  idw::Control c;
  e = cudaMemcpy(&c, h->ctrl, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e);
  if (c.error != 0) {
    cudaMemset(&h->ctrl->error, 0, sizeof(unsigned));
    return IDW_ERR_DEVICE_TIMEOUT;
  }
  return IDW_OK;
}

idw_status idw_set_option(idw_handle_t h, idw_option opt, int64_t value) {
  if (!h) return IDW_ERR_INVALID_ARG;
  switch (opt) {
    case IDW_OPT_AUTOTUNE:
      h->opt_autotune = value != 0;
      return IDW_OK;
    case IDW_OPT_SWEEP_VARIANT:
      if (value < -1 || value >= idw::kNumSweepVariants) return IDW_ERR_INVALID_ARG;
      h->opt_variant = static_cast<int>(value);
      return IDW_OK;
    case IDW_OPT_FORCE_GENERAL_POWER:
      h->opt_force_general = value != 0;
      return IDW_OK;
    case IDW_OPT_STAGING_LAYOUT:
      if (value < -1 || value > 2) return IDW_ERR_INVALID_ARG;
      h->opt_layout = static_cast<int>(value);
      return IDW_OK;
    case IDW_OPT_VALIDATE_INPUTS:
      h->opt_validate = value != 0;
      return IDW_OK;
    case IDW_OPT_LOCAL_QUERY_ORDER:
      if (value < 0 || value > 1) return IDW_ERR_INVALID_ARG;
      h->opt_query_order = static_cast<int>(value);
      return IDW_OK;
    case IDW_OPT_DETERMINISTIC:
      if (value < 0 || value > 1) return IDW_ERR_INVALID_ARG;
      h->opt_deterministic = value != 0;
      return IDW_OK;
    case IDW_OPT_FMA_LOG2:
      if (value < 0 || value > 1) return IDW_ERR_INVALID_ARG;
      h->opt_fma_log2 = value != 0;
      return IDW_OK;
    case IDW_OPT_KNN_SEARCH:
      if (value < 0 || value > 1) return IDW_ERR_INVALID_ARG;
      h->opt_knn_search = static_cast<int>(value);
      return IDW_OK;
    default:
      return IDW_ERR_INVALID_ARG;
  }
}

idw_status idw_get_option(idw_handle_t h, idw_option opt, int64_t* value) {
  if (!h || !value) return IDW_ERR_INVALID_ARG;
  switch (opt) {
    case IDW_OPT_AUTOTUNE: *value = h->opt_autotune; return IDW_OK;
    case IDW_OPT_SWEEP_VARIANT: *value = h->opt_variant; return IDW_OK;
    case IDW_OPT_FORCE_GENERAL_POWER: *value = h->opt_force_general; return IDW_OK;
    case IDW_OPT_LAST_VARIANT: *value = h->last_variant; return IDW_OK;
    case IDW_OPT_TUNED_CLASSES: *value = static_cast<int64_t>(h->tuned.size()); return IDW_OK;
    case IDW_OPT_STAGING_LAYOUT: *value = h->opt_layout; return IDW_OK;
    case IDW_OPT_VALIDATE_INPUTS: *value = h->opt_validate; return IDW_OK;
    case IDW_OPT_LOCAL_QUERY_ORDER: *value = h->opt_query_order; return IDW_OK;
    case IDW_OPT_DETERMINISTIC: *value = h->opt_deterministic; return IDW_OK;
    case IDW_OPT_FMA_LOG2: *value = h->opt_fma_log2; return IDW_OK;
    case IDW_OPT_KNN_SEARCH: *value = h->opt_knn_search; return IDW_OK;
    default: return IDW_ERR_INVALID_ARG;
  }
}

idw_status idw_profile_enable(idw_handle_t h, int enable) {
  if (!h) return IDW_ERR_INVALID_ARG;
  h->profiling = enable != 0;
  return IDW_OK;
}

idw_status idw_profile_read(idw_handle_t h, double* sweep_ms, int64_t* launches) {
  if (!h || !sweep_ms || !launches) return IDW_ERR_INVALID_ARG;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  double total = 0.0;
  for (size_t k = 0; k < h->events_used; ++k) {
    cudaError_t e = cudaEventSynchronize(h->events[k].stop);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, h->events[k].start, h->events[k].stop);
    if (e != cudaSuccess) return cuda_fail(h, e);
    total += ms;
  }
  *sweep_ms = total;
  *launches = static_cast<int64_t>(h->events_used);
  h->events_used = 0;
  return IDW_OK;
}

idw_status idw_selftest_bounded_wait(idw_handle_t h, void* stream) {
  if (!h) return IDW_ERR_INVALID_ARG;
  DeviceGuard guard(h->device);
  if (!guard.ok) return IDW_ERR_CUDA;
  cudaError_t e = idw::launch_bounded_wait_selftest(h->ctrl, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? IDW_OK : cuda_fail(h, e);
}

idw_status idw_plan_forward(int32_t sm_count, int32_t ctas, int64_t n, int64_t m, double p,
                            idw_precision prec, idw_plan_info* out) {
  if (!out || sm_count < 1 || ctas < 0 || n < 1 || n >= kMaxCount || m < 0 || m >= kMaxCount)
    return IDW_ERR_INVALID_ARG;
  if (!(p > 0.0) || !std::isfinite(p)) return IDW_ERR_INVALID_ARG;
  if (prec != IDW_PREC_F32_COMP && prec != IDW_PREC_F64_PLAIN) return IDW_ERR_INVALID_ARG;
  if (ctas == 0) ctas = prec == IDW_PREC_F32_COMP ? 2 : 4;
  Plan pl;
  make_plan(sm_count, ctas, n, m, prec, &pl);
  if (prec == IDW_PREC_F32_COMP && m > 0) {
    idw::F32Problem pb{nullptr, n, nullptr, m, nullptr, nullptr, nullptr};
    idw::BatchPlan bp;
    idw::plan_batch_f32(&pb, 1, sm_count, ctas, 0, &bp);
    pl.grid = bp.grid;
    pl.partial_slots = bp.partial_slots;
    pl.workspace_bytes = bp.workspace_bytes;
  }
  int max_pieces = 0;
  for (int64_t qt = 0; qt < pl.query_tiles; ++qt) {
    const int64_t g0 = idw::cta_of_unit(qt * pl.data_tiles, pl.units, pl.grid);
    const int64_t g1 = idw::cta_of_unit((qt + 1) * pl.data_tiles - 1, pl.units, pl.grid);
    if (g1 - g0 + 1 > max_pieces) max_pieces = static_cast<int>(g1 - g0 + 1);
  }
  out->queries_per_thread = pl.queries_per_cta / pl.threads;
  out->threads_per_cta = pl.threads;
  out->queries_per_cta = pl.queries_per_cta;
  out->records_per_tile = pl.records_per_tile;
  out->query_tiles = pl.query_tiles;
  out->data_tiles = pl.data_tiles;
  out->units = pl.units;
  out->grid = pl.grid;
  out->max_pieces_per_query_tile = max_pieces;
  out->partial_slots = pl.partial_slots;
  out->workspace_bytes = pl.workspace_bytes;
  return IDW_OK;
}

idw_status idw_debug_check_failures(int device, uint32_t* sites) {
  if (!sites) return IDW_ERR_INVALID_ARG;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return IDW_ERR_INVALID_ARG;
  DeviceGuard guard(device);
  if (!guard.ok) return IDW_ERR_CUDA;
  bool enabled = false;
  unsigned v = 0;
  if (idw::debug_check_failures(&v, &enabled) != cudaSuccess) return IDW_ERR_CUDA;
  *sites = v;
  return enabled ? IDW_OK : IDW_ERR_UNSUPPORTED;
}

idw_status idw_measure_pipe_rates(int device, double rates[6]) {
  if (!rates) return IDW_ERR_INVALID_ARG;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return IDW_ERR_INVALID_ARG;
  DeviceGuard guard(device);
  if (!guard.ok) return IDW_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return IDW_ERR_CUDA;
  cudaError_t e = idw::measure_pipe_rates(sms, rates);
  return e == cudaSuccess ? IDW_OK : IDW_ERR_CUDA;
}

idw_status idw_measure_mufu_errors(int device, double errs[4]) {
  if (!errs) return IDW_ERR_INVALID_ARG;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return IDW_ERR_INVALID_ARG;
  DeviceGuard guard(device);
  if (!guard.ok) return IDW_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return IDW_ERR_CUDA;
  cudaError_t e = idw::measure_mufu_errors(sms, errs);
  return e == cudaSuccess ? IDW_OK : IDW_ERR_CUDA;
}

}  // extern "C"
