// Internal interface of the local forms (radius-limited and k nearest
// neighbours): workspace layout and the launch sequences (the grid of cells
// is planned on the device).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace idw {

// Byte offsets of the local form's scratch inside one workspace.
struct LocalLayout {
  int64_t max_cells = 0;
  size_t off_grid = 0, off_counts_d = 0, off_counts_q = 0, off_starts_d = 0, off_starts_q = 0;
  size_t off_sums = 0, off_sorted = 0, off_qrec = 0, off_bpre = 0, off_sat = 0;
  size_t bytes = 0;
};

// Cap on the number of cells for n data points (bounds the workspace).
int64_t local_max_cells(int64_t n);
LocalLayout local_layout(int64_t n, int64_t m, int64_t max_cells);

// Enqueues the whole local form on `s`: bounding box, grid plan, counting
// sort of data and queries, gather.  No host synchronisation.
// sort_queries = false keeps the caller's query order (no query sort);
// modified = true uses the modified Shepard weights (1/d - 1/R)^p.
cudaError_t launch_local(const float* data, int64_t n, const float* queries, int64_t m, double p,
                         double radius, float* out, int32_t* count_out, void* workspace,
                         const LocalLayout& L, int sm_count, cudaStream_t s,
                         bool sort_queries = true, bool modified = false);

// Gradients of L = sum_j grad_out[j] Z(q_j) for the radius form, or with
// modified = true for modified Shepard (membership sets held fixed): the
// grid build, then one kernel per query and one per data point.  The workspace holds L.bytes plus local_grad_record_bytes(m).
// grad_z (n), grad_xy (n x 2), grad_q (m x 2) and grad_p (1) may be null.
size_t local_grad_record_bytes(int64_t m);
cudaError_t launch_local_backward(const float* data, int64_t n, const float* queries, int64_t m,
                                  double p, double radius, const float* grad_out, float* grad_z,
                                  float* grad_xy, float* grad_q, double* grad_p, void* workspace,
                                  const LocalLayout& L, int sm_count, cudaStream_t s,
                                  bool modified = false);

// Index-check failures of a debug build (bit s = check site s failed since
// the last call; cleared by the call), on the current device.  *enabled is
// false in a release build.
cudaError_t debug_check_failures(unsigned* sites, bool* enabled);

// The k-nearest-neighbour form (1 <= k <= kKnnMax): same grid build, then
// a square search per query.  nbr_out (m x k), kd2_out (m) and hit_out (m:
// the lowest coincident data index, or -1) may be null.  sort_rows = false
// leaves each row of nbr_out in heap order (the selection, unordered).
constexpr int kKnnMax = 64;
cudaError_t launch_knn(const float* data, int64_t n, const float* queries, int64_t m, double p,
                       int k, float* out, int32_t* nbr_out, float* kd2_out, void* workspace,
                       const LocalLayout& L, int sm_count, cudaStream_t s,
                       int32_t* hit_out = nullptr, bool sort_queries = true,
                       bool sort_rows = true, bool warp_search = false);

// Gradients of the k-NN form (each selection held fixed): the search with
// neighbour lists and hits kept in the workspace after L.bytes (plus
// knn_grad_scratch_bytes(n, m, k)), then one kernel per query that adds the
// data-side terms with atomics.  Outputs as launch_local_backward.
// With `deterministic`, the data-side terms are summed point by point in
// increasing query order (a stable sort of the selections by point) and
// dL/dp over queries in index order, so repeated calls give the same bits.
size_t knn_grad_scratch_bytes(int64_t n, int64_t m, int k, bool deterministic = false);
cudaError_t launch_knn_backward(const float* data, int64_t n, const float* queries, int64_t m,
                                double p, int k, const float* grad_out, float* grad_z,
                                float* grad_xy, float* grad_q, double* grad_p, void* workspace,
                                const LocalLayout& L, int sm_count, cudaStream_t s,
                                bool sort_queries = true, bool deterministic = false,
                                bool warp_search = false);

// A prepared index: the data side of a local form built once and queried
// by many calls.  The index's own buffer holds the plan, the data cell
// starts and tile bases, the sorted records, and for k-NN a copy of the data
// (read by original index), the occupancy-block prefix and the
// summed-area table.
struct IndexLayout {
  int64_t n = 0, max_cells = 0;
  bool knn = false;
  size_t off_grid = 0, off_counts = 0, off_starts = 0, off_sums = 0, off_sorted = 0;
  size_t off_data = 0, off_bpre = 0, off_sat = 0;
  size_t bytes = 0;
};
IndexLayout index_layout(int64_t n, bool knn);

// Scratch of one query call on a prepared index (in the handle's workspace).
struct QueryLayout {
  size_t off_grid = 0, off_counts = 0, off_starts = 0, off_sums = 0, off_qrec = 0;
  size_t bytes = 0;
};
QueryLayout query_layout(int64_t m, int64_t max_cells);

// Enqueues the data side: bounding box, plan (cells for `radius`, or for k
// neighbours when knn_k > 0), counting sort of the data, and for k-NN the
// data copy and both count tables.
cudaError_t launch_index_build(const float* data, int64_t n, double radius, int knn_k,
                               void* index_mem, const IndexLayout& X, int sm_count,
                               cudaStream_t s);

// One query call on a radius index (0 < radius <= the build radius), with
// the plain or (modified = true) the modified Shepard weights.
cudaError_t launch_index_local(const void* index_mem, const IndexLayout& X, const float* queries,
                               int64_t m, double p, double radius, float* out, int32_t* count_out,
                               void* workspace, const QueryLayout& Q, int sm_count,
                               cudaStream_t s, bool sort_queries = true, bool modified = false);

// One query call on a k-NN index (1 <= k <= kKnnMax).
cudaError_t launch_index_knn(const void* index_mem, const IndexLayout& X, const float* queries,
                             int64_t m, double p, int k, float* out, int32_t* nbr_out,
                             float* kd2_out, void* workspace, const QueryLayout& Q, int sm_count,
                             cudaStream_t s, bool sort_queries = true);

}  // namespace idw
