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
cudaError_t launch_local(const float* data, int64_t n, const float* queries, int64_t m, double p,
                         double radius, float* out, int32_t* count_out, void* workspace,
                         const LocalLayout& L, int sm_count, cudaStream_t s);

// Index-check failures of a debug build (bit s = check site s failed since
// the last call; cleared by the call), on the current device.  *enabled is
// false in a release build.
cudaError_t debug_check_failures(unsigned* sites, bool* enabled);

// The k-nearest-neighbour form (1 <= k <= kKnnMax): same grid build, then
// a ring search per query.  nbr_out (m x k) and kd2_out (m) may be null.
constexpr int kKnnMax = 64;
cudaError_t launch_knn(const float* data, int64_t n, const float* queries, int64_t m, double p,
                       int k, float* out, int32_t* nbr_out, float* kd2_out, void* workspace,
                       const LocalLayout& L, int sm_count, cudaStream_t s);

}  // namespace idw
