// Internal declarations shared by the kernel translation units and the C ABI
// layer.  Not installed; the public interface is include/idw.h.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace idw {

// ---------------------------------------------------------------- tiling
// FP32-compensated forward: each thread holds kQueryPairsF32 pairs of queries;
// a data tile of kRecordsF32 points is staged as (x,x,y,y) + (z,z) records.
constexpr int kThreadsF32 = 256;
constexpr int kQueryPairsF32 = 4;
constexpr int kQueriesPerCtaF32 = kThreadsF32 * 2 * kQueryPairsF32;  // 2048
constexpr int kRecordsF32 = 256;
constexpr int kStagesF32 = 3;
// Points per chunk between error-free TwoSum folds, and the shape of the
// chunk sums.  S0 is summed as a balanced binary tree, S1 as FMA chains of
// products w z joined by a tree, so every term passes through a fixed number
// of roundings before the fold: p = 2, chunks of 64: 6 (S0) and 4 + 4 (S1);
// general p, chunks of 32: 5 (S0) and 8 + 2 (S1).  The general form keeps
// shorter chunks: its longer weight arithmetic leaves fewer registers.
struct ChunkShape {
  int points, tree_levels, chain, chain_levels;
};
constexpr ChunkShape kChunkPow2{64, 6, 4, 4};
constexpr ChunkShape kChunkGeneral{32, 5, 8, 2};
// Weight sums above 2^100 (coordinates prescaled into [2^9, 2^10)) can only
// come from a point closer than 2^-50 to the query when p >= 2; such queries
// are recomputed in FP64, which keeps every d^2 of the fast path far above
// the FP32 subnormal range.
constexpr double kHugeSumPow2Up = 1.2676506002282294e30;  // 2^100
constexpr size_t kTileBytesF32 = size_t(kRecordsF32) * 24;  // 16 B (x,x,y,y) + 8 B (z,z)
// Instances per batched launch (the instance table is a kernel parameter).
constexpr int kBatchCap = 256;
// Compiled variants of the FP32 sweep (query-tile size, shared reciprocals);
// variant 0 is the default tiling above.
constexpr int kNumSweepVariants = 6;

// Plain FP64 forward: kQueriesF64 queries per thread; tiles of (x,y) + z.
constexpr int kThreadsF64 = 128;
constexpr int kQueriesF64 = 8;
constexpr int kQueriesPerCtaF64 = kThreadsF64 * kQueriesF64;  // 1024
constexpr int kRecordsF64 = 128;
constexpr int kStagesF64 = 3;
constexpr size_t kTileBytesF64 = size_t(kRecordsF64) * 24;  // 16 B (x,y) + 8 B z

// Queries whose FP32 weight sum falls below n * 2^-100 are recomputed in
// FP64: below that, weights flushed to zero could matter.
constexpr double kTinySumPerPoint = 7.888609052210118e-31;  // 2^-100

// Hit codes written by the combine / slow path.
constexpr int32_t kNoHit = -1;
constexpr int32_t kRecomputedF64 = -2;

// Device control words owned by a handle (zeroed once at creation).
struct Control {
  unsigned flagged;  // number of queries routed to the slow path this call
  unsigned error;    // sticky error bits (kErrWaitTimeout, ...)
  // Per-problem largest |coordinate| (float bits) of the FP32 forward's
  // range scan; every call leaves them zero (its combine clears them).
  unsigned maxbits[kBatchCap];
};

enum WeightMode : int { kPow2 = 0, kPowGeneral = 1 };

// Optional events recorded around the all-pairs sweep kernel.
struct SweepEvents {
  cudaEvent_t start = nullptr, stop = nullptr;
};

// --------------------------------------------------- FP32 (batched) plan
// One problem of Eq. 1 in FP32 (device pointers, caller-owned).
struct F32Problem {
  const float* data;     // n x 3
  int64_t n;
  const float* queries;  // m x 2
  int64_t m;
  float* out;
  double* s0_out;    // nullable
  int32_t* hit_out;  // nullable
};

// Launch plan of up to kBatchCap problems swept by one persistent grid.
// Work units are (query tile, data tile) pairs numbered instance by
// instance, query-tile-major; CTA g sweeps [g U / G, (g + 1) U / G).
struct BatchPlan {
  int variant = 0;
  bool force_general = false;  // evaluate p = 2 through the log2/exp2 path
  int layout = -1;             // data-tile staging layout; -1 = default for the weight form
  bool fma_log2 = false;       // general p, one problem, variant 4: 1 log2 in 16 on the FMA pipe
  int count = 0;
  std::vector<int64_t> data_tiles, query_tiles, unit_base, qtile_base, tile_offset;
  int64_t units = 0, total_query_tiles = 0, total_stage_tiles = 0;
  int grid = 0;
  int64_t partial_slots = 0;
  size_t staged_bytes = 0, partial_bytes = 0, list_bytes = 0, scale_bytes = 0;
  size_t workspace_bytes = 0;
};

// Host arithmetic only.  Problems must have n >= 1 and m >= 1.
void plan_batch_f32(const F32Problem* probs, int count, int sm_count, int ctas_per_sm,
                    int variant, BatchPlan* plan);
int sweep_variant_queries_per_cta(int variant);
int sweep_variant_points_per_unit(int variant);
// The variant actually run: sub-tile variants fall back to 0 for general p.
int resolve_sweep_variant(int variant, bool general_form);
// Default variant without tuning.  Small p = 2 problems (fewer than four
// 256-point work units per resident CTA) use the fine-grained variant 5, so
// the grid stays full and balanced; otherwise one 512-thread CTA per SM
// (variant 4) keeps all 16 warps of an SM in step, when its 4096-query
// tiles pad the queries no more than variant 0's 2048-query tiles (+1%).
int default_sweep_variant(const F32Problem* probs, int count, bool general_form, int sm_count);

// Enqueues range scan, staging, sweep, combine and slow path for the batch.
cudaError_t launch_batch_f32(const F32Problem* probs, const BatchPlan& plan, double p,
                             void* workspace, Control* ctrl, int sm_count,
                             const SweepEvents* ev, cudaStream_t stream);
int occupancy_forward_f32(bool general_p, int variant);

// Failure-detection self-test: a bounded wait on a barrier nobody completes.
cudaError_t launch_bounded_wait_selftest(Control* ctrl, cudaStream_t stream);

// ------------------------------------------------------- FP32 adjoint
struct BwdProblem {
  const float* data;     // n x 3
  int64_t n;
  const float* queries;  // m x 2
  int64_t m;
  double p;
  const float* Z;        // forward outputs (m)
  const double* s0;      // saved weight sums (m)
  const int32_t* hit;    // saved hit codes (m)
  const float* g;        // upstream gradient (m)
  float* grad_z;         // n, nullable
  float* grad_xy;        // n x 2, nullable
  float* grad_q;         // m x 2, nullable
  double* grad_p;        // 1, nullable
};

struct BwdPlan {
  int64_t data_tiles = 0, query_records_tiles = 0, query_reg_tiles = 0, data_reg_tiles = 0;
  int64_t units_q = 0, units_d = 0;
  int grid_q = 0, grid_d = 0;
  size_t staged_bytes = 0, qtiles_bytes = 0, partial_bytes = 0, gp_bytes = 0, list_bytes = 0,
         dlist_bytes = 0, scale_bytes = 0, workspace_bytes = 0;
};

void plan_backward_f32(int64_t n, int64_t m, int sm_count, int ctas_per_sm, BwdPlan* plan);
cudaError_t launch_backward_f32(const BwdProblem& pb, const BwdPlan& plan, void* workspace,
                                Control* ctrl, int sm_count, cudaStream_t stream);
int occupancy_backward_f32();

// ------------------------------------------------------------ FP64 plain
struct Plan {
  int threads, queries_per_cta, records_per_tile;
  int64_t query_tiles, data_tiles, units;
  int grid;
  int max_pieces;
  int64_t partial_slots;
  size_t staged_bytes, partial_bytes, list_bytes, workspace_bytes;
};

struct F64Problem {
  const double* data;
  int64_t n;
  const double* queries;
  int64_t m;
  double p;
  double* out;
  double* s0_out;
  int32_t* hit_out;
};
cudaError_t launch_forward_f64(const F64Problem& pb, const Plan& plan, void* workspace,
                               Control* ctrl, int sm_count, const SweepEvents* ev,
                               cudaStream_t stream);
int occupancy_forward_f64();

// The paper's naive and tiled kernels (measured baselines), in its layouts.
size_t paper_layout_bytes(int64_t n, bool fp64);
cudaError_t launch_paper_kernel(int kernel, int layout, bool fp64, const void* rows, int64_t n,
                                const void* queries, int64_t m, double p, void* out,
                                void* workspace, cudaStream_t stream);

// Pipe-rate probe: returns ops per SM per clock for the 6 probed pipes.
cudaError_t measure_pipe_rates(int sm_count, double rates[6]);
// Exhaustive accuracy of the MUFU approximations the weights use:
// errs = {max relative error of rcp, max absolute error of lg2 on [1/2, 2],
// max relative error of ex2, max error of lg2 relative to |log2 x| elsewhere}.
cudaError_t measure_mufu_errors(int sm_count, double errs[4]);

}  // namespace idw
