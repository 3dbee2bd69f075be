// Staging layouts of the plain FP64 forward pass (the paper's FP64 layout
// question, Sec. 3.5 and Sec. 4.1.2, asked of this library's own sweep).
#pragma once

#include <cstddef>

#include "idw_internal.h"

namespace idw {

// 0: Hybrid, (x, y) pairs beside z[] (24 B/point, the default);
// 1: AoaS, aligned (x, y, z, pad) records (32 B/point);
// 2: SoA, x[], y[], z[] (24 B/point).
enum F64Layout : int { kF64Hybrid = 0, kF64Aoas = 1, kF64Soa = 2 };

size_t f64_tile_bytes(int layout);
int occupancy_forward_f64_layout(int layout);
cudaError_t launch_forward_f64_layout(const F64Problem& pb, const Plan& plan, int layout,
                                      void* workspace, Control* ctrl, int sm_count,
                                      const SweepEvents* ev, cudaStream_t stream);

}  // namespace idw
