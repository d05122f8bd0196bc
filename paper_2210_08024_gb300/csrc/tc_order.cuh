// Cost-ordered work queue of the step kernel (tc_params.order_cells).
#pragma once
#include <cuda_runtime.h>

#include "tc_kernels.cuh"

namespace tcg {

// Cost classes: quarter octaves of dt / dts_1 (the first substep length of Sec. 6.1
// before its cap at dt) from 2^-16 to 2^16.
constexpr int ORDER_BUCKETS = 128;

// Fills order[0..ntotal) with the cell indices (over the concatenated boxes when batch)
// sorted by decreasing predicted substep count.  key (ntotal bytes) and hist
// (ORDER_BUCKETS counters) are workspace.  Four launches on `st`.
cudaError_t launch_order(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p, double dt,
                         long long ntotal, unsigned char* key, unsigned* hist, unsigned* order, int num_sms,
                         cudaStream_t st);

}  // namespace tcg
