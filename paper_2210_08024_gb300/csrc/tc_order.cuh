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

// Start-state source terms of the substep rule of Sec. 6.1 for every cell (tc_rates):
// rate[3 i + 0..2] = (C_H2, C_H+, H / (K T_mu)) and dts[i] = the first substep length of
// a step of dt; either output may be null.
cudaError_t launch_rates(const DevFields& f, const DevParams& p, double dt, long long ntotal, double* rate,
                         double* dts, int num_sms, cudaStream_t st);

}  // namespace tcg
