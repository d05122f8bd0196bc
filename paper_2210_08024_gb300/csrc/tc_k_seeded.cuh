// Launch helpers of the seeded step kernels, modes 3 and 4 (see tc_kernels.cuh); each
// mode is instantiated in its own translation unit (tc_k_seeded3.cu, tc_k_seeded4.cu).
// The kernels read the seed network's weights from global memory and keep its
// activations in per-thread arrays: no shared memory.
#pragma once
#include "tc_launch.h"

namespace tcg {

template <int MODE>
inline cudaError_t launch_seeded(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p,
                                 double dt, unsigned long long* cursor, long long ntotal, int grid, int block,
                                 cudaStream_t st, const MlpDev* mlp) {
  if (batch)
    k_step<MODE, true><<<grid, block, 0, st>>>(f, d_boxes, p, dt, cursor, ntotal, mlp);
  else
    k_step<MODE, false><<<grid, block, 0, st>>>(f, d_boxes, p, dt, cursor, ntotal, mlp);
  return cudaGetLastError();
}

template <int MODE>
inline int occupancy_seeded(int block) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<MODE, false>, block, 0) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

}  // namespace tcg
