// Instantiation of the mode-0 step kernel (see tc_kernels.cuh).
#include "tc_launch.h"

namespace tcg {

cudaError_t launch_mode0(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p, double dt,
                         unsigned long long* cursor, long long ntotal, int grid, int block, cudaStream_t st) {
  if (batch)
    k_step<0, true><<<grid, block, 0, st>>>(f, d_boxes, p, dt, cursor, ntotal, nullptr);
  else
    k_step<0, false><<<grid, block, 0, st>>>(f, d_boxes, p, dt, cursor, ntotal, nullptr);
  return cudaGetLastError();
}

int occupancy_mode0_impl(int block) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<0, false>, block, 0) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

}  // namespace tcg
