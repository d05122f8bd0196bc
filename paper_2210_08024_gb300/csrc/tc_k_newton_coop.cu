// Instantiation of the warp-cooperative mode-1 step kernel (four lanes per cell; see
// tc_kernels.cuh).
#include "tc_launch.h"

namespace tcg {

cudaError_t launch_mode1_coop(const DevFields& f, const DevParams& p, double dt, unsigned long long* cursor,
                              long long ntotal, int grid, int block, cudaStream_t st) {
  k_step<1, false, 4><<<grid, block, 0, st>>>(f, nullptr, p, dt, cursor, ntotal, nullptr);
  return cudaGetLastError();
}

int occupancy_mode1_coop(int block) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<1, false, 4>, block, 0) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

}  // namespace tcg
