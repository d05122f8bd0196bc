// Instantiation of the seeded step kernel, mode 3 (mixed seeded; see tc_kernels.cuh).
#include "tc_k_seeded.cuh"

namespace tcg {

cudaError_t launch_mode3(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p, double dt,
                         unsigned long long* cursor, long long ntotal, int grid, int block, cudaStream_t st,
                         const MlpDev* mlp) {
  return launch_seeded<3>(batch, f, d_boxes, p, dt, cursor, ntotal, grid, block, st, mlp);
}

int occupancy_mode3_impl(int block) { return occupancy_seeded<3>(block); }

}  // namespace tcg
