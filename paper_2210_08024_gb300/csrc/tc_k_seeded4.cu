// Instantiation of the seeded step kernel, mode 4 (FP64 Newton seeded; see tc_kernels.cuh).
#include "tc_k_seeded.cuh"

namespace tcg {

cudaError_t launch_mode4(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p, double dt,
                         unsigned long long* cursor, long long ntotal, int grid, int block, cudaStream_t st,
                         const MlpDev* mlp) {
  return launch_seeded<4>(batch, f, d_boxes, p, dt, cursor, ntotal, grid, block, st, mlp);
}

int occupancy_mode4_impl(int block) { return occupancy_seeded<4>(block); }

}  // namespace tcg
