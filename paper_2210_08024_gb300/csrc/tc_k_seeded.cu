// Instantiations of the seeded step kernels, modes 3 and 4 (see tc_kernels.cuh).  They
// keep the seed network's weights and two activation buffers per thread in dynamic
// shared memory (seed_smem_bytes).
#include "tc_launch.h"

namespace tcg {

template <int MODE>
static cudaError_t launch_seeded(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p,
                                 double dt, unsigned long long* cursor, long long ntotal, int grid, int block,
                                 cudaStream_t st, const MlpDev* mlp) {
  const size_t sm = seed_smem_bytes(block);
  cudaError_t e = cudaFuncSetAttribute(k_step<MODE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step<MODE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  if (batch)
    k_step<MODE, true><<<grid, block, sm, st>>>(f, d_boxes, p, dt, cursor, ntotal, mlp);
  else
    k_step<MODE, false><<<grid, block, sm, st>>>(f, d_boxes, p, dt, cursor, ntotal, mlp);
  return cudaGetLastError();
}

cudaError_t launch_mode3(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p, double dt,
                         unsigned long long* cursor, long long ntotal, int grid, int block, cudaStream_t st,
                         const MlpDev* mlp) {
  return launch_seeded<3>(batch, f, d_boxes, p, dt, cursor, ntotal, grid, block, st, mlp);
}

cudaError_t launch_mode4(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p, double dt,
                         unsigned long long* cursor, long long ntotal, int grid, int block, cudaStream_t st,
                         const MlpDev* mlp) {
  return launch_seeded<4>(batch, f, d_boxes, p, dt, cursor, ntotal, grid, block, st, mlp);
}

template <int MODE>
static int occupancy_seeded(int block) {
  const size_t sm = seed_smem_bytes(block);
  if (cudaFuncSetAttribute(k_step<MODE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return 1;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<MODE, false>, block, sm) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

int occupancy_mode3_impl(int block) { return occupancy_seeded<3>(block); }
int occupancy_mode4_impl(int block) { return occupancy_seeded<4>(block); }

}  // namespace tcg
