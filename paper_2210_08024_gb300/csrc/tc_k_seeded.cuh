// Launch helpers of the seeded step kernels, modes 3 and 4 (see tc_kernels.cuh); each
// mode is instantiated in its own translation unit (tc_k_seeded3.cu, tc_k_seeded4.cu).
// The kernels keep the seed network's weights and two activation buffers per thread in
// dynamic shared memory (seed_smem_bytes).
#pragma once
#include "tc_launch.h"

namespace tcg {

template <int MODE>
inline cudaError_t launch_seeded(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p,
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

template <int MODE>
inline int occupancy_seeded(int block) {
  const size_t sm = seed_smem_bytes(block);
  if (cudaFuncSetAttribute(k_step<MODE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return 1;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<MODE, false>, block, sm) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

}  // namespace tcg
