// Host-side launch entry points of the step kernels (one per translation unit).
#pragma once
#include <cuda_runtime.h>

#include "tc_kernels.cuh"

namespace tcg {
// Launches mode-M step kernels; batch selects the box-table variant.
cudaError_t launch_mode0(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p, double dt,
                         unsigned long long* cursor, long long ntotal, int grid, int block, cudaStream_t st);
cudaError_t launch_mode1(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p, double dt,
                         unsigned long long* cursor, long long ntotal, int grid, int block, cudaStream_t st);
cudaError_t launch_mode2(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p, double dt,
                         unsigned long long* cursor, long long ntotal, int grid, int block, cudaStream_t st);
// Warp-cooperative variants of modes 1 and 2 (four lanes per cell, one box); `grid`
// and `block` count threads, four per cell.
cudaError_t launch_mode1_coop(const DevFields& f, const DevParams& p, double dt, unsigned long long* cursor,
                              long long ntotal, int grid, int block, cudaStream_t st);
cudaError_t launch_mode2_coop(const DevFields& f, const DevParams& p, double dt, unsigned long long* cursor,
                              long long ntotal, int grid, int block, cudaStream_t st);
int occupancy_mode1_coop(int block);
int occupancy_mode2_coop(int block);
// Seeded modes (3: mixed, 4: FP64 Newton); mlp points to the device weight blob.
cudaError_t launch_mode3(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p, double dt,
                         unsigned long long* cursor, long long ntotal, int grid, int block, cudaStream_t st,
                         const MlpDev* mlp);
cudaError_t launch_mode4(bool batch, const DevFields& f, const BoxTable* d_boxes, const DevParams& p, double dt,
                         unsigned long long* cursor, long long ntotal, int grid, int block, cudaStream_t st,
                         const MlpDev* mlp);
// Device check of the df64 source terms (tc_df64_diag.cu; tc_df64_source_check).
cudaError_t launch_df64_source_check(const DevFields& f, const DevParams& p, double* err, cudaStream_t st);
}  // namespace tcg
