// rn_launch.h -- host-side launchers of the kernels in rn_kernels.cu and
// rn_anneal{1,2,4}.cu.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rn_device.cuh"

namespace rn {

// Layouts compiled for the warp-per-chain kernels: 1, 2 or 4 nodes per lane
// (N <= 128), 1 or 4 conditions per group, register capacity d0 for slot 0 and
// d1 for the other slots (in-edges per node up to 16).
bool anneal_layout_supported(int npl, int cg, int d0, int d1);
// Smallest compiled capacities covering in-degree D0 (slot 0) and Drest (the
// other slots); -1 if none.
void anneal_capacity(int npl, int D0, int Drest, int *d0, int *d1);

cudaError_t launch_evaluate(const DevNet &net, const int8_t *X, int64_t xstride, int32_t n,
                            int32_t *score, int32_t *score2, uint8_t *traj, int sm_count,
                            cudaStream_t st);
cudaError_t launch_anneal(const DevNet &net, int d0, int d1, const DevChains &ch,
                          const DevSched &sc, int sm_count, cudaStream_t st);
cudaError_t launch_init(const DevNet &net, const DevChains &ch, int32_t *status, cudaStream_t st);
cudaError_t launch_level_sync(const DevChains &ch, int32_t *winner, cudaStream_t st);

}  // namespace rn
