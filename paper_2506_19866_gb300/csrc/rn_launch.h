// rn_launch.h -- host-side launchers of the kernels in rn_kernels.cu and
// rn_anneal{1,2,4}.cu.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rn_device.cuh"

namespace rn {

// One resident grid; with more chains than resident warps, the steps of every
// chain are cut into chunks of 16 so that all warps stay busy to the end (the
// last round costs at most one chunk).
inline void plan_chunks(DevSched &s, int64_t n_chains, int64_t warps)
{
    const int64_t steps = s.g1 - s.g0;
    s.chunk = n_chains > warps ? (steps < 16 ? steps : 16) : steps;
    if (s.chunk < 1) s.chunk = 1;
    s.n_chunks = (int32_t)((steps + s.chunk - 1) / s.chunk);
}

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

// Single-condition networks with four chains per warp in the byte lanes
// (rn_chains4.cu): the layouts compiled for it, and its launch.
bool chains4_layout(const DevNet &net, int d0, int d1);
cudaError_t launch_anneal_chains4(const DevNet &net, int d0, int d1, const DevChains &ch,
                                  const DevSched &sc, int sm_count, cudaStream_t st);

// Hybrid path (rn_smemreg.cu): 6, 8 or 10 nodes per lane, table words in
// shared memory, node state in registers.
bool smemreg_layout(int npl);
cudaError_t launch_anneal_smemreg(const DevNet &net, const DevChains &ch, const DevSched &sc,
                                  int sm_count, cudaStream_t st);
cudaError_t launch_evaluate_smemreg(const DevNet &net, const int8_t *X, int64_t xstride,
                                    int32_t n, int32_t *score, int32_t *score2, uint8_t *traj,
                                    int grid, cudaStream_t st);

// Block path (rn_block.cu): networks of 513 .. 4096 nodes, a block of
// kBlockLanes threads per chain.  Shared memory of one block:
size_t block_path_smem_bytes(const int *D, int npl, int N);
// Whether the block's shared memory holds the second copy of the state codes
// (code_word2): the register variant, where it fits.
bool block_path_two_copies(const int *D, int npl, int N);
cudaError_t launch_evaluate_block(const DevNet &net, const int8_t *X, int64_t xstride, int32_t n,
                                  int32_t *score, int32_t *score2, uint8_t *traj, int sm_count,
                                  cudaStream_t st);
cudaError_t launch_anneal_block(const DevNet &net, const DevChains &ch, const DevSched &sc,
                                int sm_count, cudaStream_t st);
// Level-end argmin of d_best and broadcast of the winner's x_best, within groups
// of `group` consecutive chains (0: one group of all chains); winner holds one
// entry per group.
cudaError_t launch_level_sync(const DevChains &ch, int32_t *winner, int32_t group,
                              cudaStream_t st);
// One warp waits, with a short limit, on a counter nothing advances (*never = 0):
// the wait gives up and sets *err; *out = 1 if it was satisfied instead.
cudaError_t launch_wait_selftest(const int32_t *never, int32_t *err, int32_t *out,
                                 cudaStream_t st);

// Many networks in one persistent launch (rn_batch.cu).
struct DevBatch {
    int32_t n_nets, total;              // networks; chains over all networks
    int32_t total_big;                  // global chains [0, total_big) use the shared-memory tables
    int32_t large;                      // warps per block with a large region (first in the block)
    int64_t sweeps;                     // steps every chain advances
    uint32_t region_bytes;              // shared memory of a large warp region (any network)
    uint32_t region_small;              // shared memory of a small region (register-table networks)
    const DevNet *nets;                 // [n_nets]
    const DevChains *chains;            // [n_nets]
    int64_t *g0;                        // [n_nets] next step of each network (advanced on device)
    const int32_t *item_net;            // [total] network of global chain r
    const int32_t *item_chain;          // [total] chain index within its network
    const int32_t *path;                // [n_nets] 1, 2, 4: register tables; 0: shared memory
};

bool batch_path_fits(int npl, int D0, int Drest);
// Shared-table networks (path 0) run on the large-region warps.
// Table paths of a batched network: 1, 2, 4 register tables (small warp
// region); 0 shared-memory tables, 6, 8 the hybrid layouts (large region).
inline bool batch_shared_tables(int path) { return path == 0 || path > 4; }
uint32_t batch_region_bytes(int path, const int *D, int npl, int pstride, int N);
// Block shared memory of a configuration, and the resident grid it allows.
size_t batch_smem_bytes(int wpb, int large, uint32_t region_big, uint32_t region_small);
cudaError_t batch_resident_warps(int wpb, size_t smem, int sm_count, int *grid);
cudaError_t launch_batch(const DevBatch &b, const DevSched &sc, int wpb, int grid,
                         cudaStream_t st);

// A phased batch runs one launch per table path, each over that path's global
// chains [r0, r0 + n) with its own work queue (slot `queue`), warp region,
// warps per block and resident grid.
struct BatchPhase {
    int32_t path, r0, n, queue;
    uint32_t region;
    int32_t wpb, grid;
};
constexpr int kMaxPhases = 7;           // table paths 10, 8, 6, 0, 4, 2, 1
constexpr int kQueueSlots = 8;          // work-queue counters of a context
size_t batch_phase_smem(const BatchPhase &ph);
// Resident grid of the phase's kernel (sets its dynamic shared-memory limit).
cudaError_t batch_phase_grid(BatchPhase &ph, int sm_count);
// Queue and done resets, every phase in order, the step advance.  With
// `marks` (2 per phase, may be NULL) an event is recorded around each phase.
cudaError_t launch_batch_phased(const DevBatch &b, const DevSched &sc, const BatchPhase *ph,
                                int n_ph, cudaStream_t st, cudaEvent_t *marks);

}  // namespace rn
