// rn_batch.cu -- one persistent launch over the chains of many networks.
//
// Every chain of every network is one "global chain" r.  Global chains come
// in two classes with a work queue each: first the chains of networks on the
// shared-memory tables (r < total_big), then those on register tables; within
// a class grouped by table path, and within a path the network with the most
// work per chain first.  Item i of a class
// of n chains is chunk i / n of the class's chain i % n, so that, as in the
// single-network kernel, the predecessor of an item (the previous chunk of the
// same chain) was handed out n items earlier from the same queue.
//
// Shared-memory tables need a large per-warp region, register tables a small
// one.  The first `large` warps of a block get a large region and take items
// of the first class, then help with the second; the other warps get a small
// region and take only register-table items.  Sizing every warp for the
// largest network would cut the resident warps several fold.
//
// Each warp copies the descriptors of its item's network into its shared
// memory and runs the chunk with that network's table path.  Results are
// those of separate single-network runs, bit for bit (same per-chain code,
// same Philox counters).
#include "rn_kernels.cuh"

namespace rn {

// Table paths of a network in the batch: 1, 2, 4 = register tables, capacities
// slot 0 up to 16 in-edges and the other slots up to 8; 0 = the shared-memory
// path (any layout); 6, 8, 10 = the hybrid path (table words in shared memory,
// node state in registers) of 129-320-node networks (10 in phased launches
// only, whose kernel is compiled for its register need).  Which of these a
// network takes is chosen by the autotuner.
constexpr int kBatchD0 = 16, kBatchD1 = 8;

// Code region, then the per-warp copies of the item's DevNet and DevChains,
// rounded up so that the warp regions stay 256-byte aligned.
__host__ __device__ inline uint32_t batch_head_bytes(int wpb)
{
    const uint32_t b = (uint32_t)wpb * (kCodeBytesPerWarp + (uint32_t)sizeof(DevNet) +
                                        (uint32_t)sizeof(DevChains));
    return (b + 255u) & ~255u;
}

__device__ __forceinline__ void warp_copy_words(void *dst, const void *src, int bytes, int lane)
{
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    for (int k = lane; k < bytes / 4; k += 32) d[k] = __ldcg(s + k);
}

// One chunk of a chain on each table path.  Each is compiled as a function of
// its own (not inlined into the kernel), so that the register allocation of
// one path does not spill in the others.
template <int NPL, int D0, int D1>
__device__ __noinline__ void chunk_reg(const DevNet &net, const DevChains &ch, const DevSched &sc,
                                       uint8_t *sm, uint32_t codes, uint8_t *region, int chain,
                                       int64_t g_lo, int64_t g_hi, int32_t *flag, int done_value,
                                       int lane)
{
    RegPath<NPL, 4, D0, D1> P;
    P.sm = sm;
    P.codes = codes;
    int8_t *xs = reinterpret_cast<int8_t *>(region);
    uint8_t *on = region + ch.pstride, *pi = on + round16((uint32_t)net.N);
    run_chunk<decltype(P), false>(P, net, ch, sc, chain, g_lo, g_hi, xs, on, pi, flag, done_value,
                                  lane);
}

__device__ __noinline__ void chunk_smem(const DevNet &net, const DevChains &ch, const DevSched &sc,
                                        uint8_t *sm, uint32_t codes, uint8_t *region, int chain,
                                        int64_t g_lo, int64_t g_hi, int32_t *flag, int done_value,
                                        int lane)
{
    SmemPath P;
    P.sm = sm;
    P.codes = codes;
    P.npl = net.npl;
    const uint32_t lw = smem_path_lut_words(net.D, net.npl);
    P.lut = reinterpret_cast<uint32_t *>(region);
    P.node = P.lut + lw;
    uint8_t *after = reinterpret_cast<uint8_t *>(P.node + net.npl * kF_N * 32);
    int8_t *xs = reinterpret_cast<int8_t *>(after);
    uint8_t *on = after + ch.pstride, *pi = on + round16((uint32_t)net.N);
    run_chunk<decltype(P), false>(P, net, ch, sc, chain, g_lo, g_hi, xs, on, pi, flag, done_value,
                                  lane);
}

template <int NPL>
__device__ __noinline__ void chunk_smemreg(const DevNet &net, const DevChains &ch,
                                           const DevSched &sc, uint8_t *sm, uint32_t codes,
                                           uint8_t *region, int chain, int64_t g_lo, int64_t g_hi,
                                           int32_t *flag, int done_value, int lane)
{
    SmemRegPath<NPL> P;
    P.sm = sm;
    P.codes = codes;
    P.lut = reinterpret_cast<uint32_t *>(region);
    const uint32_t lw = smem_path_lut_words(net.D, net.npl);
    int8_t *xs = reinterpret_cast<int8_t *>(region + 4u * lw);
    uint8_t *on = reinterpret_cast<uint8_t *>(xs) + ch.pstride, *pi = on + round16((uint32_t)net.N);
    run_chunk<decltype(P), false>(P, net, ch, sc, chain, g_lo, g_hi, xs, on, pi, flag, done_value,
                                  lane);
}

// Global chain r's chunk cj: its network's descriptors into the warp's shared
// memory, then the chunk on the network's table path (PATH >= 0: a path fixed
// at compile time, so that only that path's code is in the kernel; -1: read
// per network).
template <int PATH>
__device__ __forceinline__ void batch_item(const DevBatch &b, const DevSched &sc, int r, int cj,
                                           DevNet *net_s, DevChains *ch_s, uint8_t *sm,
                                           uint32_t codes, uint8_t *region, int lane)
{
    const int nb = __ldg(b.item_net + r), chain = __ldg(b.item_chain + r);
    warp_copy_words(net_s, b.nets + nb, (int)sizeof(DevNet), lane);
    warp_copy_words(ch_s, b.chains + nb, (int)sizeof(DevChains), lane);
    __syncwarp();
    const DevNet &net = *net_s;
    const DevChains &ch = *ch_s;
    const int64_t g0 = __ldcg(b.g0 + nb);
    const int64_t g_lo = g0 + (int64_t)cj * sc.chunk;
    const int64_t g_hi = min(g0 + b.sweeps, g_lo + sc.chunk);
    const int path = PATH >= 0 ? PATH : __ldg(b.path + nb);
    int32_t *flag = sc.done + r;
    const int dv = cj + 1;
    if constexpr (PATH == 10) {
        chunk_smemreg<10>(net, ch, sc, sm, codes, region, chain, g_lo, g_hi, flag, dv, lane);
        return;
    }
    switch (path) {
    case 1:
        chunk_reg<1, kBatchD0, 1>(net, ch, sc, sm, codes, region, chain, g_lo, g_hi, flag, dv,
                                  lane);
        break;
    case 2:
        chunk_reg<2, kBatchD0, kBatchD1>(net, ch, sc, sm, codes, region, chain, g_lo, g_hi, flag,
                                         dv, lane);
        break;
    case 4:
        chunk_reg<4, kBatchD0, kBatchD1>(net, ch, sc, sm, codes, region, chain, g_lo, g_hi, flag,
                                         dv, lane);
        break;
    case 6:
        chunk_smemreg<6>(net, ch, sc, sm, codes, region, chain, g_lo, g_hi, flag, dv, lane);
        break;
    case 8:
        chunk_smemreg<8>(net, ch, sc, sm, codes, region, chain, g_lo, g_hi, flag, dv, lane);
        break;
    default:
        chunk_smem(net, ch, sc, sm, codes, region, chain, g_lo, g_hi, flag, dv, lane);
        break;
    }
}

__global__ void __launch_bounds__(128, 3) anneal_batch_kernel(DevBatch b, DevSched sc)
{
    extern __shared__ __align__(256) uint8_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    uint8_t *desc = sm + (uint32_t)wpb * kCodeBytesPerWarp;
    DevNet *net_s = reinterpret_cast<DevNet *>(desc) + warp;
    DevChains *ch_s =
        reinterpret_cast<DevChains *>(desc + (uint32_t)wpb * sizeof(DevNet)) + warp;
    const bool large = warp < b.large;
    uint8_t *region = sm + batch_head_bytes(wpb) +
                      (large ? (uint32_t)warp * b.region_bytes
                             : (uint32_t)b.large * b.region_bytes +
                                   (uint32_t)(warp - b.large) * b.region_small);
    const uint32_t codes = (uint32_t)warp * kCodeBytesPerWarp;
    int cls = large && b.total_big > 0 ? 0 : 1;
    for (;;) {
        const int n_cls = cls == 0 ? b.total_big : b.total - b.total_big;
        const int64_t n_items = (int64_t)sc.n_chunks * n_cls;
        unsigned int item = 0;
        if (lane == 0 && n_cls > 0) item = atomicAdd(sc.queue + cls, 1u);
        item = __shfl_sync(kFull, item, 0);
        if (n_cls == 0 || (int64_t)item >= n_items) {
            if (cls == 0) { cls = 1; continue; }
            break;
        }
        const int cj = (int)(item / (unsigned)n_cls);
        const int r = (cls == 0 ? 0 : b.total_big) + (int)(item - (unsigned)cj * (unsigned)n_cls);
        if (cj > 0 && !wait_for_chunk(sc.done + r, cj, sc.err, lane)) return;
        batch_item<-1>(b, sc, r, cj, net_s, ch_s, sm, codes, region, lane);
    }
}

// One phase of a phased batch: the chains [ph.r0, ph.r0 + ph.n) of the
// networks on table path PATH, every warp with a region sized for that path's
// largest network, and the same chunk-major queue as above (the predecessor
// of an item was handed out ph.n items earlier).
template <int PATH>
__global__ void __launch_bounds__(128, PATH == 10 ? smemreg_min_blocks<10>() : 3)
    anneal_phase_kernel(DevBatch b, DevSched sc, BatchPhase ph)
{
    extern __shared__ __align__(256) uint8_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    uint8_t *desc = sm + (uint32_t)wpb * kCodeBytesPerWarp;
    DevNet *net_s = reinterpret_cast<DevNet *>(desc) + warp;
    DevChains *ch_s =
        reinterpret_cast<DevChains *>(desc + (uint32_t)wpb * sizeof(DevNet)) + warp;
    uint8_t *region = sm + batch_head_bytes(wpb) + (uint32_t)warp * ph.region;
    const uint32_t codes = (uint32_t)warp * kCodeBytesPerWarp;
    const int64_t n_items = (int64_t)sc.n_chunks * ph.n;
    for (;;) {
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(sc.queue + ph.queue, 1u);
        item = __shfl_sync(kFull, item, 0);
        if ((int64_t)item >= n_items) break;
        const int cj = (int)(item / (unsigned)ph.n);
        const int r = ph.r0 + (int)(item - (unsigned)cj * (unsigned)ph.n);
        if (cj > 0 && !wait_for_chunk(sc.done + r, cj, sc.err, lane)) return;
        batch_item<PATH>(b, sc, r, cj, net_s, ch_s, sm, codes, region, lane);
    }
}

// Every network has advanced by `sweeps` steps.
__global__ void advance_kernel(int64_t *g0, int32_t n_nets, int64_t sweeps)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n_nets) g0[k] += sweeps;
}

bool batch_path_fits(int npl, int D0, int Drest)
{
    if (npl > kRegSlots) return false;
    if (D0 > kBatchD0) return false;
    return npl == 1 || Drest <= kBatchD1;
}

uint32_t batch_region_bytes(int path, const int *D, int npl, int pstride, int N)
{
    if (path == 6 || path == 8 || path == 10)
        return round16(smem_reg_warp_bytes(smem_path_lut_words(D, npl), pstride, N));
    return warp_region(path == 0, D, npl, pstride, N).bytes;
}

size_t batch_smem_bytes(int wpb, int large, uint32_t region_big, uint32_t region_small)
{
    return batch_head_bytes(wpb) + (size_t)large * region_big + (size_t)(wpb - large) * region_small;
}

cudaError_t batch_resident_warps(int wpb, size_t smem, int sm_count, int *grid)
{
    cudaError_t err = cudaFuncSetAttribute(anneal_batch_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, anneal_batch_kernel, wpb * 32,
                                                        smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *grid = sm_count * per_sm;
    return cudaSuccess;
}

// Queue reset, the batched kernel and the step advance, in stream order (the
// sequence that rn_anneal captures in a CUDA graph).
cudaError_t launch_batch(const DevBatch &b, const DevSched &sc, int wpb, int grid,
                         cudaStream_t st)
{
    const size_t smem = batch_smem_bytes(wpb, b.large, b.region_bytes, b.region_small);
    cudaError_t err = cudaMemsetAsync(sc.queue, 0, kQueueSlots * sizeof(unsigned int), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(sc.done, 0, sizeof(int32_t) * (size_t)b.total, st);
    if (err != cudaSuccess) return err;
    anneal_batch_kernel<<<grid, wpb * 32, smem, st>>>(b, sc);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    advance_kernel<<<(b.n_nets + 127) / 128, 128, 0, st>>>(b.g0, b.n_nets, b.sweeps);
    return cudaGetLastError();
}

namespace {
using PhaseKernel = void (*)(DevBatch, DevSched, BatchPhase);

PhaseKernel phase_kernel(int path)
{
    switch (path) {
    case 1: return anneal_phase_kernel<1>;
    case 2: return anneal_phase_kernel<2>;
    case 4: return anneal_phase_kernel<4>;
    case 6: return anneal_phase_kernel<6>;
    case 8: return anneal_phase_kernel<8>;
    case 10: return anneal_phase_kernel<10>;
    default: return anneal_phase_kernel<0>;
    }
}
}  // namespace

size_t batch_phase_smem(const BatchPhase &ph)
{
    return batch_head_bytes(ph.wpb) + (size_t)ph.wpb * ph.region;
}

cudaError_t batch_phase_grid(BatchPhase &ph, int sm_count)
{
    const PhaseKernel k = phase_kernel(ph.path);
    const size_t smem = batch_phase_smem(ph);
    cudaError_t err =
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, ph.wpb * 32, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    ph.grid = sm_count * per_sm;
    return cudaSuccess;
}

cudaError_t launch_batch_phased(const DevBatch &b, const DevSched &sc, const BatchPhase *ph,
                                int n_ph, cudaStream_t st, cudaEvent_t *marks)
{
    cudaError_t err = cudaMemsetAsync(sc.queue, 0, kQueueSlots * sizeof(unsigned int), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(sc.done, 0, sizeof(int32_t) * (size_t)b.total, st);
    if (err != cudaSuccess) return err;
    for (int k = 0; k < n_ph; ++k) {
        DevSched s = sc;
        // chunks of 16 steps once the phase's chains outnumber its resident warps
        plan_chunks(s, ph[k].n, (int64_t)ph[k].grid * ph[k].wpb);
        if (marks) cudaEventRecord(marks[2 * k], st);
        phase_kernel(ph[k].path)<<<ph[k].grid, ph[k].wpb * 32, batch_phase_smem(ph[k]), st>>>(
            b, s, ph[k]);
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        if (marks) cudaEventRecord(marks[2 * k + 1], st);
    }
    advance_kernel<<<(b.n_nets + 127) / 128, 128, 0, st>>>(b.g0, b.n_nets, b.sweeps);
    return cudaGetLastError();
}

}  // namespace rn
