// rn_smemreg.cu -- kernels of the hybrid path (rn_smem.cuh SmemRegPath): 6, 8
// or 10 nodes per lane, table words in the warp's shared memory, byte-SIMD node
// state in registers.  Same persistent work queue and per-chain code as the
// other warp-per-chain kernels (rn_kernels.cuh).
#include "rn_kernels.cuh"

namespace rn {
namespace {

template <int NPL>
struct SmemRegPathR : SmemRegPath<NPL> {
    uint32_t lut_words;
    __device__ uint8_t *node_end() const
    {
        return reinterpret_cast<uint8_t *>(this->lut + lut_words);
    }
};

template <int NPL>
__device__ __forceinline__ SmemRegPathR<NPL> make_path(uint8_t *sm, int warp, int wpb,
                                                       uint32_t region_bytes, uint32_t lut_words)
{
    SmemRegPathR<NPL> P;
    P.sm = sm;
    P.codes = (uint32_t)warp * kCodeBytesPerWarp;
    P.lut = reinterpret_cast<uint32_t *>(sm + (uint32_t)wpb * kCodeBytesPerWarp +
                                         (uint32_t)warp * region_bytes);
    P.lut_words = lut_words;
    return P;
}

template <int NPL>
__global__ void __launch_bounds__(128, smemreg_min_blocks<NPL>())
    anneal_smemreg_kernel(DevNet net, DevChains ch, DevSched sc, uint32_t region_bytes,
                          uint32_t lut_words)
{
    extern __shared__ __align__(256) uint8_t sm[];
    anneal_items(net, ch, sc, sm, region_bytes, [&](int warp, int wpb) {
        return make_path<NPL>(sm, warp, wpb, region_bytes, lut_words);
    });
}

template <int NPL>
__global__ void __launch_bounds__(128)
    evaluate_smemreg_kernel(DevNet net, const int8_t *__restrict__ X, int64_t xstride, int32_t n,
                            int32_t *__restrict__ score, int32_t *__restrict__ score2,
                            uint8_t *__restrict__ traj, uint32_t region_bytes, uint32_t lut_words)
{
    extern __shared__ __align__(256) uint8_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    auto P = make_path<NPL>(sm, warp, wpb, region_bytes, lut_words);
    for (int v = blockIdx.x * wpb + warp; v < n; v += gridDim.x * wpb) {
        P.load(net, X + (size_t)v * xstride, lane);
        __syncwarp();
        uint8_t *tv = traj ? traj + (size_t)v * net.C * net.T * net.N : nullptr;
        const int32_t y = P.simulate(net, lane, tv);
        if (lane == 0) {
            score[v] = y;
            if (score2) score2[v] = y;
        }
        __syncwarp();
    }
}

template <int NPL>
cudaError_t launch_anneal_t(const DevNet &net, const DevChains &ch, const DevSched &sc,
                            int sm_count, cudaStream_t st)
{
    int wpb = 4;
    const uint32_t lw = smem_path_lut_words(net.D, net.npl);
    const uint32_t rb = round16(smem_reg_warp_bytes(lw, ch.pstride, net.N));
    size_t smem = (size_t)wpb * (kCodeBytesPerWarp + rb);
    cudaError_t err = cudaFuncSetAttribute(anneal_smemreg_kernel<NPL>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, anneal_smemreg_kernel<NPL>,
                                                        wpb * 32, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = sm_count * per_sm;
    if (ch.n > 0 && ch.n < grid * wpb) {
        // fewer chains than resident warps: a block of one warp per chain, which
        // the hardware spreads evenly over the SMs
        wpb = 1;
        grid = ch.n;
        smem = kCodeBytesPerWarp + rb;
    }
    DevSched s = sc;
    plan_chunks(s, ch.n, (int64_t)grid * wpb);
    err = cudaMemsetAsync(s.queue, 0, sizeof(unsigned int), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(s.done, 0, sizeof(int32_t) * (size_t)ch.n, st);
    if (err != cudaSuccess) return err;
    anneal_smemreg_kernel<NPL><<<grid, wpb * 32, smem, st>>>(net, ch, s, rb, lw);
    return cudaGetLastError();
}

template <int NPL>
cudaError_t launch_evaluate_t(const DevNet &net, const int8_t *X, int64_t xstride, int32_t n,
                              int32_t *score, int32_t *score2, uint8_t *traj, int grid,
                              cudaStream_t st)
{
    const uint32_t lw = smem_path_lut_words(net.D, net.npl);
    const uint32_t rb = round16(smem_reg_warp_bytes(lw, 0, net.N));
    const size_t smem = 4 * ((size_t)kCodeBytesPerWarp + rb);
    const cudaError_t e = cudaFuncSetAttribute(evaluate_smemreg_kernel<NPL>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
    evaluate_smemreg_kernel<NPL><<<grid, 128, smem, st>>>(net, X, xstride, n, score, score2, traj,
                                                          rb, lw);
    return cudaGetLastError();
}

}  // namespace

bool smemreg_layout(int npl)
{
    return npl == kSmemRegSlots[0] || npl == kSmemRegSlots[1] || npl == kSmemRegSlots[2];
}

cudaError_t launch_anneal_smemreg(const DevNet &net, const DevChains &ch, const DevSched &sc,
                                  int sm_count, cudaStream_t st)
{
    if (net.npl == 6) return launch_anneal_t<6>(net, ch, sc, sm_count, st);
    if (net.npl == 8) return launch_anneal_t<8>(net, ch, sc, sm_count, st);
    if (net.npl == 10) return launch_anneal_t<10>(net, ch, sc, sm_count, st);
    return cudaErrorNotSupported;
}

cudaError_t launch_evaluate_smemreg(const DevNet &net, const int8_t *X, int64_t xstride,
                                    int32_t n, int32_t *score, int32_t *score2, uint8_t *traj,
                                    int grid, cudaStream_t st)
{
    if (net.npl == 6) return launch_evaluate_t<6>(net, X, xstride, n, score, score2, traj, grid, st);
    if (net.npl == 8) return launch_evaluate_t<8>(net, X, xstride, n, score, score2, traj, grid, st);
    if (net.npl == 10)
        return launch_evaluate_t<10>(net, X, xstride, n, score, score2, traj, grid, st);
    return cudaErrorNotSupported;
}

}  // namespace rn
