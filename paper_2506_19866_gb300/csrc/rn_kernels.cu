// rn_kernels.cu -- initialisation, level-sync and evaluate kernels, and the
// dispatch of every launch to its compiled layout.
//
//   init_kernel      the seeded sample-and-repair x0 of each chain
//   argmin_kernel / broadcast_kernel
//                    the serial argmin + broadcast that ends a level of Table 1
//   evaluate_kernel  (rn_kernels.cuh) instantiated with register capacity 16
#include "rn_kernels.cuh"

namespace rn {

// Seeded sample-and-repair x0 (the paper draws x0 with a constraint solver),
// one warp per chain: uniform draws, then an activating in-edge for every node
// without one, then a nonzero out-edge for every node without one.  Lane l
// draws parameters 4b .. 4b + 3 of blocks b = l, l + 32, ... from one Philox
// call per block (counter (b, 0, chain, 1), word j % 4 for parameter j) and
// stores them as one 32-bit word, so the row is written in whole lines.  In
// the repairs the lanes take the nodes: a node's first repair reads and writes
// only its own in-edges, its second only its own out-edges, so the nodes of a
// repair are independent and the lanes give the result of the node-by-node
// order (the second repair sees all of the first).
__global__ void init_kernel(DevNet net, DevChains ch, int32_t *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t chain = (int64_t)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (chain >= ch.n) return;   // whole warps
    int8_t *x = ch.x_cur + (size_t)chain * ch.pstride;
    const int E = net.E, N = net.N, P = net.P;
    for (int b = lane; b < ch.pstride / 4; b += 32) {
        uint32_t word4 = 0;
        const int j0 = 4 * b;
        if (j0 < P) {
            const uint4 r = philox(ch.seed, (uint32_t)b, 0u, (uint32_t)chain, 1u);
            const uint32_t words[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = j0 + q;
                if (j >= P) break;
                int8_t v;
                if (net.frozen && net.frozen[j]) {
                    v = net.frozen_val[j];
                } else {
                    int kind, idx;
                    if (j < E) { kind = 0; idx = j; }
                    else if (j < 2 * E) { kind = 1; idx = j - E; }
                    else if (j < 3 * E) { kind = 2; idx = j - 2 * E; }
                    else if (j < 3 * E + N) { kind = 3; idx = j - 3 * E; }
                    else if (j < 3 * E + 2 * N) { kind = 4; idx = j - 3 * E - N; }
                    else { kind = 5; idx = j - 3 * E - 2 * N; }
                    int8_t vals[6];
                    const int nd = domain(kind, kind == 3 && net.fast[idx], vals);
                    v = vals[pick(words[q], (uint32_t)nd)];
                }
                word4 |= (uint32_t)(uint8_t)v << (8 * q);
            }
        }
        reinterpret_cast<uint32_t *>(x)[b] = word4;
    }
    __syncwarp();
    int ok = 1;
    for (int i = lane; i < N; i += 32) {
        int has = 0, n_cand = 0;
        for (int k = net.in_ptr[i]; k < net.in_ptr[i + 1]; ++k) {
            const int e = net.in_edges[k];
            has |= (x[e] != 0) && (x[E + e] == 1);
            const bool p_ok = !(net.frozen && net.frozen[E + e]) || net.frozen_val[E + e] == 1;
            const bool w_ok = !(net.frozen && net.frozen[e]) || net.frozen_val[e] != 0;
            n_cand += p_ok && w_ok;
        }
        if (has) continue;
        if (n_cand == 0) { ok = 0; continue; }
        const uint4 q = philox(ch.seed, (uint32_t)i, 0u, (uint32_t)chain, 3u);
        int want = (int)pick(q.x, (uint32_t)n_cand);
        for (int k = net.in_ptr[i]; k < net.in_ptr[i + 1]; ++k) {
            const int e = net.in_edges[k];
            const bool p_ok = !(net.frozen && net.frozen[E + e]) || net.frozen_val[E + e] == 1;
            const bool w_ok = !(net.frozen && net.frozen[e]) || net.frozen_val[e] != 0;
            if (!(p_ok && w_ok)) continue;
            if (want-- != 0) continue;
            if (!(net.frozen && net.frozen[E + e])) x[E + e] = 1;
            if (!(net.frozen && net.frozen[e])) x[e] = (int8_t)(1 + (q.y & 1u));
            break;
        }
    }
    ok = __all_sync(0xffffffffu, ok);
    __syncwarp();
    if (ok) {
        for (int i = lane; i < N; i += 32) {
            int has = 0, n_cand = 0;
            for (int k = net.out_ptr[i]; k < net.out_ptr[i + 1]; ++k) {
                const int e = net.out_edges[k];
                has |= x[e] != 0;
                n_cand += !(net.frozen && net.frozen[e]);
            }
            if (has) continue;
            if (n_cand == 0) { ok = 0; continue; }
            const uint4 q = philox(ch.seed, (uint32_t)i, 1u, (uint32_t)chain, 3u);
            int want = (int)pick(q.x, (uint32_t)n_cand);
            for (int k = net.out_ptr[i]; k < net.out_ptr[i + 1]; ++k) {
                const int e = net.out_edges[k];
                if (net.frozen && net.frozen[e]) continue;
                if (want-- != 0) continue;
                x[e] = (int8_t)(1 + (q.y & 1u));
                break;
            }
        }
        ok = __all_sync(0xffffffffu, ok);
    }
    __syncwarp();
    const uint4 *src = reinterpret_cast<const uint4 *>(x);
    uint4 *dst = reinterpret_cast<uint4 *>(ch.x_best + (size_t)chain * ch.pstride);
    for (int k = lane; k < ch.pstride / 16; k += 32) dst[k] = src[k];
    if (lane == 0) {
        ch.cnt[3 * (size_t)chain + 0] = 0;
        ch.cnt[3 * (size_t)chain + 1] = 0;
        ch.cnt[3 * (size_t)chain + 2] = 0;
        status[chain] = ok ? 0 : -2;
    }
}

// Table 1, end of a level: the lowest delta_best over the chains (lowest chain
// index on ties).  One block.
__global__ void argmin_kernel(const int32_t *__restrict__ d_best, int32_t n, int32_t group,
                              int32_t *out)
{
    // block b: the chains of group b, [b * group, min(n, (b + 1) * group))
    __shared__ unsigned long long best[32];
    unsigned long long b = ~0ull;
    const int first = blockIdx.x * group;
    const int end = min(n, first + group);
    for (int k = first + threadIdx.x; k < end; k += blockDim.x) {
        const unsigned long long key =
            ((unsigned long long)(uint32_t)d_best[k] << 32) | (uint32_t)k;
        b = min(b, key);
    }
    for (int o = 16; o > 0; o >>= 1) b = min(b, __shfl_xor_sync(kFull, b, o));
    if ((threadIdx.x & 31) == 0) best[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x < 32) {
        b = threadIdx.x < (blockDim.x >> 5) ? best[threadIdx.x] : ~0ull;
        for (int o = 16; o > 0; o >>= 1) b = min(b, __shfl_xor_sync(kFull, b, o));
        if (threadIdx.x == 0) out[blockIdx.x] = (int32_t)(uint32_t)b;
    }
}

// ... and its broadcast into every chain's x_best (from its group's winner).
__global__ void broadcast_kernel(DevChains ch, const int32_t *win, int32_t group)
{
    const int rows_per_block = blockDim.x / 32;
    const int lane = threadIdx.x & 31;
    const int chain = blockIdx.x * rows_per_block + (threadIdx.x >> 5);
    if (chain >= ch.n) return;
    const int w = win[chain / group];
    if (chain == w) return;
    warp_copy16(ch.x_best + (size_t)chain * ch.pstride, ch.x_best + (size_t)w * ch.pstride,
                ch.pstride, lane);
    if (lane == 0) ch.d_best[chain] = ch.d_best[w];
}

// Simulate(x) with the shared-memory tables (networks of more than 128 nodes).
__global__ void __launch_bounds__(128) evaluate_smem_kernel(DevNet net, const int8_t *__restrict__ X,
                                                            int64_t xstride, int32_t n,
                                                            int32_t *__restrict__ score,
                                                            int32_t *__restrict__ score2,
                                                            uint8_t *__restrict__ traj,
                                                            uint32_t region_bytes,
                                                            uint32_t lut_words)
{
    extern __shared__ __align__(256) uint8_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    SmemPath P = make_smem_path(net, sm, warp, wpb, region_bytes, lut_words);
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

// The annealing kernel with the shared-memory tables.
__global__ void __launch_bounds__(128, 2)
    anneal_smem_kernel(DevNet net, DevChains ch, DevSched sc, uint32_t region_bytes,
                       uint32_t lut_words)
{
    extern __shared__ __align__(256) uint8_t sm[];
    anneal_items(net, ch, sc, sm, region_bytes, [&](int warp, int wpb) {
        SmemPathR P;
        static_cast<SmemPath &>(P) = make_smem_path(net, sm, warp, wpb, region_bytes, lut_words);
        return P;
    });
}

template <int NPL, int CG>
static cudaError_t launch_eval_t(const DevNet &net, const int8_t *X, int64_t xstride, int32_t n,
                                 int32_t *score, int32_t *score2, uint8_t *traj, int grid,
                                 cudaStream_t st)
{
    evaluate_kernel<NPL, CG, 16, 16><<<grid, 128, 4 * kCodeBytesPerWarp, st>>>(
        net, X, xstride, n, score, score2, traj);
    return cudaGetLastError();
}

cudaError_t launch_evaluate(const DevNet &net, const int8_t *X, int64_t xstride, int32_t n,
                            int32_t *score, int32_t *score2, uint8_t *traj, int sm_count,
                            cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (net.lanes != 32) return launch_evaluate_block(net, X, xstride, n, score, score2, traj,
                                                      sm_count, st);
    int grid = (n + 3) / 4;
    if (grid > sm_count * 16) grid = sm_count * 16;
    if (smemreg_layout(net.npl))
        return launch_evaluate_smemreg(net, X, xstride, n, score, score2, traj, grid, st);
    if (net.npl > kRegSlots) {
        const WarpRegion R = warp_region(true, net.D, net.npl, 0, 0);
        const size_t smem = 4 * ((size_t)kCodeBytesPerWarp + R.bytes);
        cudaError_t e = cudaFuncSetAttribute(evaluate_smem_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        evaluate_smem_kernel<<<grid, 128, smem, st>>>(net, X, xstride, n, score, score2, traj,
                                                      R.bytes, R.lut_words);
        return cudaGetLastError();
    }
#define RN_EV(NPL_, CG_)                                                                  \
    if (net.npl == NPL_ && net.cg == CG_)                                                 \
        return launch_eval_t<NPL_, CG_>(net, X, xstride, n, score, score2, traj, grid, st);
    RN_EV(1, 1) RN_EV(1, 4) RN_EV(2, 1) RN_EV(2, 4) RN_EV(4, 1) RN_EV(4, 4)
#undef RN_EV
    return cudaErrorNotSupported;
}

bool anneal_layout_supported(int npl, int cg, int d0, int d1)
{
    if (cg != 1 && cg != 4) return false;
    if (npl == 1) return d0 == 4 || d0 == 8 || d0 == 12 || d0 == 16;
    if (npl != 2 && npl != 4) return false;
    static const int pairs[][2] = {{4, 4}, {8, 4}, {8, 8}, {12, 8}, {16, 8}, {16, 16}};
    for (auto &p : pairs)
        if (p[0] == d0 && p[1] == d1) return true;
    return false;
}

void anneal_capacity(int npl, int D0, int Drest, int *d0, int *d1)
{
    auto up = [](int d) { return d <= 4 ? 4 : d <= 8 ? 8 : d <= 12 ? 12 : d <= 16 ? 16 : -1; };
    *d0 = up(D0);
    if (npl == 1) {
        *d1 = 1;
        return;
    }
    static const int pairs[][2] = {{4, 4}, {8, 4}, {8, 8}, {12, 8}, {16, 8}, {16, 16}};
    *d1 = -1;
    for (auto &p : pairs)   // smallest compiled pair covering (D0, Drest)
        if (p[0] >= D0 && p[1] >= Drest) {
            *d0 = p[0];
            *d1 = p[1];
            return;
        }
    *d0 = -1;
}

static cudaError_t launch_anneal_smem(const DevNet &net, const DevChains &ch, const DevSched &sc,
                                      int sm_count, cudaStream_t st)
{
    int wpb = 4;
    const WarpRegion R = warp_region(true, net.D, net.npl, ch.pstride, net.N);
    size_t smem = (size_t)wpb * (kCodeBytesPerWarp + R.bytes);
    cudaError_t err = cudaFuncSetAttribute(anneal_smem_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, anneal_smem_kernel, wpb * 32,
                                                        smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = sm_count * per_sm;
    if (ch.n > 0 && ch.n < grid * wpb) {
        // fewer chains than resident warps: a block of one warp per chain, which
        // the hardware spreads evenly over the SMs
        wpb = 1;
        grid = ch.n;
        smem = kCodeBytesPerWarp + R.bytes;
    }
    DevSched s = sc;
    plan_chunks(s, ch.n, (int64_t)grid * wpb);
    err = cudaMemsetAsync(s.queue, 0, sizeof(unsigned int), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(s.done, 0, sizeof(int32_t) * (size_t)ch.n, st);
    if (err != cudaSuccess) return err;
    anneal_smem_kernel<<<grid, wpb * 32, smem, st>>>(net, ch, s, R.bytes, R.lut_words);
    return cudaGetLastError();
}

cudaError_t launch_anneal(const DevNet &net, int d0, int d1, const DevChains &ch,
                          const DevSched &sc, int sm_count, cudaStream_t st)
{
    if (ch.n <= 0 || sc.g1 <= sc.g0) return cudaSuccess;
    // one condition: four chains per warp in the byte lanes once the chains
    // outnumber the one-chain kernel's resident warps (12 per SM).  Below that
    // every chain has a warp of its own and one chain per warp finishes a step
    // sooner (measured on the 102- and 723-parameter networks: one chain per
    // warp ahead at 1024 chains, four per warp ahead at 2048 and 3072).
    // Exact early rejection stops a single chain's simulation, so it keeps one
    // chain per warp.
    if (!sc.early_reject && ch.n >= 12 * sm_count && chains4_layout(net, d0, d1))
        return launch_anneal_chains4(net, d0, d1, ch, sc, sm_count, st);
    if (smemreg_layout(net.npl)) return launch_anneal_smemreg(net, ch, sc, sm_count, st);
    if (net.npl > kRegSlots) return launch_anneal_smem(net, ch, sc, sm_count, st);
    switch (net.npl) {
    case 1: return launch_anneal_npl1(net, d0, d1, ch, sc, sm_count, st);
    case 2: return launch_anneal_npl2(net, d0, d1, ch, sc, sm_count, st);
    case 4: return launch_anneal_npl4(net, d0, d1, ch, sc, sm_count, st);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_init(const DevNet &net, const DevChains &ch, int32_t *status, cudaStream_t st)
{
    init_kernel<<<(unsigned)((ch.n + 3) / 4), 128, 0, st>>>(net, ch, status);
    return cudaGetLastError();
}

// One warp runs the work queue's wait, with a short poll limit, on a counter
// that nothing advances: the wait gives up, sets the error flag and returns,
// without any fault.  out = 1 if the wait was (wrongly) satisfied, else 0.
constexpr int kSelftestPolls = 1 << 12;

__global__ void wait_selftest_kernel(const int32_t *never, int32_t *err, int32_t *out)
{
    const bool ok = wait_for_chunk<kSelftestPolls>(never, 1, err, (int)(threadIdx.x & 31));
    if (threadIdx.x == 0) *out = ok ? 1 : 0;
}

cudaError_t launch_wait_selftest(const int32_t *never, int32_t *err, int32_t *out,
                                 cudaStream_t st)
{
    wait_selftest_kernel<<<1, 32, 0, st>>>(never, err, out);
    return cudaGetLastError();
}

cudaError_t launch_level_sync(const DevChains &ch, int32_t *winner, int32_t group,
                              cudaStream_t st)
{
    const int G = group > 0 && group < ch.n ? group : ch.n;
    const int groups = (ch.n + G - 1) / G;
    const int threads = G >= 1024 ? 1024 : ((G + 31) / 32) * 32;
    argmin_kernel<<<groups, threads, 0, st>>>(ch.d_best, ch.n, G, winner);
    broadcast_kernel<<<(ch.n + 7) / 8, 256, 0, st>>>(ch, winner, G);
    return cudaGetLastError();
}

}  // namespace rn
