// rn_kernels.cuh -- kernel templates of the annealing path (instantiated in
// rn_anneal{1,2,4}.cu and rn_kernels.cu).
//
//   evaluate_kernel  Simulate(x) of Table 1 for a batch of vectors, warp each
//   anneal_kernel    persistent annealing kernel, warp per chain (Table 1 inner
//                    loop: GetCandidate, Simulate, Metropolis acceptance)
#pragma once

#include "rn_device.cuh"
#include "rn_launch.h"

namespace rn {

// Shared-memory layout of one warp in the annealing kernel; every warp's base
// is 256-byte aligned (the state-code offsets in the table words are one byte).
struct WarpSmem {
    uint32_t per_warp;   // bytes per warp (multiple of 256)
    uint32_t x_off;      // current vector x (pstride bytes)
    uint32_t out_off;    // out_nz[N]: out-edges with w != 0
    uint32_t pos_off;    // pos_in[N]: in-edges with w != 0 and p = +1
};

__host__ __device__ inline WarpSmem warp_smem(int pstride, int N)
{
    WarpSmem s;
    s.x_off = 256u;
    s.out_off = s.x_off + (uint32_t)pstride;
    s.pos_off = s.out_off + (((uint32_t)N + 15u) & ~15u);
    s.per_warp = (s.pos_off + (((uint32_t)N + 15u) & ~15u) + 255u) & ~255u;
    return s;
}

// ---------------------------------------------------------------- evaluate --
template <int NPL, int CG, int D0, int D1>
__global__ void __launch_bounds__(128) evaluate_kernel(DevNet net, const int8_t *__restrict__ X,
                                                       int64_t xstride, int32_t n,
                                                       int32_t *__restrict__ score,
                                                       int32_t *__restrict__ score2,
                                                       uint8_t *__restrict__ traj)
{
    extern __shared__ __align__(256) uint8_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t base = (uint32_t)warp * 256u;
    const int wpb = blockDim.x >> 5;
    for (int v = blockIdx.x * wpb + warp; v < n; v += gridDim.x * wpb) {
        Regs<NPL, D0, D1> R;
        load_regs<NPL, D0, D1>(R, net, X + (size_t)v * xstride, lane);
        uint8_t *tv = traj ? traj + (size_t)v * net.C * net.T * net.N : nullptr;
        const int32_t y = simulate<NPL, CG, D0, D1>(R, net, sm, base, lane, tv);
        if (lane == 0) {
            score[v] = y;
            if (score2) score2[v] = y;
        }
        __syncwarp();
    }
}

// -------------------------------------------------------------- annealing --

// Domain of parameter kind k (Section 2.1: w, p, t; Section 2.2: u, m, d).
__device__ __forceinline__ int domain(int kind, bool fast, int8_t (&vals)[6])
{
    switch (kind) {
    case 0: vals[0] = 0; vals[1] = 1; vals[2] = 2; return 3;
    case 1: vals[0] = -1; vals[1] = 0; vals[2] = 1; return 3;
    case 2: vals[0] = 1; vals[1] = 2; return 2;
    case 3:
        if (fast) { vals[0] = 10; vals[1] = 11; vals[2] = 12; return 3; }
#pragma unroll
        for (int k = 0; k < 6; ++k) vals[k] = (int8_t)(k + 1);
        return 6;
    case 4: vals[0] = 0; vals[1] = 1; vals[2] = 2; return 3;
    default: vals[0] = 1; vals[1] = 2; return 2;
    }
}

// Rebuild the per-chain constraint counters of Section 2.5.3 from x.
__device__ __forceinline__ void count_constraints(const DevNet &net, const int8_t *x,
                                                  uint8_t *out_nz, uint8_t *pos_in, int lane)
{
    for (int i = lane; i < net.N; i += 32) {
        int o = 0, q = 0;
        for (int k = net.out_ptr[i]; k < net.out_ptr[i + 1]; ++k) o += x[net.out_edges[k]] != 0;
        for (int k = net.in_ptr[i]; k < net.in_ptr[i + 1]; ++k) {
            const int e = net.in_edges[k];
            q += (x[e] != 0) && (x[net.E + e] == 1);
        }
        out_nz[i] = (uint8_t)min(o, 255);
        pos_in[i] = (uint8_t)min(q, 255);
    }
}

__device__ __forceinline__ void warp_copy16(void *dst, const void *src, int bytes, int lane)
{
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    for (int k = lane; k < (bytes >> 4); k += 32) d[k] = s[k];
}

// Replace the table word of (slot, d) == kd (encoded slot * 32 + d).
template <int NPL, int D0, int D1>
__device__ __forceinline__ void set_word(Regs<NPL, D0, D1> &R, int kd, uint32_t w)
{
    for_each_word<NPL, D0, D1>(R, [&](int k, int d, uint32_t &word) {
        word = (k * 32 + d == kd) ? w : word;
    });
}

template <int NPL, int D0, int D1>
__device__ __forceinline__ void set_node(Regs<NPL, D0, D1> &R, int kind, int slot, int v)
{
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
        if (k != slot) continue;
        if (kind == 3) R.u[k] = v;
        else if (kind == 4) R.m1[k] = v + 1;
        else R.d2[k] = v == 2;
    }
}

// Three 4-warp blocks per SM (at most 168 registers a thread) unless the
// register tables alone need more room.
template <int NPL, int D0, int D1>
constexpr int anneal_min_blocks()
{
    return D0 + (NPL - 1) * D1 <= 40 ? 3 : 2;
}

template <int NPL, int CG, int D0, int D1>
__global__ void __launch_bounds__(128, (anneal_min_blocks<NPL, D0, D1>()))
    anneal_kernel(DevNet net, DevChains ch, DevSched sc)
{
    extern __shared__ __align__(256) uint8_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const WarpSmem L = warp_smem(ch.pstride, net.N);
    const uint32_t base = (uint32_t)warp * L.per_warp;
    int8_t *xs = reinterpret_cast<int8_t *>(sm + base + L.x_off);
    uint8_t *out_nz = sm + base + L.out_off;
    uint8_t *pos_in = sm + base + L.pos_off;
    const int E = net.E, N = net.N;

    // chain c is processed by block c % gridDim.x, so every block gets the same
    // number of chains within one
    for (int chain = blockIdx.x + gridDim.x * warp; chain < ch.n; chain += gridDim.x * wpb) {
        int8_t *xg = ch.x_cur + (size_t)chain * ch.pstride;
        int8_t *xb = ch.x_best + (size_t)chain * ch.pstride;
        warp_copy16(xs, xg, ch.pstride, lane);
        __syncwarp();
        Regs<NPL, D0, D1> R;
        load_regs<NPL, D0, D1>(R, net, xs, lane);
        count_constraints(net, xs, out_nz, pos_in, lane);
        __syncwarp();
        int32_t d_cur = ch.d_cur[chain], d_best = ch.d_best[chain];
        int32_t n_acc = 0, n_up = 0, n_null = 0;

        int64_t level = sc.g0 / sc.iters;
        int64_t in_level = sc.g0 - level * sc.iters;
        for (int64_t g = sc.g0; g < sc.g1; ++g) {
            if (in_level == sc.iters) {
                in_level = 0;
                ++level;
            }
            if (sc.reset_to_best && in_level == 0) {
                // Table 1: every level starts from the chain's x_best
                warp_copy16(xs, xb, ch.pstride, lane);
                __syncwarp();
                load_regs<NPL, D0, D1>(R, net, xs, lane);
                count_constraints(net, xs, out_nz, pos_in, lane);
                __syncwarp();
                d_cur = d_best;
            }
            ++in_level;
            const uint4 r = philox(ch.seed, (uint32_t)g, (uint32_t)((uint64_t)g >> 32),
                                   (uint32_t)chain, 0u);
            if (net.n_free == 0) {
                ++n_null;
                continue;
            }
            // GetCandidate: the pick(r0)-th free parameter ...
            const int j = net.free_list[pick(r.x, (uint32_t)net.n_free)];
            int kind, idx;
            if (j < 3 * E) { kind = j / E; idx = j - kind * E; }
            else { const int t = j - 3 * E; kind = 3 + t / N; idx = t - (kind - 3) * N; }
            const int cur = xs[j];
            int8_t vals[6];
            const int nd = domain(kind, kind == 3 && net.fast[idx], vals);
            // ... and the pick(r1)-th of its values != current that keep the
            // constraints of Section 2.5.3
            bool blocked0 = false, blocked_all = false;
            if (kind == 0 && cur != 0) {
                const int a = net.src[idx], b = net.dst[idx];
                blocked0 = out_nz[a] < 2 || (xs[E + idx] == 1 && pos_in[b] < 2);
            } else if (kind == 1 && cur == 1 && xs[idx] != 0) {
                blocked_all = pos_in[net.dst[idx]] < 2;
            }
            int8_t alts[6];
            int n_alt = 0;
            if (!blocked_all) {
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    if (k >= nd) break;
                    const int v = vals[k];
                    if (v == cur || (blocked0 && v == 0)) continue;
                    alts[n_alt++] = (int8_t)v;
                }
            }
            if (n_alt == 0) {
                ++n_null;
                continue;
            }
            const int v = alts[pick(r.y, (uint32_t)n_alt)];

            // apply the candidate to the owner lane's registers
            int owner, slot_or_kd;
            uint32_t w_old = 0;
            if (kind < 3) {
                const int pos = net.edge_pos[idx];
                owner = pos >> 16;
                slot_or_kd = ((pos >> 8) & 0xff) * 32 + (pos & 0xff);
                int w = xs[idx], p = xs[E + idx], t = xs[2 * E + idx];
                const uint32_t q2 = net.edge_q2[idx];
                w_old = edge_word(w, p, t, q2);
                if (kind == 0) w = v; else if (kind == 1) p = v; else t = v;
                if (lane == owner) set_word<NPL, D0, D1>(R, slot_or_kd, edge_word(w, p, t, q2));
            } else {
                const int q = net.node_q[idx];
                owner = q / NPL;
                slot_or_kd = q - owner * NPL;
                if (lane == owner) set_node<NPL, D0, D1>(R, kind, slot_or_kd, v);
            }
            const int32_t d_cand = simulate<NPL, CG, D0, D1>(R, net, sm, base, lane, nullptr);

            // Metropolis acceptance against the host-computed threshold table
            const int32_t dE = d_cand - d_cur;
            bool accept = dE <= 0;
            if (!accept) {
                const int64_t l = level - sc.level0;
                if (dE <= sc.thr_len[l]) accept = r.z < __ldg(sc.thr + sc.thr_off[l] + dE - 1);
            }
            if (accept) {
                if (lane == 0) {
                    if (kind == 0 && (cur == 0) != (v == 0)) {
                        const int delta = v != 0 ? 1 : -1;
                        out_nz[net.src[idx]] += delta;
                        if (xs[E + idx] == 1) pos_in[net.dst[idx]] += delta;
                    } else if (kind == 1 && xs[idx] != 0) {
                        if (cur == 1) pos_in[net.dst[idx]] -= 1;
                        if (v == 1) pos_in[net.dst[idx]] += 1;
                    }
                    xs[j] = (int8_t)v;
                }
                __syncwarp();
                d_cur = d_cand;
                ++n_acc;
                n_up += dE > 0;
                if (d_cand < d_best) {
                    d_best = d_cand;
                    warp_copy16(xb, xs, ch.pstride, lane);
                }
            } else if (lane == owner) {
                if (kind < 3) set_word<NPL, D0, D1>(R, slot_or_kd, w_old);
                else set_node<NPL, D0, D1>(R, kind, slot_or_kd, cur);
            }
            __syncwarp();
        }
        warp_copy16(xg, xs, ch.pstride, lane);
        if (lane == 0) {
            ch.d_cur[chain] = d_cur;
            ch.d_best[chain] = d_best;
            ch.cnt[3 * (size_t)chain + 0] += n_acc;
            ch.cnt[3 * (size_t)chain + 1] += n_up;
            ch.cnt[3 * (size_t)chain + 2] += n_null;
        }
        __syncwarp();
    }
}

template <int NPL, int CG, int D0, int D1>
cudaError_t launch_anneal_t(const DevNet &net, const DevChains &ch, const DevSched &sc,
                            int sm_count, cudaStream_t st)
{
    const int wpb = 4;
    const WarpSmem L = warp_smem(ch.pstride, net.N);
    const size_t smem = (size_t)wpb * L.per_warp;
    auto kern = anneal_kernel<NPL, CG, D0, D1>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = sm_count * per_sm;
    const int need = (ch.n + wpb - 1) / wpb;
    if (grid > need) grid = need;
    kern<<<grid, wpb * 32, smem, st>>>(net, ch, sc);
    return cudaGetLastError();
}

// Register capacities (D0 for slot 0, D1 for the other slots) compiled for the
// annealing kernel; the evaluate kernel uses (16, 16) throughout.
#define RN_ANNEAL_PAIRS(X, NPL_, CG_)                                           \
    X(NPL_, CG_, 4, 4) X(NPL_, CG_, 8, 4) X(NPL_, CG_, 8, 8) X(NPL_, CG_, 12, 8) \
    X(NPL_, CG_, 16, 8) X(NPL_, CG_, 16, 16)

cudaError_t launch_anneal_npl1(const DevNet &net, int d0, int d1, const DevChains &ch,
                               const DevSched &sc, int sm_count, cudaStream_t st);
cudaError_t launch_anneal_npl2(const DevNet &net, int d0, int d1, const DevChains &ch,
                               const DevSched &sc, int sm_count, cudaStream_t st);
cudaError_t launch_anneal_npl4(const DevNet &net, int d0, int d1, const DevChains &ch,
                               const DevSched &sc, int sm_count, cudaStream_t st);

}  // namespace rn
