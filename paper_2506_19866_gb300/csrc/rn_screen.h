// rn_screen.h -- arguments and candidate selection of the screened annealing
// step (the learned proposal screen, an addition to Table 1), shared by the
// warp-path kernels (rn_mlp.cu) and the block-path finish (rn_block.cu).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rn_kernels.cuh"

namespace rn {

struct ScreenArgs {
    DevNet net;
    DevChains ch;
    int64_t g;                          // global step
    int32_t K, top, H1, nparts;
    uint64_t eps_thr;                   // fallback iff word 3 < eps_thr (<= 2^32)
    const int32_t *row_base;
    const __nv_bfloat16 *W1b;           // [Dp][H1]
    const float *b3;
    float *A1;                          // [chains][H1]
    __nv_bfloat16 *hc;                  // [M][H1] (hidden rows through memory)
    int2 *rows;                         // [M] W1 rows (new, old) per candidate (produced in the GEMM)
    const float *pc;                    // [M][nparts]
    int32_t *cand;                      // [chains][K]
};

constexpr int kScreenWarps = 4;
constexpr int kMaxGroups = 4;           // H1 <= 4 * 256
constexpr int kMaxTop = 4;

__device__ __forceinline__ uint4 step_draw(const DevChains &ch, int64_t g, int chain, uint32_t tag)
{
    return philox(ch.seed, (uint32_t)g, (uint32_t)((uint64_t)g >> 32), (uint32_t)chain, tag);
}

// Order-preserving key of a float (NaN: largest).
__device__ __forceinline__ uint32_t float_key(float y)
{
    if (y != y) return 0xFFFFFFFEu;
    const uint32_t u = __float_as_uint(y);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// One warp: the moves of chain c to simulate exactly, chosen[0 .. top) (-1 for
// none), the same in every lane.  With the fallback (word 3 of the step draw r
// below eps) only candidate 0; otherwise the `top` distinct moves of lowest
// predicted y (b3 + the layer-2 partial sums), lowest candidate index on ties.
__device__ __forceinline__ void select_candidates(const ScreenArgs &a, int c, int lane,
                                                  const uint4 &r, int (&chosen)[kMaxTop])
{
    const bool fallback = (uint64_t)r.w < a.eps_thr;
    const int mv = lane < a.K ? a.cand[(size_t)c * a.K + lane] : -1;
    uint32_t key = 0xFFFFFFFFu;
    if (mv >= 0 && (!fallback || lane == 0)) {
        if (fallback) {
            key = 0;
        } else {
            float s = 0.f;
            const float *p = a.pc + ((size_t)c * a.K + lane) * a.nparts;
            for (int q = 0; q < a.nparts; ++q) s += p[q];
            key = float_key(*a.b3 + s);
        }
    }
    bool alive = key != 0xFFFFFFFFu;
#pragma unroll
    for (int s = 0; s < kMaxTop; ++s) {
        chosen[s] = -1;
        if (s >= a.top) continue;
        const uint32_t m = __reduce_min_sync(0xffffffffu, alive ? key : 0xFFFFFFFFu);
        if (m == 0xFFFFFFFFu) continue;
        const int w = __ffs(__ballot_sync(0xffffffffu, alive && key == m)) - 1;
        chosen[s] = __shfl_sync(0xffffffffu, mv, w);
        if (mv == chosen[s]) alive = false;   // the winner and its duplicates
    }
}

// One warp: the Metropolis test of Table 1 for chain c's chosen move `best`
// (exact score d) against the host threshold tables (word 2 of the step draw
// r), and on acceptance the commit: x_cur, delta_cur, the counters, the best
// vector (strict improvement) and the chain's layer-1 pre-activations A1.
__device__ __forceinline__ void screen_accept(const ScreenArgs &a, const DevSched &sc, int c,
                                              int lane, const uint4 &r, int best, int32_t d)
{
    int8_t *x = a.ch.x_cur + (size_t)c * a.ch.pstride;
    int64_t *cnt = a.ch.cnt + 3 * (size_t)c;
    const int32_t d_cur = a.ch.d_cur[c], d_best = a.ch.d_best[c];
    const int32_t dE = d - d_cur;
    bool accept = dE <= 0;
    if (!accept) {
        const int64_t l = a.g / sc.iters - sc.level0;
        if (dE <= sc.thr_len[l]) accept = r.z < sc.thr[sc.thr_off[l] + dE - 1];
    }
    if (!accept) return;
    const int j = best >> 8;
    const int v = (int8_t)(best & 255);
    const int rn = a.row_base[j] + v, ro = a.row_base[j] + x[j];
    __syncwarp();
    if (lane == 0) {
        x[j] = (int8_t)v;
        a.ch.d_cur[c] = d;
        cnt[0] += 1;
        cnt[1] += dE > 0;
    }
    __syncwarp();
    if (d < d_best) {
        warp_copy16(a.ch.x_best + (size_t)c * a.ch.pstride, x, a.ch.pstride, lane);
        if (lane == 0) a.ch.d_best[c] = d;
    }
    for (int h = lane; h < a.H1; h += 32)
        a.A1[(size_t)c * a.H1 + h] += __bfloat162float(a.W1b[(size_t)rn * a.H1 + h]) -
                                      __bfloat162float(a.W1b[(size_t)ro * a.H1 + h]);
}

// Finish of a screened step for single-condition networks whose layout has a
// four-chains-per-warp kernel (rn_chains4.cu) and top <= 2: two chains per
// warp, their chosen moves simulated together in the byte lanes.  Returns
// cudaErrorNotSupported (launching nothing) for any other network; d0, d1 are
// the network's register-table capacities.
cudaError_t launch_finish_chains4(const ScreenArgs &a, const DevSched &sc, int d0, int d1,
                                  cudaStream_t st);

// Finish of a screened step for block-path networks (a block of 256 threads
// per chain): the chosen moves simulated exactly, Metropolis, commit.
cudaError_t launch_finish_block(const ScreenArgs &a, const DevSched &sc, int sm_count,
                                cudaStream_t st);

}  // namespace rn
