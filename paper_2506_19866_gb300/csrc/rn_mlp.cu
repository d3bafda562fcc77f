// rn_mlp.cu -- the learned proposal screen: an MLP on the one-hot parameter
// vector, trained on the GPU by its own forward/backward kernels and Adam, and
// the screened annealing step that ranks K candidate moves per chain with it.
//
// Training batch of B rows (B a multiple of 128; D padded to Dp):
//   onehot     OH [B][Dp] and OH^T [Dp][B] (bf16 0/1) from int8 vectors
//   GEMM 1     h1 = relu(OH W1 + b1)                  bf16 [B][H1]
//   GEMM 2     h2 = relu(h1 W2 + b2), partials of w3 . h2 per 64 columns
//   head       y, dy = 2 (y - t) / n, dh2 = dy w3 [h2 > 0]
//   GEMMs      dW2 = h1^T dh2,  dh1 = (dh2 W2^T) [h1 > 0],  dW1 = OH^T dh1
//   colsums    db1, db2, dw3 = sum_b dy h2, db3 = sum_b dy
//   Adam       on the FP32 masters, then the BF16 copies are refreshed
// Screened step of C chains (M = C K candidate rows):
//   propose    K candidates per chain (GetCandidate of Table 1) and their
//              hidden rows relu(A1 + W1[new] - W1[old]) from the chain's
//              layer-1 pre-activation A1 (sparse FP32 update: one parameter
//              changes one row of the one-hot sum)
//   GEMM 2     partials of w3 . relu(h1 W2 + b2)
//   finish     top candidates by predicted y, each simulated exactly on the
//              chain's tables (Table 1's Simulate and score), Metropolis test
//              of Table 1 against the host threshold tables; x, delta, best,
//              counters and A1 follow an accepted move
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "rn_context.h"
#include "rn_gemm.cuh"
#include "rn_kernels.cuh"
#include "rn_screen.h"
#include "rn_umma.cuh"

namespace rn {
namespace {

using bf16 = __nv_bfloat16;

inline bf16 *bp(DevBuf<uint16_t> &b) { return reinterpret_cast<bf16 *>(b.p); }

// ---------------------------------------------------------------- kernels --

// Rows b < B: OH[b][row_base[j] + x_bj] = 1 and OHT[row][b] = 1 (buffers zeroed
// before).  Row b reads vector idx[b] of X (idx null: vector b); padding rows
// b >= n repeat the first vector.  A value whose row falls outside the
// parameter's block [row_off[j], row_off[j + 1]) is skipped.
__global__ void onehot_kernel(const int8_t *__restrict__ X, int64_t xstride,
                              const int32_t *__restrict__ idx, int32_t n, int32_t P,
                              const int32_t *__restrict__ row_base,
                              const int32_t *__restrict__ row_off, bf16 *OH, int32_t ldo,
                              bf16 *OHT, int32_t ldt)
{
    const int b = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P) return;
    const int r0 = b < n ? b : 0;
    const int64_t src = idx ? idx[r0] : r0;
    const int r = row_base[j] + X[src * xstride + j];
    if (r < row_off[j] || r >= row_off[j + 1]) return;
    const bf16 one = __float2bfloat16(1.0f);
    if (OH) OH[(size_t)b * ldo + r] = one;
    if (OHT) OHT[(size_t)r * ldt + b] = one;
}

// out[c][r] = in[r][c] (R x C, both multiples of 32), 32 x 8 threads per tile.
template <typename Tin>
__global__ void transpose_kernel(const Tin *__restrict__ in, int ldi, bf16 *__restrict__ out,
                                 int ldo)
{
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const Tin v = in[(size_t)(r0 + k) * ldi + c0 + threadIdx.x];
        if constexpr (sizeof(Tin) == 4) tile[k][threadIdx.x] = (float)v;
        else tile[k][threadIdx.x] = __bfloat162float(v);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8)
        out[(size_t)(c0 + k) * ldo + r0 + threadIdx.x] = __float2bfloat16(tile[threadIdx.x][k]);
}

__global__ void to_bf16_kernel(const float *__restrict__ in, bf16 *__restrict__ out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16(in[i]);
}

// Warp per row b < B: y_b = b3 + sum of the layer-2 partials.  With targets:
// dy_b = 2 (y_b - t_b) / n for b < n (0 for padding rows), the squared errors
// summed into *sse, and dh2[b][k] = dy_b w3[k] [h2[b][k] > 0].
__global__ void head_kernel(const float *__restrict__ part, int nparts, const float *__restrict__ b3,
                            int32_t B, int32_t n, float *__restrict__ y,
                            const float *__restrict__ tgt, float *__restrict__ dy,
                            double *__restrict__ sse, const bf16 *__restrict__ h2,
                            const float *__restrict__ w3, bf16 *__restrict__ dh2, int H2)
{
    const int lane = threadIdx.x & 31;
    const int b = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (b >= B) return;
    float s = lane < nparts ? part[(size_t)b * nparts + lane] : 0.f;
#pragma unroll
    for (int k = 16; k; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    const float yb = *b3 + s;
    if (lane == 0 && y) y[b] = yb;
    if (!tgt) return;
    const float e = b < n ? yb - tgt[b] : 0.f;
    const float d = 2.f * e / (float)n;
    if (lane == 0) {
        dy[b] = d;
        if (b < n) atomicAdd(sse, (double)e * (double)e);
    }
    for (int k = lane * 8; k < H2; k += 256) {
        const uint4 hv = *reinterpret_cast<const uint4 *>(h2 + (size_t)b * H2 + k);
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&hv);
        uint4 ov;
        __nv_bfloat162 *o = reinterpret_cast<__nv_bfloat162 *>(&ov);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 f = __bfloat1622float2(h[q]);
            o[q] = __floats2bfloat162_rn(f.x > 0.f ? d * w3[k + 2 * q] : 0.f,
                                         f.y > 0.f ? d * w3[k + 2 * q + 1] : 0.f);
        }
        *reinterpret_cast<uint4 *>(dh2 + (size_t)b * H2 + k) = ov;
    }
}

// part[s][c] = sum over the rows of split s of coef[r] A[r][c] (coef null: 1);
// 32 x 8 threads, 64 columns per block, blockIdx.y = split.
__global__ void colsum_kernel(const bf16 *__restrict__ A, int lda, int R,
                              const float *__restrict__ coef, int rows_per_split,
                              float *__restrict__ part, int C)
{
    __shared__ float red[8][64];
    const int c = blockIdx.x * 64 + threadIdx.x * 2;
    const int r0 = blockIdx.y * rows_per_split, r1 = min(R, r0 + rows_per_split);
    float s0 = 0.f, s1 = 0.f;
    for (int r = r0 + threadIdx.y; r < r1; r += 8) {
        const float2 v =
            __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(A + (size_t)r * lda + c));
        const float w = coef ? coef[r] : 1.f;
        s0 += w * v.x;
        s1 += w * v.y;
    }
    red[threadIdx.y][threadIdx.x * 2] = s0;
    red[threadIdx.y][threadIdx.x * 2 + 1] = s1;
    __syncthreads();
    if (threadIdx.y == 0) {
        float t0 = 0.f, t1 = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            t0 += red[k][threadIdx.x * 2];
            t1 += red[k][threadIdx.x * 2 + 1];
        }
        part[(size_t)blockIdx.y * C + c] = t0;
        part[(size_t)blockIdx.y * C + c + 1] = t1;
    }
}

// out[c] = sum_s part[s][c]; with v != null also out[C] = sum_{r < nv} v[r]
// (one extra thread block).
__global__ void colsum_finish_kernel(const float *__restrict__ part, int S, int C,
                                     float *__restrict__ out, const float *__restrict__ v, int nv)
{
    if (blockIdx.x == gridDim.x - 1 && v) {
        __shared__ float red[256];
        float s = 0.f;
        for (int r = threadIdx.x; r < nv; r += blockDim.x) s += v[r];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w; w >>= 1) {
            if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[C] = red[0];
        return;
    }
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    for (int k = 0; k < S; ++k) s += part[(size_t)k * C + c];
    out[c] = s;
}

// Adam (Kingma & Ba, 2015) on the FP32 masters; the bias corrections of step k
// of the call (k = *kstep) are cc[2k] = 1 / (1 - beta1^t), cc[2k + 1] =
// 1 / (1 - beta2^t), computed on the host in double.
__global__ void adam_kernel(float *__restrict__ theta, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, size_t n, float lr,
                            float beta1, float beta2, const float *__restrict__ cc,
                            const uint32_t *__restrict__ kstep, float eps)
{
    const uint32_t k = *kstep;
    const float c1 = cc[2 * (size_t)k], c2 = cc[2 * (size_t)k + 1];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = beta1 * m[i] + (1.f - beta1) * gi;
        const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// Minibatch rows: slot idx[b] of the training set, drawn uniformly from the
// `count` held pairs by Philox counter (step, 0, b, 8), step = *kstep (the
// step within the call); tgt[b] its target.
__global__ void sample_kernel(uint64_t seed, const uint32_t *__restrict__ kstep, int32_t B,
                              uint32_t count, const float *__restrict__ set_y,
                              int32_t *__restrict__ idx, float *__restrict__ tgt, float mu,
                              float inv_sigma)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const uint4 r = philox(seed, *kstep, 0u, (uint32_t)b, 8u);
    const uint32_t k = pick(r.x, count);
    idx[b] = (int32_t)k;
    tgt[b] = (set_y[k] - mu) * inv_sigma;
}

// The step counter of a training call, advanced once per step.
__global__ void advance_step_kernel(uint32_t *kstep) { *kstep += 1u; }

// Output layer w3 <- a w3, b3 <- a b3 + c (one block).
__global__ void affine_head_kernel(float *__restrict__ w3, int H2, float *__restrict__ b3,
                                   float a, float c)
{
    for (int k = threadIdx.x; k < H2; k += blockDim.x) w3[k] *= a;
    if (threadIdx.x == 0) *b3 = *b3 * a + c;
}

// Warp per chain: its x_cur row and delta_cur * scale into ring slot
// (head + chain) % cap.
__global__ void log_chains_kernel(DevChains ch, int8_t *__restrict__ set_x,
                                  float *__restrict__ set_y, int64_t head, int64_t cap,
                                  float scale)
{
    const int lane = threadIdx.x & 31;
    const int c = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (c >= ch.n) return;
    const int64_t slot = (head + c) % cap;
    warp_copy16(set_x + slot * ch.pstride, ch.x_cur + (size_t)c * ch.pstride, ch.pstride, lane);
    if (lane == 0) set_y[slot] = (float)ch.d_cur[c] * scale;
}

// Block per chain: A1[c][h] = b1[h] + sum_j W1[row(j, x_j)][h] (the BF16
// weights), h over the block's threads.
// A1 rows c0 .. c0 + n - 1 from the one-hot GEMM's rows: + b1.
__global__ void embed_bias_kernel(const float *__restrict__ prod, int32_t n, int32_t H1,
                                  const float *__restrict__ b1, float *__restrict__ A1)
{
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)n * H1) return;
    A1[k] = prod[k] + b1[k % H1];
}

__global__ void embed_chains_kernel(DevChains ch, int32_t P, const int32_t *__restrict__ row_base,
                                    const bf16 *__restrict__ W1b, const float *__restrict__ b1,
                                    int H1, float *__restrict__ A1)
{
    const int c = blockIdx.x;
    const int8_t *x = ch.x_cur + (size_t)c * ch.pstride;
    for (int h = threadIdx.x; h < H1; h += blockDim.x) {
        float a = b1[h];
        for (int j = 0; j < P; ++j)
            a += __bfloat162float(W1b[(size_t)(row_base[j] + x[j]) * H1 + h]);
        A1[(size_t)c * H1 + h] = a;
    }
}

// Warp per chain: K candidates (lane k draws candidate k), then either (ROWS)
// each candidate's two W1 rows (new value, old value; -1 without a candidate)
// for the GEMM that forms the hidden rows itself, or the K hidden rows
// relu(A1 + W1[new] - W1[old]) in BF16.  Shared memory per warp: x_cur,
// out_nz[N], pos_in[N].
template <bool ROWS>
__global__ void __launch_bounds__(kScreenWarps * 32) screen_propose_kernel(ScreenArgs a,
                                                                           int region)
{
    extern __shared__ __align__(256) uint8_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * (blockDim.x >> 5) + warp;
    if (c >= a.ch.n) return;
    int8_t *xs = reinterpret_cast<int8_t *>(sm + warp * region);
    uint8_t *out_nz = reinterpret_cast<uint8_t *>(xs) + a.ch.pstride;
    uint8_t *pos_in = out_nz + ((a.net.N + 15) & ~15);
    warp_copy16(xs, a.ch.x_cur + (size_t)c * a.ch.pstride, a.ch.pstride, lane);
    __syncwarp();
    count_constraints(a.net, xs, out_nz, pos_in, lane);
    __syncwarp();
    int j = 0, kind, idx, cur = 0, v = 0;
    bool ok = false;
    if (lane < a.K && a.net.n_free > 0) {
        const uint4 r = step_draw(a.ch, a.g, c, lane == 0 ? 0u : 16u + (uint32_t)lane);
        ok = get_candidate<true>(a.net, xs, out_nz, pos_in, r.x, r.y, j, kind, idx, cur, v);
    }
    if (lane < a.K) a.cand[(size_t)c * a.K + lane] = ok ? (j << 8) | (v & 255) : -1;
    // lane k: the W1 rows of candidate k's new and old value (-1: no candidate)
    const int rn_l = ok ? a.row_base[j] + v : -1;
    const int ro_l = ok ? a.row_base[j] + cur : -1;
    if constexpr (ROWS) {
        if (lane < a.K) a.rows[(size_t)c * a.K + lane] = make_int2(rn_l, ro_l);
        return;
    }

    const int groups = a.H1 >> 8;
    float base[kMaxGroups][8];
#pragma unroll
    for (int q = 0; q < kMaxGroups; ++q) {
        if (q >= groups) break;
        const float4 *p = reinterpret_cast<const float4 *>(a.A1 + (size_t)c * a.H1 + q * 256 + lane * 8);
        const float4 u0 = p[0], u1 = p[1];
        base[q][0] = u0.x; base[q][1] = u0.y; base[q][2] = u0.z; base[q][3] = u0.w;
        base[q][4] = u1.x; base[q][5] = u1.y; base[q][6] = u1.z; base[q][7] = u1.w;
    }
    // four candidates per pass, their eight W1 row loads issued before any use
    constexpr int U = 4;
    for (int k0 = 0; k0 < a.K; k0 += U) {
#pragma unroll
        for (int q = 0; q < kMaxGroups; ++q) {
            if (q >= groups) break;
            const int col = q * 256 + lane * 8;
            uint4 wn[U], wo[U];
            int rn[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = min(k0 + u, a.K - 1);
                rn[u] = __shfl_sync(0xffffffffu, rn_l, k);
                const int ro = __shfl_sync(0xffffffffu, ro_l, k);
                wn[u] = wo[u] = make_uint4(0u, 0u, 0u, 0u);
                if (rn[u] >= 0) {
                    wn[u] = *reinterpret_cast<const uint4 *>(a.W1b + (size_t)rn[u] * a.H1 + col);
                    wo[u] = *reinterpret_cast<const uint4 *>(a.W1b + (size_t)ro * a.H1 + col);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (k0 + u >= a.K) break;
                float h[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) h[e] = base[q][e];
                if (rn[u] >= 0) {
                    const __nv_bfloat162 *pn = reinterpret_cast<const __nv_bfloat162 *>(&wn[u]);
                    const __nv_bfloat162 *po = reinterpret_cast<const __nv_bfloat162 *>(&wo[u]);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float2 fn = __bfloat1622float2(pn[e]), fo = __bfloat1622float2(po[e]);
                        h[2 * e] += fn.x - fo.x;
                        h[2 * e + 1] += fn.y - fo.y;
                    }
                }
                uint4 ov;
                __nv_bfloat162 *o = reinterpret_cast<__nv_bfloat162 *>(&ov);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    o[e] = __floats2bfloat162_rn(fmaxf(h[2 * e], 0.f), fmaxf(h[2 * e + 1], 0.f));
                bf16 *out = a.hc + ((size_t)c * a.K + k0 + u) * a.H1;
                *reinterpret_cast<uint4 *>(out + col) = ov;
            }
        }
    }
}

// Warp per chain, after the layer-2 GEMM: the candidates to simulate
// (fallback: candidate 0 only; otherwise the `top` distinct moves of lowest
// predicted y, lowest candidate index on ties), each simulated exactly on the
// chain's tables (change, Simulate, undo: Table 1's Simulate of x with one
// parameter changed), the one of lowest exact score (first on ties) to the
// Metropolis test of Table 1 against the host threshold tables (word 2 of the
// step draw).  An accepted move updates x_cur, delta_cur, the best vector
// (strict improvement), the counters and A1.  A step without a candidate is a
// null move.
template <class Path>
__device__ __forceinline__ void screen_finish(const ScreenArgs &a, const DevSched &sc, Path &P,
                                              int c, int lane)
{
    const DevNet &net = a.net;
    const uint4 r = step_draw(a.ch, a.g, c, 0u);
    int chosen[kMaxTop];
    select_candidates(a, c, lane, r, chosen);
    int64_t *cnt = a.ch.cnt + 3 * (size_t)c;
    if (chosen[0] < 0) {
        if (lane == 0) cnt[2] += 1;
        return;
    }
    int8_t *x = a.ch.x_cur + (size_t)c * a.ch.pstride;
    P.load(net, x, lane);
    __syncwarp();
    const int E = net.E, N = net.N;
    int best = -1;
    int32_t d = 0;
#pragma unroll
    for (int s = 0; s < kMaxTop; ++s) {
        const int move = chosen[s];
        if (move < 0) continue;
        const int j = move >> 8, v = (int8_t)(move & 255);
        int kind, idx, owner;
        param_kind(j, E, N, kind, idx);
        if (kind < 3) {
            const int pos = net.edge_pos[idx];
            owner = pos >> 16;
            int w = x[idx], p = x[E + idx], t = x[2 * E + idx];
            if (kind == 0) w = v; else if (kind == 1) p = v; else t = v;
            P.change_edge(net, lane, owner, pos, w, p, t, idx);
        } else {
            const int q = net.node_q[idx];
            owner = q / net.npl;
            P.change_node(lane, owner, q - owner * net.npl, kind, v);
        }
        __syncwarp();
        const int32_t ds = P.simulate(net, lane, nullptr);
        P.undo(lane, owner);
        __syncwarp();
        if (best < 0 || ds < d) { best = move; d = ds; }
    }
    screen_accept(a, sc, c, lane, r, best, d);
}

// Register-table path (N <= 128), as evaluate_kernel: in-degree capacity 16.
template <int NPL, int CG>
__global__ void __launch_bounds__(kScreenWarps * 32) screen_finish_reg_kernel(ScreenArgs a,
                                                                              DevSched sc)
{
    extern __shared__ __align__(256) uint8_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * kScreenWarps + warp;
    if (c >= a.ch.n) return;
    RegPath<NPL, CG, 16, 16> P;
    P.sm = sm;
    P.codes = (uint32_t)warp * kCodeBytesPerWarp;
    screen_finish(a, sc, P, c, lane);
}

// Shared-memory-table path (129 .. 512 nodes).
__global__ void __launch_bounds__(kScreenWarps * 32)
    screen_finish_smem_kernel(ScreenArgs a, DevSched sc, uint32_t region_bytes, uint32_t lut_words)
{
    extern __shared__ __align__(256) uint8_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * kScreenWarps + warp;
    if (c >= a.ch.n) return;
    SmemPath P = make_smem_path(a.net, sm, warp, kScreenWarps, region_bytes, lut_words);
    screen_finish(a, sc, P, c, lane);
}

cudaError_t launch_finish(const ScreenArgs &a, const DevSched &sc, cudaStream_t st)
{
    const int blocks = (a.ch.n + kScreenWarps - 1) / kScreenWarps;
    if (a.net.npl > kRegSlots) {
        const WarpRegion R = warp_region(true, a.net.D, a.net.npl, 0, 0);
        const size_t smem = kScreenWarps * ((size_t)kCodeBytesPerWarp + R.bytes);
        const cudaError_t e = cudaFuncSetAttribute(
            screen_finish_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        screen_finish_smem_kernel<<<blocks, kScreenWarps * 32, smem, st>>>(a, sc, R.bytes,
                                                                           R.lut_words);
        return cudaGetLastError();
    }
    const size_t smem = kScreenWarps * (size_t)kCodeBytesPerWarp;
#define RN_FIN(NPL_, CG_)                                                                      \
    if (a.net.npl == NPL_ && a.net.cg == CG_) {                                                \
        screen_finish_reg_kernel<NPL_, CG_><<<blocks, kScreenWarps * 32, smem, st>>>(a, sc);  \
        return cudaGetLastError();                                                             \
    }
    RN_FIN(1, 1) RN_FIN(1, 4) RN_FIN(2, 1) RN_FIN(2, 4) RN_FIN(4, 1) RN_FIN(4, 4)
#undef RN_FIN
    return cudaErrorNotSupported;
}

// ------------------------------------------------------------------ host --

Mlp *get_mlp(rn_ctx *ctx, int32_t id)
{
    if (!ctx || id < 0 || id >= (int32_t)ctx->mlps.size()) return nullptr;
    return ctx->mlps[(size_t)id].get();
}

int lookup(rn_ctx *ctx, int32_t id, Mlp *&m, Network *&n)
{
    m = get_mlp(ctx, id);
    if (!m) return fail(ctx, RN_EINVAL, "unknown screen %d", id);
    n = get_net(ctx, m->net);
    if (!n) return fail(ctx, RN_EINVAL, "the screen's network is gone");
    return RN_OK;
}

int check_launch(rn_ctx *ctx, const char *what, int kernels = 1)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    ctx->launches += kernels;
    return RN_OK;
}

// tcgen05 tensor-core GEMM where the shape allows (every shape of the screen:
// widths are multiples of 256, Dp of 128, batches of 128), else mma.sync.
int gemm(rn_ctx *ctx, int epi, const GemmArgs &g)
{
    const cudaError_t e = gemm_tc_supported(g)
                              ? launch_gemm_tc(epi, g, ctx->dev_err.p, ctx->sm_count, ctx->stream)
                              : launch_gemm(epi, g, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "BF16 GEMM");
    ctx->launches += 1;
    return RN_OK;
}

// Scratch of a batch of up to B rows (multiple of 128).
int ensure_batch(rn_ctx *ctx, Mlp &m, int32_t B)
{
    if (B <= m.Bcap) return RN_OK;
    const size_t Dp = (size_t)m.Dp, H1 = (size_t)m.H1, H2 = (size_t)m.H2, b = (size_t)B;
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    RN_CUDA(ctx, m.oh.alloc(b * Dp));
    RN_CUDA(ctx, m.ohT.alloc(Dp * b));
    RN_CUDA(ctx, m.h1.alloc(b * H1));
    RN_CUDA(ctx, m.h1T.alloc(H1 * b));
    RN_CUDA(ctx, m.h2.alloc(b * H2));
    RN_CUDA(ctx, m.dh2.alloc(b * H2));
    RN_CUDA(ctx, m.dh2T.alloc(H2 * b));
    RN_CUDA(ctx, m.dh1.alloc(b * H1));
    RN_CUDA(ctx, m.dh1T.alloc(H1 * b));
    RN_CUDA(ctx, m.part.alloc(b * (H2 / 64)));
    RN_CUDA(ctx, m.y.alloc(b));
    RN_CUDA(ctx, m.dy.alloc(b));
    RN_CUDA(ctx, m.tgt.alloc(b));
    RN_CUDA(ctx, m.idx.alloc(b));
    RN_CUDA(ctx, m.xrows.alloc(b * (size_t)m.pstride));
    RN_CUDA(ctx, m.colpart.alloc(64 * std::max(H1, H2)));
    m.Bcap = B;
    return RN_OK;
}

// BF16 copies of W1 and W2 from the FP32 masters.
int refresh_copies(rn_ctx *ctx, Mlp &m)
{
    const float *W1 = m.theta.p, *W2 = m.theta.p + m.off_W2();
    const dim3 t(32, 8);
    transpose_kernel<float><<<dim3(m.H1 / 32, m.Dp / 32), t, 0, ctx->stream>>>(W1, m.H1, bp(m.W1T), m.Dp);
    transpose_kernel<float><<<dim3(m.H2 / 32, m.H1 / 32), t, 0, ctx->stream>>>(W2, m.H2, bp(m.W2T), m.H1);
    to_bf16_kernel<<<512, 256, 0, ctx->stream>>>(W1, bp(m.W1b), (size_t)m.Dp * m.H1);
    to_bf16_kernel<<<256, 256, 0, ctx->stream>>>(W2, bp(m.W2b), (size_t)m.H1 * m.H2);
    m.a1_valid = false;
    return check_launch(ctx, "weight copies", 4);
}

// Column sums of a bf16 [R][C] matrix (coef-weighted) into out[C] (and, with
// v, out[C] = sum of v[0..nv)).
int colsum(rn_ctx *ctx, Mlp &m, const bf16 *A, int R, int C, const float *coef, float *out,
           const float *v = nullptr, int nv = 0)
{
    const int S = 64, rows = (R + S - 1) / S;
    colsum_kernel<<<dim3(C / 64, S), dim3(32, 8), 0, ctx->stream>>>(A, C, R, coef, rows,
                                                                     m.colpart.p, C);
    const int blocks = (C + 255) / 256 + (v ? 1 : 0);
    colsum_finish_kernel<<<blocks, 256, 0, ctx->stream>>>(m.colpart.p, S, C, out, v, nv);
    return check_launch(ctx, "column sums", 2);
}

// One batch of B rows (n real): forward, and with targets the loss and every
// gradient into m.grad.  Rows come from X (stride xstride) through idx (or in
// order).
int run_batch(rn_ctx *ctx, Mlp &m, const int8_t *X, int64_t xstride, const int32_t *idx,
              int32_t n, int32_t B, const float *tgt)
{
    const bool train = tgt != nullptr;
    const int Dp = m.Dp, H1 = m.H1, H2 = m.H2, P = m.P;
    cudaStream_t st = ctx->stream;
    RN_CUDA(ctx, cudaMemsetAsync(m.oh.p, 0, sizeof(uint16_t) * (size_t)B * Dp, st));
    if (train) RN_CUDA(ctx, cudaMemsetAsync(m.ohT.p, 0, sizeof(uint16_t) * (size_t)B * Dp, st));
    onehot_kernel<<<dim3((P + 255) / 256, B), 256, 0, st>>>(
        X, xstride, idx, n, P, m.row_base.p, m.row_base.p + P, bp(m.oh), Dp,
        train ? bp(m.ohT) : nullptr, B);
    int rc = check_launch(ctx, "one-hot kernel");
    if (rc) return rc;
    const float *th = m.theta.p;
    GemmArgs g{};
    // h1 = relu(OH W1 + b1)
    g.A = bp(m.oh); g.lda = Dp; g.B = bp(m.W1T); g.ldb = Dp;
    g.M = B; g.N = H1; g.K = Dp; g.out_bf16 = bp(m.h1); g.ldc = H1; g.bias = th + m.off_b1();
    if ((rc = gemm(ctx, kBiasReluBf16, g))) return rc;
    // h2 = relu(h1 W2 + b2); partials of w3 . h2
    g = GemmArgs{};
    g.A = bp(m.h1); g.lda = H1; g.B = bp(m.W2T); g.ldb = H1;
    g.M = B; g.N = H2; g.K = H1; g.out_bf16 = train ? bp(m.h2) : nullptr; g.ldc = H2;
    g.bias = th + m.off_b2(); g.w = th + m.off_w3(); g.part = m.part.p;
    if ((rc = gemm(ctx, kBiasReluDot, g))) return rc;
    if (train) RN_CUDA(ctx, cudaMemsetAsync(m.loss.p, 0, sizeof(double), st));
    head_kernel<<<(B + 7) / 8, 256, 0, st>>>(m.part.p, H2 / 64, th + m.off_b3(), B, n, m.y.p,
                                             tgt, m.dy.p, m.loss.p, bp(m.h2),
                                             th + m.off_w3(), bp(m.dh2), H2);
    if ((rc = check_launch(ctx, "head kernel"))) return rc;
    if (!train) return RN_OK;
    float *gr = m.grad.p;
    const dim3 t(32, 8);
    // dW2 = h1^T dh2
    transpose_kernel<bf16><<<dim3(H1 / 32, B / 32), t, 0, st>>>(bp(m.h1), H1, bp(m.h1T), B);
    transpose_kernel<bf16><<<dim3(H2 / 32, B / 32), t, 0, st>>>(bp(m.dh2), H2, bp(m.dh2T), B);
    if ((rc = check_launch(ctx, "transposes", 2))) return rc;
    g = GemmArgs{};
    g.A = bp(m.h1T); g.lda = B; g.B = bp(m.dh2T); g.ldb = B;
    g.M = H1; g.N = H2; g.K = B; g.out_f32 = gr + m.off_W2(); g.ldc = H2;
    if ((rc = gemm(ctx, kStoreF32, g))) return rc;
    // dh1 = (dh2 W2^T) [h1 > 0]
    g = GemmArgs{};
    g.A = bp(m.dh2); g.lda = H2; g.B = bp(m.W2b); g.ldb = H2;
    g.M = B; g.N = H1; g.K = H2; g.out_bf16 = bp(m.dh1); g.ldc = H1; g.mask = bp(m.h1);
    if ((rc = gemm(ctx, kMaskBf16, g))) return rc;
    // dW1 = OH^T dh1
    transpose_kernel<bf16><<<dim3(H1 / 32, B / 32), t, 0, st>>>(bp(m.dh1), H1, bp(m.dh1T), B);
    if ((rc = check_launch(ctx, "transpose"))) return rc;
    g = GemmArgs{};
    g.A = bp(m.ohT); g.lda = B; g.B = bp(m.dh1T); g.ldb = B;
    g.M = Dp; g.N = H1; g.K = B; g.out_f32 = gr; g.ldc = H1;
    if ((rc = gemm(ctx, kStoreF32, g))) return rc;
    // bias and output-layer gradients
    if ((rc = colsum(ctx, m, bp(m.dh1), B, H1, nullptr, gr + m.off_b1()))) return rc;
    if ((rc = colsum(ctx, m, bp(m.dh2), B, H2, nullptr, gr + m.off_b2()))) return rc;
    // dw3 = sum_b dy_b h2[b] and, in the slot after it, db3 = sum_b dy_b
    return colsum(ctx, m, bp(m.h2), B, H2, m.dy.p, gr + m.off_w3(), m.dy.p, B);
}

int32_t round_up(int32_t v, int32_t k) { return (v + k - 1) / k * k; }

// Every value inside its parameter's domain (the one-hot encoding needs no more).
int check_domains(rn_ctx *ctx, const Network &n, const int8_t *x, int64_t which)
{
    for (int32_t j = 0; j < n.P; ++j) {
        int8_t vals[6];
        const int k = domain_of(n, j, vals);
        bool in = false;
        for (int a = 0; a < k; ++a) in |= vals[a] == x[j];
        if (!in)
            return fail(ctx, RN_EINVAL, "vector %lld: parameter %d = %d is outside its domain",
                        (long long)which, j, (int)x[j]);
    }
    return RN_OK;
}

// Host vectors [n][P] into the staging rows (values checked against their domains).
int stage_rows(rn_ctx *ctx, Mlp &m, const Network &net, const int8_t *x, int32_t n)
{
    std::vector<int8_t> rows((size_t)n * m.pstride, 0);
    for (int32_t r = 0; r < n; ++r) {
        const int8_t *xr = x + (size_t)r * m.P;
        if (int rc = check_domains(ctx, net, xr, r)) return rc;
        std::memcpy(&rows[(size_t)r * m.pstride], xr, (size_t)m.P);
    }
    RN_CUDA(ctx, cudaMemcpyAsync(m.xrows.p, rows.data(), rows.size(), cudaMemcpyHostToDevice,
                                 ctx->stream));
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return RN_OK;
}

int weights_io(rn_ctx *ctx, Mlp &m, bool set, float *W1, float *b1, float *W2, float *b2,
               float *w3, float *b3)
{
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<float> th(m.n_theta, 0.f);
    if (!set)
        RN_CUDA(ctx, cudaMemcpy(th.data(), m.theta.p, th.size() * sizeof(float),
                                cudaMemcpyDeviceToHost));
    const size_t D = (size_t)m.D, H1 = (size_t)m.H1, H2 = (size_t)m.H2;
    struct Part { float *p; size_t off, n; } parts[] = {
        {W1, 0, D * H1}, {b1, m.off_b1(), H1}, {W2, m.off_W2(), H1 * H2},
        {b2, m.off_b2(), H2}, {w3, m.off_w3(), H2}, {b3, m.off_b3(), 1}};
    for (auto &p : parts) {
        if (!p.p) continue;
        if (set) std::memcpy(&th[p.off], p.p, p.n * sizeof(float));
        else std::memcpy(p.p, &th[p.off], p.n * sizeof(float));
    }
    if (!set) return RN_OK;
    RN_CUDA(ctx, cudaMemcpy(m.theta.p, th.data(), th.size() * sizeof(float),
                            cudaMemcpyHostToDevice));
    RN_CUDA(ctx, cudaMemset(m.adam_m.p, 0, m.n_theta * sizeof(float)));
    RN_CUDA(ctx, cudaMemset(m.adam_v.p, 0, m.n_theta * sizeof(float)));
    m.adam_t = 0;
    return refresh_copies(ctx, m);
}

// Candidate buffers of the screened step for the network's chains.
// A1 of every chain (the layer-1 pre-activation b1 + sum_j W1[onehot(x)_j]).
// Small parameter vectors: a block per chain sums its P rows of W1 in order.
// Large ones (the block path's thousands of parameters): one-hot rows of
// kEmbedRows chains at a time times W1 on the tensor cores (FP32 accumulation,
// so the rounding order differs from the per-chain sum).
constexpr int kEmbedRows = 1024;

int embed_chains(rn_ctx *ctx, Mlp &m, const DevChains &ch)
{
    cudaStream_t st = ctx->stream;
    if ((int64_t)m.P * m.H1 <= ((int64_t)1 << 22)) {
        embed_chains_kernel<<<ch.n, 256, 0, st>>>(ch, m.P, m.row_base.p, bp(m.W1b),
                                                  m.theta.p + m.off_b1(), m.H1, m.A1.p);
        return check_launch(ctx, "embed kernel");
    }
    const size_t Dp = (size_t)m.Dp, H1 = (size_t)m.H1;
    RN_CUDA(ctx, m.emb_oh.reserve(kEmbedRows * Dp));
    RN_CUDA(ctx, m.emb_out.reserve(kEmbedRows * H1));
    for (int32_t c0 = 0; c0 < ch.n; c0 += kEmbedRows) {
        const int32_t n = std::min(kEmbedRows, ch.n - c0);
        RN_CUDA(ctx, cudaMemsetAsync(m.emb_oh.p, 0, sizeof(uint16_t) * kEmbedRows * Dp, st));
        onehot_kernel<<<dim3((m.P + 255) / 256, kEmbedRows), 256, 0, st>>>(
            ch.x_cur + (size_t)c0 * ch.pstride, ch.pstride, nullptr, n, m.P, m.row_base.p,
            m.row_base.p + m.P, bp(m.emb_oh), m.Dp, nullptr, 0);
        if (int rc = check_launch(ctx, "one-hot kernel")) return rc;
        GemmArgs g{};
        g.A = bp(m.emb_oh); g.lda = m.Dp; g.B = bp(m.W1T); g.ldb = m.Dp;
        g.M = kEmbedRows; g.N = m.H1; g.K = m.Dp; g.out_f32 = m.emb_out.p; g.ldc = m.H1;
        if (int rc = gemm(ctx, kStoreF32, g)) return rc;
        const size_t cnt = (size_t)n * H1;
        embed_bias_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(
            m.emb_out.p, n, m.H1, m.theta.p + m.off_b1(), m.A1.p + (size_t)c0 * H1);
        if (int rc = check_launch(ctx, "embed bias kernel")) return rc;
    }
    return RN_OK;
}

int ensure_screen(rn_ctx *ctx, Mlp &m, const Network &n, int32_t K, int32_t top)
{
    if (m.chains == n.n_chains && m.K == K && m.top == top) return RN_OK;
    const size_t C = (size_t)n.n_chains;
    const size_t M = (size_t)round_up((int32_t)(C * K), 128);
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    RN_CUDA(ctx, m.A1.alloc(C * m.H1));
    RN_CUDA(ctx, m.rows.alloc(M));
    RN_CUDA(ctx, m.pc.alloc(M * (m.H2 / 64)));
    RN_CUDA(ctx, m.cand.alloc(C * K));
    m.chains = n.n_chains;
    m.K = K;
    m.top = top;
    m.a1_valid = false;
    return RN_OK;
}

}  // namespace
}  // namespace rn

using namespace rn;

extern "C" {

int rn_mlp_create(rn_ctx *ctx, int32_t net, int32_t h1, int32_t h2, int64_t capacity,
                  int32_t *mlp_id, int32_t *onehot_width)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Network *n = get_net(ctx, net);
    if (!n) return fail(ctx, RN_EINVAL, "unknown network %d", net);
    if (!mlp_id) return fail(ctx, RN_EINVAL, "mlp_id is NULL");
    if (h1 < 256 || h1 > 1024 || h1 % 256 || h2 < 256 || h2 > 1024 || h2 % 256)
        return fail(ctx, RN_EINVAL, "hidden widths must be 256, 512, 768 or 1024");
    if (capacity < 1 || capacity > ((int64_t)1 << 31) - 1)
        return fail(ctx, RN_EINVAL, "capacity must be in 1 .. 2^31 - 1");
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    auto m = std::make_unique<Mlp>();
    m->net = net;
    m->P = n->P;
    m->pstride = (n->P + 15) & ~15;
    m->H1 = h1;
    m->H2 = h2;
    // one-hot blocks: parameter j's value v sits at row_base[j] + v, inside
    // [row_off[j], row_off[j + 1])
    std::vector<int32_t> tab(2 * (size_t)n->P + 1);
    int32_t D = 0;
    for (int32_t j = 0; j < n->P; ++j) {
        int8_t vals[6];
        const int k = domain_of(*n, j, vals);
        tab[(size_t)j] = D - vals[0];
        tab[(size_t)n->P + j] = D;
        D += k;
    }
    tab[2 * (size_t)n->P] = D;
    m->D = D;
    m->Dp = round_up(D, 128);
    m->scale = n->n_obs > 0 ? 1.0 / (double)n->n_obs : 1.0;
    RN_CUDA(ctx, m->row_base.upload(tab));
    m->n_theta = m->off_b3() + 1;
    RN_CUDA(ctx, m->theta.alloc(m->n_theta));
    RN_CUDA(ctx, m->grad.alloc(m->n_theta));
    RN_CUDA(ctx, m->adam_m.alloc(m->n_theta));
    RN_CUDA(ctx, m->adam_v.alloc(m->n_theta));
    for (DevBuf<float> *b : {&m->theta, &m->grad, &m->adam_m, &m->adam_v})
        RN_CUDA(ctx, cudaMemset(b->p, 0, m->n_theta * sizeof(float)));
    RN_CUDA(ctx, m->W1T.alloc((size_t)m->Dp * h1));
    RN_CUDA(ctx, m->W1b.alloc((size_t)m->Dp * h1));
    RN_CUDA(ctx, m->W2T.alloc((size_t)h1 * h2));
    RN_CUDA(ctx, m->W2b.alloc((size_t)h1 * h2));
    RN_CUDA(ctx, m->loss.alloc(1));
    m->cap = capacity;
    RN_CUDA(ctx, m->set_x.alloc((size_t)capacity * m->pstride));
    RN_CUDA(ctx, m->set_y.alloc((size_t)capacity));
    if (int rc = refresh_copies(ctx, *m)) return rc;
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->mlps.push_back(std::move(m));
    *mlp_id = (int32_t)ctx->mlps.size() - 1;
    if (onehot_width) *onehot_width = D;
    return RN_OK;
}

int rn_mlp_set_weights(rn_ctx *ctx, int32_t mlp, const float *W1, const float *b1,
                       const float *W2, const float *b2, const float *w3, float b3)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Mlp *m;
    Network *n;
    if (int rc = lookup(ctx, mlp, m, n)) return rc;
    if (!W1 || !b1 || !W2 || !b2 || !w3) return fail(ctx, RN_EINVAL, "weight array is NULL");
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    float b3v = b3;
    return weights_io(ctx, *m, true, const_cast<float *>(W1), const_cast<float *>(b1),
                      const_cast<float *>(W2), const_cast<float *>(b2), const_cast<float *>(w3),
                      &b3v);
}

int rn_mlp_get_weights(rn_ctx *ctx, int32_t mlp, float *W1, float *b1, float *W2, float *b2,
                       float *w3, float *b3)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Mlp *m;
    Network *n;
    if (int rc = lookup(ctx, mlp, m, n)) return rc;
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    return weights_io(ctx, *m, false, W1, b1, W2, b2, w3, b3);
}

int rn_mlp_forward(rn_ctx *ctx, int32_t mlp, int32_t n_vec, const int8_t *x, float *y)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Mlp *m;
    Network *n;
    if (int rc = lookup(ctx, mlp, m, n)) return rc;
    if (n_vec < 0 || (n_vec > 0 && (!x || !y))) return fail(ctx, RN_EINVAL, "bad vectors");
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    const int32_t chunk = 8192;
    for (int32_t r0 = 0; r0 < n_vec; r0 += chunk) {
        const int32_t k = std::min(chunk, n_vec - r0), B = round_up(k, 128);
        int rc;
        if ((rc = ensure_batch(ctx, *m, B))) return rc;
        if ((rc = stage_rows(ctx, *m, *n, x + (size_t)r0 * m->P, k))) return rc;
        if ((rc = run_batch(ctx, *m, m->xrows.p, m->pstride, nullptr, k, B, nullptr))) return rc;
        RN_CUDA(ctx, cudaMemcpyAsync(y + r0, m->y.p, sizeof(float) * k, cudaMemcpyDeviceToHost,
                                     ctx->stream));
        RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if ((rc = check_device_flag(ctx))) return rc;
    }
    return RN_OK;
}

int rn_mlp_gradients(rn_ctx *ctx, int32_t mlp, int32_t n_vec, const int8_t *x, const float *target,
                     float *loss, float *gW1, float *gb1, float *gW2, float *gb2, float *gw3,
                     float *gb3)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Mlp *m;
    Network *n;
    if (int rc = lookup(ctx, mlp, m, n)) return rc;
    if (n_vec < 1 || n_vec > 65536 || !x || !target)
        return fail(ctx, RN_EINVAL, "need 1 .. 65536 vectors and targets");
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    const int32_t B = round_up(n_vec, 128);
    int rc;
    if ((rc = ensure_batch(ctx, *m, B))) return rc;
    if ((rc = stage_rows(ctx, *m, *n, x, n_vec))) return rc;
    RN_CUDA(ctx, cudaMemcpyAsync(m->tgt.p, target, sizeof(float) * n_vec, cudaMemcpyHostToDevice,
                                 ctx->stream));
    if ((rc = run_batch(ctx, *m, m->xrows.p, m->pstride, nullptr, n_vec, B, m->tgt.p))) return rc;
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if ((rc = check_device_flag(ctx))) return rc;
    std::vector<float> g(m->n_theta);
    RN_CUDA(ctx, cudaMemcpy(g.data(), m->grad.p, g.size() * sizeof(float), cudaMemcpyDeviceToHost));
    double sse = 0;
    RN_CUDA(ctx, cudaMemcpy(&sse, m->loss.p, sizeof sse, cudaMemcpyDeviceToHost));
    if (loss) *loss = (float)(sse / n_vec);
    const size_t D = (size_t)m->D, H1 = (size_t)m->H1, H2 = (size_t)m->H2;
    if (gW1) std::memcpy(gW1, &g[0], D * H1 * sizeof(float));
    if (gb1) std::memcpy(gb1, &g[m->off_b1()], H1 * sizeof(float));
    if (gW2) std::memcpy(gW2, &g[m->off_W2()], H1 * H2 * sizeof(float));
    if (gb2) std::memcpy(gb2, &g[m->off_b2()], H2 * sizeof(float));
    if (gw3) std::memcpy(gw3, &g[m->off_w3()], H2 * sizeof(float));
    if (gb3) *gb3 = g[m->off_b3()];
    return RN_OK;
}

int rn_mlp_add_samples(rn_ctx *ctx, int32_t mlp, int32_t n_vec, const int8_t *x,
                       const float *target, int64_t *count)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Mlp *m;
    Network *n;
    if (int rc = lookup(ctx, mlp, m, n)) return rc;
    if (n_vec < 0 || (n_vec > 0 && (!x || !target))) return fail(ctx, RN_EINVAL, "bad samples");
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    // the last min(n, cap) pairs survive; copied in at most two runs of the ring
    const int64_t keep = std::min<int64_t>(n_vec, m->cap), first = n_vec - keep;
    std::vector<int8_t> rows((size_t)keep * m->pstride, 0);
    for (int64_t r = 0; r < keep; ++r) {
        const int8_t *xr = x + (size_t)(first + r) * m->P;
        if (int rc = check_domains(ctx, *n, xr, first + r)) return rc;
        std::memcpy(&rows[(size_t)r * m->pstride], xr, (size_t)m->P);
    }
    m->head = (m->head + first) % m->cap;
    for (int64_t r = 0; r < keep;) {
        const int64_t run = std::min(keep - r, m->cap - m->head);
        RN_CUDA(ctx, cudaMemcpy(m->set_x.p + m->head * m->pstride, &rows[(size_t)r * m->pstride],
                                (size_t)run * m->pstride, cudaMemcpyHostToDevice));
        RN_CUDA(ctx, cudaMemcpy(m->set_y.p + m->head, target + first + r, sizeof(float) * run,
                                cudaMemcpyHostToDevice));
        m->head = (m->head + run) % m->cap;
        r += run;
    }
    m->count = std::min(m->count + n_vec, m->cap);
    if (count) *count = m->count;
    return RN_OK;
}

int rn_mlp_log_chains(rn_ctx *ctx, int32_t mlp, int64_t *count)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Mlp *m;
    Network *n;
    if (int rc = lookup(ctx, mlp, m, n)) return rc;
    if (!n->chains_valid) return fail(ctx, RN_ESTATE, "the network has no chains");
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    const DevChains ch = n->chains();
    log_chains_kernel<<<(ch.n + 7) / 8, 256, 0, ctx->stream>>>(ch, m->set_x.p, m->set_y.p,
                                                               m->head, m->cap, (float)m->scale);
    if (int rc = check_launch(ctx, "log kernel")) return rc;
    m->head = (m->head + ch.n) % m->cap;
    m->count = std::min(m->count + ch.n, m->cap);
    if (count) *count = m->count;
    return RN_OK;
}

int rn_mlp_train(rn_ctx *ctx, int32_t mlp, int32_t steps, int32_t batch, float lr, uint64_t seed,
                 float *loss)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Mlp *m;
    Network *n;
    if (int rc = lookup(ctx, mlp, m, n)) return rc;
    if (steps < 0 || batch < 128 || batch > 65536 || batch % 128)
        return fail(ctx, RN_EINVAL, "batch must be a multiple of 128 in 128 .. 65536");
    if (!(lr > 0.f) || !std::isfinite(lr)) return fail(ctx, RN_EINVAL, "bad learning rate");
    if (m->count == 0) return fail(ctx, RN_ESTATE, "the training set is empty");
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    int rc;
    if ((rc = ensure_batch(ctx, *m, batch))) return rc;
    // Where the targets' spread is small against their level (below 1/16 of
    // it), they are standardised by the training set's mean and spread, so that
    // the fit spends the BF16 activations' precision (2^-8 relative) on the
    // differences between states rather than on their common level; the output
    // layer is mapped to the standardised scale for the steps and back
    // afterwards, so predictions stay in the targets' units.  An output layer
    // that has never been trained is taken to be on the standardised scale
    // already (mapping it would multiply its random outputs by 1 / sigma).
    std::vector<float> ys((size_t)m->count);
    RN_CUDA(ctx, cudaMemcpyAsync(ys.data(), m->set_y.p, sizeof(float) * ys.size(),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double mean = 0, var = 0;
    for (float v : ys) mean += v;
    mean /= (double)ys.size();
    for (float v : ys) var += ((double)v - mean) * ((double)v - mean);
    const double sd = std::sqrt(var / (double)ys.size());
    const bool standardise = sd > 1e-12 && sd < std::fabs(mean) / 16.0;
    const double mu = standardise ? mean : 0.0, sigma = standardise ? sd : 1.0;
    float *w3 = m->theta.p + m->off_w3(), *b3p = m->theta.p + m->off_b3();
    if (standardise && m->adam_t > 0) {
        affine_head_kernel<<<1, 256, 0, ctx->stream>>>(w3, m->H2, b3p, (float)(1.0 / sigma),
                                                       (float)(-mu / sigma));
        if ((rc = check_launch(ctx, "output-layer scaling"))) return rc;
    }
    // Each step's values that change from step to step (its index, for the
    // minibatch draw, and Adam's bias corrections) are read on the device, so
    // that every step is the same sequence of launches: step 0 runs directly
    // (it also settles every first-use set-up), the sequence of step 1 is
    // captured in a CUDA graph and replayed for the remaining steps, without a
    // host launch per kernel.
    const double b1 = 0.9, b2 = 0.999;
    if (steps > 0) {
        std::vector<float> cc(2 * (size_t)steps);
        for (int32_t s = 0; s < steps; ++s) {
            const double t = (double)(m->adam_t + s + 1);
            cc[2 * (size_t)s] = (float)(1.0 / (1.0 - std::pow(b1, t)));
            cc[2 * (size_t)s + 1] = (float)(1.0 / (1.0 - std::pow(b2, t)));
        }
        RN_CUDA(ctx, m->adam_c.reserve(cc.size()));
        RN_CUDA(ctx, m->train_k.reserve(1));
        RN_CUDA(ctx, cudaMemcpyAsync(m->adam_c.p, cc.data(), sizeof(float) * cc.size(),
                                     cudaMemcpyHostToDevice, ctx->stream));
        RN_CUDA(ctx, cudaMemsetAsync(m->train_k.p, 0, sizeof(uint32_t), ctx->stream));
        // the copy reads cc before the call goes on (pageable source)
        RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    auto one_step = [&]() -> int {
        sample_kernel<<<(batch + 255) / 256, 256, 0, ctx->stream>>>(
            seed, m->train_k.p, batch, (uint32_t)m->count, m->set_y.p, m->idx.p, m->tgt.p,
            (float)mu, (float)(1.0 / sigma));
        int r = check_launch(ctx, "sample kernel");
        if (r) return r;
        if ((r = run_batch(ctx, *m, m->set_x.p, m->pstride, m->idx.p, batch, batch, m->tgt.p)))
            return r;
        adam_kernel<<<1024, 256, 0, ctx->stream>>>(m->theta.p, m->grad.p, m->adam_m.p,
                                                   m->adam_v.p, m->n_theta, lr, (float)b1,
                                                   (float)b2, m->adam_c.p, m->train_k.p, 1e-8f);
        if ((r = check_launch(ctx, "Adam kernel"))) return r;
        if ((r = refresh_copies(ctx, *m))) return r;
        advance_step_kernel<<<1, 1, 0, ctx->stream>>>(m->train_k.p);
        return check_launch(ctx, "step counter");
    };
    if (steps > 0 && (rc = one_step())) return rc;
    if (steps > 1) {
        const int64_t before = ctx->launches;
        RN_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        const int rs = one_step();
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(ctx->stream, &graph);
        if (rs != RN_OK || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            (void)cudaGetLastError();
            ctx->launches = before;
            return rs != RN_OK ? rs : cuda_fail(ctx, ec, "training step (capture)");
        }
        const int64_t per_step = ctx->launches - before;
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        for (int32_t s = 1; e == cudaSuccess && s < steps; ++s) e = cudaGraphLaunch(exec, ctx->stream);
        if (exec) cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "training step (graph)");
        ctx->launches = before + per_step * (int64_t)(steps - 1);
    }
    m->adam_t += steps;
    if (standardise) {
        affine_head_kernel<<<1, 256, 0, ctx->stream>>>(w3, m->H2, b3p, (float)sigma, (float)mu);
        if ((rc = check_launch(ctx, "output-layer scaling"))) return rc;
    }
    if (loss) {
        double sse = 0;
        RN_CUDA(ctx, cudaMemcpyAsync(&sse, m->loss.p, sizeof sse, cudaMemcpyDeviceToHost,
                                     ctx->stream));
        RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if ((rc = check_device_flag(ctx))) return rc;
        *loss = steps > 0 ? (float)(sse / batch) : 0.f;
    }
    return RN_OK;
}

int rn_mlp_set_hidden_mode(rn_ctx *ctx, int32_t mlp, int32_t mode)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Mlp *m = get_mlp(ctx, mlp);
    if (!m) return fail(ctx, RN_EINVAL, "unknown screen %d", mlp);
    if (mode != 0 && mode != 1) return fail(ctx, RN_EINVAL, "hidden-row mode %d is not 0 or 1", mode);
    m->hidden_mode = mode;
    return RN_OK;
}

int rn_anneal_screened(rn_ctx *ctx, int32_t mlp, const rn_schedule *s, int32_t K, int32_t top,
                       double eps, int64_t sweeps)
{
    if (!ctx) return RN_EINVAL;
    ctx->err.clear();
    Mlp *m;
    Network *n;
    if (int rc = lookup(ctx, mlp, m, n)) return rc;
    if (!s) return fail(ctx, RN_EINVAL, "schedule is NULL");
    if (K < 1 || K > 32 || top < 1 || top > 4 || top > K)
        return fail(ctx, RN_EINVAL, "need 1 <= top <= 4, top <= K <= 32");
    if (!(eps >= 0.0 && eps <= 1.0)) return fail(ctx, RN_EINVAL, "eps must be in [0, 1]");
    if (sweeps < 0 || s->iters_per_level < 1) return fail(ctx, RN_EINVAL, "bad sweeps/schedule");
    if (!(s->T0 > 0.0) || !(s->alpha > 0.0) || !std::isfinite(s->T0) || !std::isfinite(s->alpha))
        return fail(ctx, RN_EINVAL, "T0 and alpha must be positive");
    if (s->reset_to_best || s->global_sync)
        return fail(ctx, RN_EUNSUPPORTED, "screened annealing runs without reset/global sync");
    if (!n->chains_valid) return fail(ctx, RN_ESTATE, "no chains (call rn_init_chains)");
    // propose: a warp per chain, its x and constraint counters in shared memory
    const int region = (int)(n->pstride + 2 * ((n->N + 15) & ~15));
    int smem_limit = 0;
    RN_CUDA(ctx, cudaDeviceGetAttribute(&smem_limit, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                        ctx->device));
    const int pwarps = std::min(kScreenWarps, smem_limit / std::max(region, 1));
    if (pwarps < 1)
        return fail(ctx, RN_EUNSUPPORTED, "x of %d bytes is too large for the screened step",
                    n->pstride);
    RN_CUDA(ctx, cudaSetDevice(ctx->device));
    if (sweeps == 0) return RN_OK;
    int rc;
    if ((rc = ensure_screen(ctx, *m, *n, K, top))) return rc;
    ctx->batch.g0_synced = false;
    const DevChains ch = n->chains();
    if (!m->a1_valid || m->a1_gen != ctx->gen || m->a1_step != n->step) {
        if ((rc = embed_chains(ctx, *m, ch))) return rc;
        m->a1_valid = true;
        m->a1_gen = ctx->gen;
    }
    const int64_t iters = s->iters_per_level;
    DevSched sc{};
    bool cached = false;
    if ((rc = thresholds_for(ctx, *s, n->step / iters, (n->step + sweeps - 1) / iters,
                             n->max_score, sc, cached)))
        return rc;
    sc.iters = iters;
    ScreenArgs a{};
    a.net = n->dev();
    a.ch = ch;
    a.K = K;
    a.top = top;
    a.H1 = m->H1;
    a.nparts = m->H2 / 64;
    const double et = std::floor(eps * 4294967296.0);
    a.eps_thr = et >= 4294967296.0 ? ((uint64_t)1 << 32) : (uint64_t)et;
    a.row_base = m->row_base.p;
    a.W1b = bp(m->W1b);
    a.b3 = m->theta.p + m->off_b3();
    a.A1 = m->A1.p;
    a.rows = m->rows.p;
    a.pc = m->pc.p;
    a.cand = m->cand.p;
    const size_t smem = (size_t)pwarps * region;
    const int pblocks = (ch.n + pwarps - 1) / pwarps;
    const int32_t M = round_up(ch.n * K, 128);
    GemmArgs g{};
    g.lda = m->H1; g.B = bp(m->W2T); g.ldb = m->H1;
    g.M = M; g.N = m->H2; g.K = m->H1; g.ldc = m->H2;
    g.bias = m->theta.p + m->off_b2(); g.w = m->theta.p + m->off_w3(); g.part = m->pc.p;
    // layer 2 of the K candidates: hidden rows written by the propose kernel
    // and read back by TMA (mode 1, the default), or formed inside the GEMM
    // (mode 0; widths above 512 and fewer than 8 candidates use mode 1)
    const bool fused = m->hidden_mode == 0 && gemm_hidden_supported(g, K);
    HiddenArgs hid{};
    if (fused) {
        hid.rows = m->rows.p;
        hid.A1 = m->A1.p;
        hid.W1b = bp(m->W1b);
        hid.K = K;
        hid.n_rows = ch.n * K;
    } else if (m->hc.n < (size_t)M * m->H1) {
        RN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        RN_CUDA(ctx, m->hc.alloc((size_t)M * m->H1));
        RN_CUDA(ctx, cudaMemset(m->hc.p, 0, (size_t)M * m->H1 * sizeof(uint16_t)));
    }
    a.hc = bp(m->hc);
    g.A = a.hc;
    auto propose = fused ? screen_propose_kernel<true> : screen_propose_kernel<false>;
    RN_CUDA(ctx, cudaFuncSetAttribute(propose, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    for (int64_t k = 0; k < sweeps; ++k) {
        a.g = n->step + k;
        propose<<<pblocks, pwarps * 32, smem, ctx->stream>>>(a, region);
        if ((rc = check_launch(ctx, "screen propose kernel"))) return rc;
        if (fused) {
            const cudaError_t e = launch_gemm_hidden(g, hid, ctx->dev_err.p, ctx->sm_count,
                                                     ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "layer-2 GEMM with hidden rows");
            ctx->launches += 1;
        } else if ((rc = gemm(ctx, kBiasReluDot, g))) {
            return rc;
        }
        cudaError_t e;
        if (n->lanes != 32) {
            e = launch_finish_block(a, sc, ctx->sm_count, ctx->stream);
        } else {
            // single-condition networks: the moves of two chains in one warp's byte lanes
            e = launch_finish_chains4(a, sc, n->d0, n->d1, ctx->stream);
            if (e == cudaErrorNotSupported) e = launch_finish(a, sc, ctx->stream);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "screen finish kernel");
        ctx->launches += 1;
    }
    n->step += sweeps;
    m->a1_step = n->step;
    return RN_OK;
}

}  // extern "C"
