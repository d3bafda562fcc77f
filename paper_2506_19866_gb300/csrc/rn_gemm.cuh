// rn_gemm.cuh -- BF16 tensor-core GEMM with FP32 accumulation and fused
// epilogues, for the learned proposal screen.
//
//   C[M][N] = A[M][K] * B[N][K]^T        (both operands K-major, row-major storage)
//
// Block tile 128 x 128 x 32, four warps of 64 x 64, operands staged in shared
// memory by 16-byte cp.async (double buffered), fragments by ldmatrix, math by
// mma.sync m16n8k16 (bf16 x bf16 -> f32).  M and N must be multiples of 128
// and K a multiple of 32 (callers pad).
//
// Epilogues:
//   kStoreF32      C as float
//   kBiasReluBf16  relu(C + bias[n]) as bf16
//   kBiasReluDot   relu(C + bias[n]) . w[n], summed per row over the 64 columns
//                  of each warp into part[row][N / 64] (and, when out != null,
//                  relu(C + bias) as bf16 too)
//   kMaskBf16      C * [mask > 0] as bf16 (mask: a bf16 matrix with C's layout),
//                  the back-propagation of a ReLU layer
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace rn {

enum GemmEpilogue : int { kStoreF32 = 0, kBiasReluBf16 = 1, kBiasReluDot = 2, kMaskBf16 = 3 };

struct GemmArgs {
    const __nv_bfloat16 *A;
    const __nv_bfloat16 *B;
    int lda, ldb;
    int M, N, K;
    float *out_f32;             // kStoreF32
    __nv_bfloat16 *out_bf16;    // kBiasReluBf16 / kBiasReluDot (optional)
    int ldc;
    const float *bias;          // [N]
    const float *w;             // [N] (kBiasReluDot)
    float *part;                // [M][N / 64] (kBiasReluDot)
    const __nv_bfloat16 *mask;  // [M][ldc] (kMaskBf16)
};

// The screen's layer-2 A operand produced inside the tcgen05 GEMM instead of
// read from memory: row R (candidate R % K of chain R / K) is
//   relu(A1[R / K] + (W1[rows[R].x] - W1[rows[R].y]))   rounded to BF16,
// relu(A1[R / K]) when rows[R].x < 0 (no candidate), and 0 for R >= n_rows.
struct HiddenArgs {
    const int2 *rows;           // [M] (W1 row of the new value, W1 row of the old value)
    const float *A1;            // [chains][K dimension of the GEMM] layer-1 pre-activations
    const __nv_bfloat16 *W1b;   // [Dp][K dimension] BF16 layer-1 weights
    int K;                      // candidates per chain
    int n_rows;                 // chains * K
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void *smem)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int EPI>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(GemmArgs g)
{
    constexpr int BM = 128, BN = 128, BK = 32, LDS = BK + 8;   // padded rows: 80 bytes
    __shared__ __align__(16) __nv_bfloat16 sA[2][BM][LDS];
    __shared__ __align__(16) __nv_bfloat16 sB[2][BN][LDS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

    float acc[4][8][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[i][j][v] = 0.f;

    // each thread moves 4 chunks of 8 elements of A and of B per stage
    auto load_stage = [&](int buf, int k0) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int chunk = tid + c * 128;        // 0 .. 511
            const int row = chunk >> 2, col = (chunk & 3) * 8;
            cp_async16(&sA[buf][row][col], g.A + (size_t)(m0 + row) * g.lda + k0 + col);
            cp_async16(&sB[buf][row][col], g.B + (size_t)(n0 + row) * g.ldb + k0 + col);
        }
        cp_async_commit();
    };

    const int n_k = g.K / BK;
    load_stage(0, 0);
    for (int kt = 0; kt < n_k; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < n_k) {
            load_stage(buf ^ 1, (kt + 1) * BK);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t a[4][4], b[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                ldmatrix_x4(a[i], &sA[buf][wm * 64 + i * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
                ldmatrix_x4(b[jj], &sB[buf][wn * 64 + jj * 16 + (lane & 7) + ((lane >> 4) << 3)]
                                      [kk + ((lane >> 3) & 1) * 8]);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    mma_bf16(acc[i][2 * jj], a[i], b[jj][0], b[jj][1]);
                    mma_bf16(acc[i][2 * jj + 1], a[i], b[jj][2], b[jj][3]);
                }
        }
        __syncthreads();
    }

    // epilogue: accumulator (i, j, v) is row wm*64 + i*16 + lane/4 (+8 for v >= 2),
    // column wn*64 + j*8 + (lane%4)*2 (+1 for odd v)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int row = m0 + wm * 64 + i * 16 + (lane >> 2) + h * 8;
            float dot = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int col = n0 + wn * 64 + j * 8 + (lane & 3) * 2;
                float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
                if constexpr (EPI == kStoreF32) {
                    *reinterpret_cast<float2 *>(g.out_f32 + (size_t)row * g.ldc + col) =
                        make_float2(v0, v1);
                } else if constexpr (EPI == kMaskBf16) {
                    const float2 m = __bfloat1622float2(
                        *reinterpret_cast<const __nv_bfloat162 *>(g.mask + (size_t)row * g.ldc + col));
                    *reinterpret_cast<__nv_bfloat162 *>(g.out_bf16 + (size_t)row * g.ldc + col) =
                        __floats2bfloat162_rn(m.x > 0.f ? v0 : 0.f, m.y > 0.f ? v1 : 0.f);
                } else {
                    v0 = fmaxf(v0 + g.bias[col], 0.f);
                    v1 = fmaxf(v1 + g.bias[col + 1], 0.f);
                    if (g.out_bf16)
                        *reinterpret_cast<__nv_bfloat162 *>(g.out_bf16 + (size_t)row * g.ldc +
                                                            col) = __floats2bfloat162_rn(v0, v1);
                    if constexpr (EPI == kBiasReluDot) dot += v0 * g.w[col] + v1 * g.w[col + 1];
                }
            }
            if constexpr (EPI == kBiasReluDot) {
                dot += __shfl_xor_sync(0xffffffffu, dot, 1);
                dot += __shfl_xor_sync(0xffffffffu, dot, 2);
                if ((lane & 3) == 0)
                    g.part[(size_t)row * (g.N / 64) + (n0 + wn * 64) / 64] = dot;
            }
        }
    }
}

inline cudaError_t launch_gemm(int epi, const GemmArgs &g, cudaStream_t st)
{
    if (g.M % 128 || g.N % 128 || g.K % 32 || g.M <= 0 || g.N <= 0 || g.K <= 0)
        return cudaErrorInvalidValue;
    const dim3 grid(g.N / 128, g.M / 128);
    switch (epi) {
    case kStoreF32: gemm_bf16_kernel<kStoreF32><<<grid, 128, 0, st>>>(g); break;
    case kBiasReluBf16: gemm_bf16_kernel<kBiasReluBf16><<<grid, 128, 0, st>>>(g); break;
    case kBiasReluDot: gemm_bf16_kernel<kBiasReluDot><<<grid, 128, 0, st>>>(g); break;
    case kMaskBf16: gemm_bf16_kernel<kMaskBf16><<<grid, 128, 0, st>>>(g); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace rn
