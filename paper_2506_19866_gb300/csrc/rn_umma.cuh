// rn_umma.cuh -- BF16 GEMM on the fifth-generation tensor cores: tcgen05.mma
// with FP32 accumulators in tensor memory (TMEM), operands staged in shared
// memory by TMA, fused epilogues read back with tcgen05.ld.
//
//   C[M][N] = A[M][K] * B[N][K]^T      (both operands K-major, BF16)
//
// Persistent kernel, one CTA per SM, 128 x 256 output tiles (one
// M = 128, N = 256 MMA per K step of 16), K in blocks of 64 (one 128-byte
// swizzle atom per operand row):
//   warp 0      TMA producer: A and B tiles of each K block into a 4-stage ring
//   warp 1      allocates 512 TMEM columns (two accumulators); one lane issues
//               the MMAs and commits each stage back to the producer and each
//               finished accumulator to the epilogue
//   warps 2-5   epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its
//               subpartition), i.e. those rows of the tile, 32 columns at a
//               time, applies the epilogue of rn_gemm.cuh and stores
// Two accumulators let the epilogue of one tile overlap the MMAs of the next.
// Every mbarrier wait is bounded: past kWaitCycles (or when another role has
// given up) the role stops, the CTA records the failure in *err, waits (again
// bounded) for its copies and MMAs in flight, frees TMEM and returns.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "rn_gemm.cuh"

namespace rn {
namespace umma {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;              // 16 KiB
constexpr int B_BYTES = BN * BK * 2;              // 32 KiB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t TMEM_COLS = 2 * BN;             // two FP32 accumulators
constexpr int THREADS = 192;
constexpr long long kWaitCycles = 4000000000LL;    // about 2 s of SM clock
constexpr int kErrCode = 2;                        // value written to *err

struct Ctl {
    uint64_t full[STAGES];     // stage loaded (TMA transaction bytes)
    uint64_t empty[STAGES];    // stage consumed (MMA commit)
    uint64_t tfull[2];         // accumulator complete (MMA commit)
    uint64_t tempty[2];        // accumulator read (one arrival per epilogue warp)
    uint64_t done;             // every issued MMA complete
    uint32_t tmem;             // TMEM base address written by tcgen05.alloc
    int abort;
    int consumed;              // stages the MMA role consumed
    int pflag[2];              // the hidden-row producers' shared wait result (per parity)
};

constexpr size_t SMEM_BYTES = 1024 + (size_t)STAGES * STAGE_BYTES + sizeof(Ctl) + 64;

__device__ __forceinline__ uint32_t su32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// As mbar_test, but the thread may sleep up to about `ns` nanoseconds inside
// the try_wait (woken when the phase completes), so that waiting roles take
// few issue slots from the warps that work.
__device__ __forceinline__ bool mbar_test_sleep(uint64_t *b, uint32_t parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Wait for the phase of parity `parity` to complete.  Gives up (false) when
// another role has aborted (watch_abort) or after kWaitCycles, then marks the
// CTA aborted and records the failure.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, Ctl *c, int *err,
                                          bool watch_abort = true, uint32_t sleep_ns = 0)
{
    if (mbar_test(b, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (sleep_ns ? mbar_test_sleep(b, parity, sleep_ns) : mbar_test(b, parity)) return true;
        if (watch_abort && *(volatile int *)&c->abort) return false;
        if (clock64() - t0 > kWaitCycles) {
            *(volatile int *)&c->abort = 1;
            atomicExch(err, kErrCode);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile stored with the 128-byte
// swizzle (rows of 128 bytes, 8-row groups 1024 bytes apart, tile base
// 1024-byte aligned): start address >> 4, leading offset 16 B (unused for this
// layout), stride offset 1024 B, descriptor version 1, swizzle mode 2 (128 B).
__device__ __forceinline__ uint64_t sw128_desc(const void *tile)
{
    const uint64_t a = su32(tile);
    return ((a >> 4) & 0x3FFFull) | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane; the wait is in the
// same statement so that no use of the registers precedes it.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
        "[%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Epilogue of 32 columns [col, col + 32) of row `row`.
template <int EPI>
__device__ __forceinline__ void epilogue32(const GemmArgs &g, int row, int col, const float (&v)[32],
                                           float &dot)
{
    if constexpr (EPI == kStoreF32) {
        float4 *o = reinterpret_cast<float4 *>(g.out_f32 + (size_t)row * g.ldc + col);
#pragma unroll
        for (int i = 0; i < 8; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else if constexpr (EPI == kMaskBf16) {
        const uint4 *mk = reinterpret_cast<const uint4 *>(g.mask + (size_t)row * g.ldc + col);
        uint4 *o = reinterpret_cast<uint4 *>(g.out_bf16 + (size_t)row * g.ldc + col);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint4 m = mk[i];
            const __nv_bfloat162 *m2 = reinterpret_cast<const __nv_bfloat162 *>(&m);
            uint4 ov;
            __nv_bfloat162 *o2 = reinterpret_cast<__nv_bfloat162 *>(&ov);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(m2[e]);
                o2[e] = __floats2bfloat162_rn(f.x > 0.f ? v[8 * i + 2 * e] : 0.f,
                                              f.y > 0.f ? v[8 * i + 2 * e + 1] : 0.f);
            }
            o[i] = ov;
        }
    } else {
        // relu(acc + bias), 8 columns at a time (bias and w as float4)
        const float4 *bias4 = reinterpret_cast<const float4 *>(g.bias + col);
        const float4 *w4 = reinterpret_cast<const float4 *>(g.w + col);
        uint4 *o = g.out_bf16 ? reinterpret_cast<uint4 *>(g.out_bf16 + (size_t)row * g.ldc + col)
                              : nullptr;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 b0 = __ldg(bias4 + 2 * i), b1 = __ldg(bias4 + 2 * i + 1);
            float h[8] = {v[8 * i] + b0.x, v[8 * i + 1] + b0.y, v[8 * i + 2] + b0.z,
                          v[8 * i + 3] + b0.w, v[8 * i + 4] + b1.x, v[8 * i + 5] + b1.y,
                          v[8 * i + 6] + b1.z, v[8 * i + 7] + b1.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) h[e] = fmaxf(h[e], 0.f);
            if (o) {
                uint4 ov;
                __nv_bfloat162 *o2 = reinterpret_cast<__nv_bfloat162 *>(&ov);
#pragma unroll
                for (int e = 0; e < 4; ++e) o2[e] = __floats2bfloat162_rn(h[2 * e], h[2 * e + 1]);
                o[i] = ov;
            }
            if constexpr (EPI == kBiasReluDot) {
                const float4 w0 = __ldg(w4 + 2 * i), w1 = __ldg(w4 + 2 * i + 1);
                dot += h[0] * w0.x + h[1] * w0.y + h[2] * w0.z + h[3] * w0.w + h[4] * w1.x +
                       h[5] * w1.y + h[6] * w1.z + h[7] * w1.w;
            }
        }
    }
}

template <int EPI>
__global__ void __launch_bounds__(THREADS, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   GemmArgs g, int *err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    Ctl *c = reinterpret_cast<Ctl *>(base + (size_t)STAGES * STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tn = g.N / BN, tiles = (g.M / BM) * tn, nk = g.K / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&c->full[s], 1);
            mbar_init(&c->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&c->tfull[a], 1);
            mbar_init(&c->tempty[a], 4);
        }
        mbar_init(&c->done, 1);
        c->abort = 0;
        c->consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&c->tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = c->tmem;
    int issued = 0;

    if (warp == 0 && lane == 0) {
        // TMA producer
        int stage = 0;
        uint32_t phase = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
            const int m0 = (t / tn) * BM, n0 = (t % tn) * BN;
            bool ok = true;
            for (int kb = 0; kb < nk; ++kb) {
                if (!mbar_wait(&c->empty[stage], phase ^ 1u, c, err)) { ok = false; break; }
                uint8_t *sa = base + (size_t)stage * STAGE_BYTES;
                mbar_expect_tx(&c->full[stage], STAGE_BYTES);
                tma_load_2d(sa, &tmA, &c->full[stage], kb * BK, m0);
                tma_load_2d(sa + A_BYTES, &tmB, &c->full[stage], kb * BK, n0);
                ++issued;
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
            if (!ok) break;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        int stage = 0, acc = 0, consumed = 0;
        uint32_t phase = 0, aphase = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
            if (!mbar_wait(&c->tempty[acc], aphase ^ 1u, c, err)) break;
            fence_after();
            const uint32_t d = tmem + (uint32_t)acc * BN;
            bool ok = true;
            for (int kb = 0; kb < nk; ++kb) {
                if (!mbar_wait(&c->full[stage], phase, c, err)) { ok = false; break; }
                fence_after();
                ++consumed;
                const uint8_t *sa = base + (size_t)stage * STAGE_BYTES;
                const uint64_t da = sw128_desc(sa), db = sw128_desc(sa + A_BYTES);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    mma_bf16(d, da + 2ull * kk, db + 2ull * kk, (kb | kk) != 0);
                mma_commit(&c->empty[stage]);
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
            if (!ok) break;
            mma_commit(&c->tfull[acc]);
            acc ^= 1;
            if (acc == 0) aphase ^= 1u;
        }
        c->consumed = consumed;
        // every MMA this thread issued has completed before TMEM is released
        mma_commit(&c->done);
        mbar_wait(&c->done, 0, c, err, false);
    } else if (warp >= 2) {
        // epilogue: rows 32 (warp % 4) + lane of each tile
        const int q = warp & 3;
        int acc = 0;
        uint32_t aphase = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
            // lane 0 waits for the whole warp, so that the .sync.aligned TMEM
            // loads below run converged
            int ok = 0;
            if (lane == 0) ok = mbar_wait(&c->tfull[acc], aphase, c, err);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            fence_after();
            const int m0 = (t / tn) * BM, n0 = (t % tn) * BN;
            const int row = m0 + q * 32 + lane;
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)acc * BN;
            float part[BN / 64];
#pragma unroll 1
            for (int h = 0; h < BN / 64; ++h) {
                float dot = 0.f;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    float v[32];
                    tmem_ld32(ta + (uint32_t)(h * 64 + s * 32), v);
                    epilogue32<EPI>(g, row, n0 + h * 64 + s * 32, v, dot);
                }
                part[h] = dot;
            }
            if constexpr (EPI == kBiasReluDot) {
                float4 *o = reinterpret_cast<float4 *>(g.part + (size_t)row * (g.N / 64) + n0 / 64);
#pragma unroll
                for (int h = 0; h < BN / 256; ++h)
                    o[h] = make_float4(part[4 * h], part[4 * h + 1], part[4 * h + 2], part[4 * h + 3]);
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&c->tempty[acc]);
            acc ^= 1;
            if (acc == 0) aphase ^= 1u;
        }
    }
    __syncthreads();
    if (warp == 0 && lane == 0 && *(volatile int *)&c->abort) {
        // loads issued but never consumed land before the CTA exits
        for (int i = c->consumed; i < issued; ++i)
            mbar_wait(&c->full[i % STAGES], (uint32_t)((i / STAGES) & 1), c, err, false);
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

// ---- layer-2 GEMM of the screen with its A operand produced in the kernel ----
//
// The same warp roles as gemm_tc_kernel, with TMA loading only B (W2^T) and
// eight more warps (6-13) producing each A stage from the candidates' W1 rows
// and A1 (HiddenArgs): thread p of the producers owns row p / 2 of the tile and
// its 32-column half p % 2 of the K block.  Its two W1 row segments (new and
// old value, 64 bytes each) and the A1 rows of the tile's chains come through
// a ring of HDEPTH staging slots filled by cp.async HDEPTH K blocks ahead, so
// that the gathers' L2 latency overlaps the arithmetic and the MMAs.  Each producer thread writes its BF16 values into
// the stage in the 128-byte-swizzled K-major layout that TMA would have
// written and makes them visible to the tensor core's proxy
// (fence.proxy.async.shared::cta); after a named barrier over the producers
// one of them arrives on the stage's full barrier (one TMA arrival plus one
// producer arrival: 256 arrivals on one barrier word would serialise).  The
// same producer waits on the stage's empty barrier (bounded) and passes the
// result to the others through the named barrier, so that all producers leave
// together when a wait gives up.  This
// avoids the HBM round trip of the hidden rows (written by the propose
// kernel, read back by TMA: for 4096 chains x 32 candidates x 512 columns,
// 134 MB each way per step), but it runs slower on GB300: per K block each SM
// takes in 32 KB of scattered W1 segments beside the 32 KB B tile, and the A
// stage is rebuilt for every 256-column output tile, so the library's default
// is the round trip (rn_mlp_set_hidden_mode).
constexpr int HSTAGES = 2;                                  // GEMM stages (A produced, B by TMA)
constexpr uint32_t kSleepNs = 2000;                         // try_wait sleep hint of waiting roles
constexpr int HDEPTH = 3;                                   // staging slots (K blocks ahead)
constexpr int HPROD = 256;                                  // producer threads
constexpr int HTHREADS = 192 + HPROD;
constexpr int HMIN_K = 8;                                   // candidates per chain, at least
constexpr int HSTAGING_BYTES = BM * 2 * BK * 2;             // new and old W1 rows of a K block
constexpr int HA1_BYTES = (BM / HMIN_K + 2) * BK * 4;       // A1 of the tile's chains
constexpr int HSLOT_BYTES = HSTAGING_BYTES + HA1_BYTES;
constexpr size_t HSMEM_BYTES =
    1024 + (size_t)HSTAGES * STAGE_BYTES + (size_t)HDEPTH * HSLOT_BYTES + sizeof(Ctl) + 64;
static_assert(HSMEM_BYTES <= 232448, "one CTA's shared memory");

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void producers_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(HPROD) : "memory");
}

template <int EPI>
__global__ void __launch_bounds__(HTHREADS, 1)
    gemm_hidden_kernel(const __grid_constant__ CUtensorMap tmB, GemmArgs g, HiddenArgs h, int *err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    uint8_t *staging = base + (size_t)HSTAGES * STAGE_BYTES;
    Ctl *c = reinterpret_cast<Ctl *>(staging + (size_t)HDEPTH * HSLOT_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tn = g.N / BN, tiles = (g.M / BM) * tn, nk = g.K / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < HSTAGES; ++s) {
            mbar_init(&c->full[s], 2);
            mbar_init(&c->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&c->tfull[a], 1);
            mbar_init(&c->tempty[a], 4);
        }
        mbar_init(&c->done, 1);
        c->abort = 0;
        c->consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(&c->tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = c->tmem;
    int issued = 0;

    if (warp == 0 && lane == 0) {
        // TMA producer of B
        int stage = 0;
        uint32_t phase = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
            const int n0 = (t % tn) * BN;
            bool ok = true;
            for (int kb = 0; kb < nk; ++kb) {
                if (!mbar_wait(&c->empty[stage], phase ^ 1u, c, err, true, kSleepNs)) { ok = false; break; }
                uint8_t *sa = base + (size_t)stage * STAGE_BYTES;
                mbar_expect_tx(&c->full[stage], B_BYTES);
                tma_load_2d(sa + A_BYTES, &tmB, &c->full[stage], kb * BK, n0);
                ++issued;
                if (++stage == HSTAGES) { stage = 0; phase ^= 1u; }
            }
            if (!ok) break;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        int stage = 0, acc = 0, consumed = 0;
        uint32_t phase = 0, aphase = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
            if (!mbar_wait(&c->tempty[acc], aphase ^ 1u, c, err, true, kSleepNs)) break;
            fence_after();
            const uint32_t d = tmem + (uint32_t)acc * BN;
            bool ok = true;
            for (int kb = 0; kb < nk; ++kb) {
                if (!mbar_wait(&c->full[stage], phase, c, err, true, kSleepNs)) { ok = false; break; }
                fence_after();
                ++consumed;
                const uint8_t *sa = base + (size_t)stage * STAGE_BYTES;
                const uint64_t da = sw128_desc(sa), db = sw128_desc(sa + A_BYTES);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    mma_bf16(d, da + 2ull * kk, db + 2ull * kk, (kb | kk) != 0);
                mma_commit(&c->empty[stage]);
                if (++stage == HSTAGES) { stage = 0; phase ^= 1u; }
            }
            if (!ok) break;
            mma_commit(&c->tfull[acc]);
            acc ^= 1;
            if (acc == 0) aphase ^= 1u;
        }
        c->consumed = consumed;
        mma_commit(&c->done);
        mbar_wait(&c->done, 0, c, err, false);
    } else if (warp >= 2 && warp < 6) {
        // epilogue (EPI = kBiasReluDot, the screen's layer 2): rows 32 (warp % 4)
        // + lane of each tile
        static_assert(EPI == kBiasReluDot, "the partial sums of the screen's layer 2");
        const int q = warp & 3;
        int acc = 0;
        uint32_t aphase = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
            int ok = 0;
            if (lane == 0) ok = mbar_wait(&c->tfull[acc], aphase, c, err, true, kSleepNs);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            fence_after();
            const int m0 = (t / tn) * BM, n0 = (t % tn) * BN;
            const int row = m0 + q * 32 + lane;
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)acc * BN;
            float part[BN / 64];
#pragma unroll 1
            for (int hh = 0; hh < BN / 64; ++hh) {
                float dot = 0.f;
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    float v[32];
                    tmem_ld32(ta + (uint32_t)(hh * 64 + s * 32), v);
                    epilogue32<EPI>(g, row, n0 + hh * 64 + s * 32, v, dot);
                }
                part[hh] = dot;
            }
            float4 *o = reinterpret_cast<float4 *>(g.part + (size_t)row * (g.N / 64) + n0 / 64);
#pragma unroll
            for (int hh = 0; hh < BN / 256; ++hh)
                o[hh] = make_float4(part[4 * hh], part[4 * hh + 1], part[4 * hh + 2], part[4 * hh + 3]);
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&c->tempty[acc]);
            acc ^= 1;
            if (acc == 0) aphase ^= 1u;
        }
    } else if (warp >= 6) {
        // producers of A
        const int p = threadIdx.x - 192;
        const int r = p >> 1, half = p & 1;
        const int my_tiles = blockIdx.x < tiles ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
        const int n_iter = my_tiles * nk;
        const int ldw = g.K;   // W1 and A1 rows are K-dimension long
        // A K block of this CTA, advanced one block at a time (divisions only
        // when it enters a new tile): the tile's first row, this thread's row
        // R and its W1 rows, and the tile's first chain.
        struct Pos {
            int i, kb, tile, R, c0, cl;   // cl: this row's chain, counted from c0
            int2 rw;
        };
        auto enter_tile = [&](Pos &q) {
            const int m0 = (q.tile / tn) * BM;
            q.R = m0 + r;
            q.c0 = m0 / h.K;
            q.cl = q.R / h.K - q.c0;
            q.rw = q.R < h.n_rows ? __ldg(h.rows + q.R) : make_int2(-1, -1);
        };
        auto start = [&](int i) {
            Pos q;
            q.i = i;
            q.kb = i % nk;
            q.tile = blockIdx.x + (i / nk) * gridDim.x;
            enter_tile(q);
            return q;
        };
        auto advance = [&](Pos &q) {
            ++q.i;
            if (++q.kb == nk) {
                q.kb = 0;
                q.tile += gridDim.x;
                if (q.i < n_iter) enter_tile(q);
            }
        };
        // staging slot i % HDEPTH: this thread's W1 segments, then the tile's
        // A1 segments (chains c0 .. of the tile's rows)
        auto issue = [&](const Pos &q) {
            if (q.i < n_iter) {
                uint8_t *slot = staging + (size_t)(q.i % HDEPTH) * HSLOT_BYTES;
                if (q.R < h.n_rows && q.rw.x >= 0) {
                    const __nv_bfloat16 *wn = h.W1b + (size_t)q.rw.x * ldw + q.kb * BK + half * 32;
                    const __nv_bfloat16 *wo = h.W1b + (size_t)q.rw.y * ldw + q.kb * BK + half * 32;
#pragma unroll
                    for (int ch = 0; ch < 4; ++ch) {
                        cp_async16(slot + ((size_t)ch * HPROD + p) * 16, wn + ch * 8);
                        cp_async16(slot + ((size_t)(4 + ch) * HPROD + p) * 16, wo + ch * 8);
                    }
                }
                // A1: 16 chunks of 16 bytes per chain of the tile
                const int m0 = q.R - r;
                const int last = min(m0 + BM, h.n_rows) - 1;
                const int n_chunks = last >= m0 ? (last / h.K - q.c0 + 1) * 16 : 0;
                for (int k = p; k < n_chunks; k += HPROD)
                    cp_async16(slot + HSTAGING_BYTES + (size_t)k * 16,
                               h.A1 + (size_t)(q.c0 + (k >> 4)) * ldw + q.kb * BK + (k & 15) * 4);
            }
            cp_async_commit();
        };
        Pos qc = start(0), qi = start(0);
#pragma unroll 1
        for (int k = 0; k < HDEPTH; ++k) {
            issue(qi);
            advance(qi);
        }
        int stage = 0;
        uint32_t phase = 0;
        for (int i = 0; i < n_iter; ++i) {
            cp_async_wait<HDEPTH - 1>();
            if (p == 0) c->pflag[i & 1] = mbar_wait(&c->empty[stage], phase ^ 1u, c, err, true, kSleepNs) ? 1 : 0;
            producers_sync();
            if (!*(volatile int *)&c->pflag[i & 1]) break;
            const bool valid = qc.R < h.n_rows;
            const uint8_t *slot = staging + (size_t)(i % HDEPTH) * HSLOT_BYTES;
            const float *a1 = reinterpret_cast<const float *>(slot + HSTAGING_BYTES) +
                              (valid ? qc.cl * BK : 0) + half * 32;
            uint8_t *sa = base + (size_t)stage * STAGE_BYTES + (size_t)r * 128;
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                const float4 lo = *reinterpret_cast<const float4 *>(a1 + ch * 8);
                const float4 hi = *reinterpret_cast<const float4 *>(a1 + ch * 8 + 4);
                float v[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
                if (valid && qc.rw.x >= 0) {
                    const uint4 wn = *reinterpret_cast<const uint4 *>(slot + ((size_t)ch * HPROD + p) * 16);
                    const uint4 wo =
                        *reinterpret_cast<const uint4 *>(slot + ((size_t)(4 + ch) * HPROD + p) * 16);
                    const __nv_bfloat162 *pn = reinterpret_cast<const __nv_bfloat162 *>(&wn);
                    const __nv_bfloat162 *po = reinterpret_cast<const __nv_bfloat162 *>(&wo);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float2 fn = __bfloat1622float2(pn[e]), fo = __bfloat1622float2(po[e]);
                        v[2 * e] += fn.x - fo.x;
                        v[2 * e + 1] += fn.y - fo.y;
                    }
                }
                uint4 ov = make_uint4(0u, 0u, 0u, 0u);
                if (valid) {
                    __nv_bfloat162 *o2 = reinterpret_cast<__nv_bfloat162 *>(&ov);
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        o2[e] = __floats2bfloat162_rn(fmaxf(v[2 * e], 0.f), fmaxf(v[2 * e + 1], 0.f));
                }
                // 16-byte chunk (half * 4 + ch) of the row, 128-byte swizzle
                const int cc = (half * 4 + ch) ^ (r & 7);
                *reinterpret_cast<uint4 *>(sa + cc * 16) = ov;
            }
            fence_proxy_async();
            producers_sync();
            if (p == 0) mbar_arrive(&c->full[stage]);
            issue(qi);
            advance(qi);
            advance(qc);
            if (++stage == HSTAGES) { stage = 0; phase ^= 1u; }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0 && lane == 0 && *(volatile int *)&c->abort) {
        for (int i = c->consumed; i < issued; ++i)
            mbar_wait(&c->full[i % HSTAGES], (uint32_t)((i / HSTAGES) & 1), c, err, false);
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

}  // namespace umma

// Shapes the fused layer-2 kernel covers: those of gemm_tc_supported with
// N <= 512 (wider layers repeat the A production per 256 columns) and at
// least 8 candidates per chain (the A1 rows of a tile's chains are staged).
inline bool gemm_hidden_supported(const GemmArgs &g, int candidates)
{
    return g.M > 0 && g.M % umma::BM == 0 && g.N > 0 && g.N % umma::BN == 0 && g.N <= 512 &&
           g.K > 0 && g.K % umma::BK == 0 && g.ldb % 8 == 0 && g.part && g.bias && g.w &&
           candidates >= umma::HMIN_K;
}

// The fused launch (rn_umma.cu); *err is set by a CTA whose wait gave up.
cudaError_t launch_gemm_hidden(const GemmArgs &g, const HiddenArgs &h, int *err, int sm_count,
                               cudaStream_t st);

// Shapes the tcgen05 kernel covers: M % 128, N % 256, K % 64, 16-byte aligned
// rows.
inline bool gemm_tc_supported(const GemmArgs &g)
{
    return g.M > 0 && g.N > 0 && g.K > 0 && g.M % umma::BM == 0 && g.N % umma::BN == 0 &&
           g.K % umma::BK == 0 && g.lda % 8 == 0 && g.ldb % 8 == 0 && g.ldc % 8 == 0;
}

// Launch on the tcgen05 path (rn_umma.cu); *err is set by a CTA whose wait gave up.
cudaError_t launch_gemm_tc(int epi, const GemmArgs &g, int *err, int sm_count, cudaStream_t st);

}  // namespace rn
