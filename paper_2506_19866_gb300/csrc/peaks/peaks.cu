// peaks.cu -- microbenchmarks of the per-SM issue rates that bound the
// annealing kernel: 32-bit integer ALU operations (LOP3/IADD3-class and
// IMAD-class) and shared-memory byte loads.  Each block records its SM and
// its start and end on that SM's clock (clock64 with a memory clobber, so no
// load moves across it); the rate of an SM is the work of its blocks over the
// span from the first start to the last end.  The result is in operations per
// SM clock, independent of the clock the GPU runs at.  Measurement
// infrastructure for the benchmark; not part of the annealing library.
#include <algorithm>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace {

constexpr int kIters = 4096;

__device__ __forceinline__ unsigned long long stamp()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%clock64;" : "=l"(t)::"memory");
    return t;
}

__device__ __forceinline__ unsigned smid()
{
    unsigned s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

__device__ __forceinline__ void record(unsigned long long *rec, unsigned long long t0,
                                       unsigned long long t1)
{
    if (threadIdx.x == 0) {
        rec[3 * blockIdx.x + 0] = smid();
        rec[3 * blockIdx.x + 1] = t0;
        rec[3 * blockIdx.x + 2] = t1;
    }
}

// 8 independent dependency chains per thread, 2 instructions per chain step
// (an IADD3 with three operands, then a LOP3 of three operands): 16 per step.
__global__ void alu_kernel(uint32_t seed, uint32_t *sink, unsigned long long *rec)
{
    uint32_t a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed * (threadIdx.x + 7 * k + 1);
    const uint32_t b = seed ^ blockIdx.x, c = seed + 0x9E3779B9u, d = seed * 3u;
    __syncthreads();
    const unsigned long long t0 = stamp();
#pragma unroll 4
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            a[k] = a[k] + b + c;
            a[k] = (a[k] ^ d) & (a[k] | c);
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r ^= a[k];
    if (r == 0x12345678u) sink[0] = r;
    __syncthreads();
    record(rec, t0, stamp());
}

// 8 independent chains of multiply-add (IMAD class): 16 per step.
__global__ void imad_kernel(uint32_t seed, uint32_t *sink, unsigned long long *rec)
{
    uint32_t a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed * (threadIdx.x + 7 * k + 1);
    const uint32_t b = seed | 1u, c = seed + 0x9E3779B9u;
    __syncthreads();
    const unsigned long long t0 = stamp();
#pragma unroll 4
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            a[k] = a[k] * b + c;
            a[k] = a[k] * c + b;
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r ^= a[k];
    if (r == 0x12345678u) sink[0] = r;
    __syncthreads();
    record(rec, t0, stamp());
}

// Byte loads from a 128-byte shared array at data-dependent addresses (the
// gather pattern of the simulator): 8 independent chains per thread.  A chain
// of loads cannot be scheduled outside the timed span: the first addresses
// take a term of the start stamp (zero in practice, unknown to the compiler)
// and the end stamp, after the barrier, is read under a branch on the loaded
// values (a warp reaches the barrier only after all but its last load).
__global__ void lds_kernel(uint32_t seed, uint32_t *sink, unsigned long long *rec)
{
    __shared__ uint8_t tab[128];
    if (threadIdx.x < 128) tab[threadIdx.x] = (uint8_t)((threadIdx.x * 37u + seed) & 127u);
    __syncthreads();
    const unsigned long long t0 = stamp();
    const uint32_t z = (uint32_t)(t0 >> 62);
    uint32_t a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = ((threadIdx.x * 5u + 11u * k) ^ z) & 127u;
#pragma unroll 4
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = tab[a[k]];
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r ^= a[k];
    __syncthreads();
    unsigned long long t1 = 0;
    if (r != seed) t1 = stamp();   // always taken: r < 128 <= seed
    else sink[0] = r;
    record(rec, t0, t1);
}

}  // namespace

// Runs one of the kernels (0: ALU, 1: IMAD, 2: shared byte loads; seed 12345,
// at least 128 as the shared-load kernel requires) with
// `blocks_per_sm` blocks of 256 threads per SM; returns the median over SMs of
// operations per SM clock (ALU / IMAD: per-lane operations; shared loads:
// warp-level load instructions), or a negative value on failure.
extern "C" double rnpk_ops_per_sm_clock(int which, int blocks_per_sm)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1.0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * blocks_per_sm, threads = 256;
    uint32_t *sink = nullptr;
    unsigned long long *rec = nullptr;
    if (cudaMalloc(&sink, 4) != cudaSuccess) return -2.0;
    if (cudaMalloc(&rec, sizeof(unsigned long long) * 3 * blocks) != cudaSuccess) {
        cudaFree(sink);
        return -2.0;
    }
    for (int rep = 0; rep < 2; ++rep) {   // the first run warms up
        if (which == 0) alu_kernel<<<blocks, threads>>>(12345u, sink, rec);
        else if (which == 1) imad_kernel<<<blocks, threads>>>(12345u, sink, rec);
        else lds_kernel<<<blocks, threads>>>(12345u, sink, rec);
    }
    double result = -3.0;
    if (cudaDeviceSynchronize() == cudaSuccess) {
        std::vector<unsigned long long> h((size_t)3 * blocks);
        cudaMemcpy(h.data(), rec, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost);
        std::vector<unsigned long long> lo((size_t)sms, ~0ull), hi((size_t)sms, 0ull);
        std::vector<int> cnt((size_t)sms, 0);
        for (int b = 0; b < blocks; ++b) {
            const unsigned s = (unsigned)h[3 * (size_t)b];
            if (s >= (unsigned)sms) continue;
            lo[s] = std::min(lo[s], h[3 * (size_t)b + 1]);
            hi[s] = std::max(hi[s], h[3 * (size_t)b + 2]);
            cnt[s]++;
        }
        const double per_block = which == 2 ? (double)kIters * 8 * (threads / 32)
                                            : (double)kIters * 16 * threads;
        std::vector<double> rate;
        for (int s = 0; s < sms; ++s)
            if (cnt[(size_t)s] > 0 && hi[(size_t)s] > lo[(size_t)s])
                rate.push_back(per_block * cnt[(size_t)s] / (double)(hi[(size_t)s] - lo[(size_t)s]));
        if (!rate.empty()) {
            std::sort(rate.begin(), rate.end());
            result = rate[rate.size() / 2];
        }
    }
    cudaFree(sink);
    cudaFree(rec);
    return result;
}
