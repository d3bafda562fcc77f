// rn_noalloc.cu -- rn_level_sync_noalloc: the level-end argmin and broadcast on
// caller-owned device buffers, with its scratch in a fixed device array so that
// the call allocates nothing.
//
// Its scratch is g_noalloc_scratch below: one 64-bit key (objective << 32 |
// chain index) per block of the first pass and one for the winner, 8 KiB in
// all, resident on every device that loads the library until the process
// exits.  Host code never uses the array's name as an address: the address is
// resolved once per device with cudaGetSymbolAddress and handed to the
// kernels.
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/rnanneal.h"

namespace rn {
void set_detached_error(const char *fmt, ...);
int check_device_span(const void *p, size_t bytes, int device, const char *name, char *why,
                      size_t why_len);
}

namespace {

constexpr int kThreads = 1024;                  // chains per first-pass block
constexpr int kBlocks = 1024;                   // first-pass blocks (scratch slots)
constexpr int64_t kMaxChains = (int64_t)kThreads * kBlocks;   // 1,048,576
constexpr int kMaxDevices = 64;

// Every call shares this array and leaves its contents behind.  Each call
// writes every slot it later reads (slots 0 .. blocks-1, then the winner slot)
// before reading it, so nothing has to start at zero.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kBlocks + 1];

__device__ __forceinline__ unsigned long long block_min(unsigned long long v)
{
    __shared__ unsigned long long part[32];
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : ~0ull;
        for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}

// Pass 1: the lowest (objective, chain) key of each block's chains.
__global__ void partial_min(const int32_t *__restrict__ d_best, int32_t n,
                            unsigned long long *scratch)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long key =
        k < n ? (((unsigned long long)(uint32_t)d_best[k] << 32) | (uint32_t)k) : ~0ull;
    const unsigned long long m = block_min(key);
    if (threadIdx.x == 0) scratch[blockIdx.x] = m;
}

// Pass 2: the lowest key over the blocks, stored in the winner slot.
__global__ void final_min(int32_t blocks, unsigned long long *scratch)
{
    const unsigned long long key = (int)threadIdx.x < blocks ? scratch[threadIdx.x] : ~0ull;
    const unsigned long long m = block_min(key);
    if (threadIdx.x == 0) scratch[kBlocks] = m;
}

// Pass 3: copy the winner's row and objective into every other chain.
__global__ void broadcast_rows(int8_t *x_best, int32_t *d_best, int32_t n, int64_t row_bytes,
                               int32_t n_params, const unsigned long long *scratch)
{
    const int w = (int)(uint32_t)scratch[kBlocks];
    const int chain = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (chain >= n || chain == w) return;
    const int8_t *src = x_best + (int64_t)w * row_bytes;
    int8_t *dst = x_best + (int64_t)chain * row_bytes;
    for (int j = lane; j < n_params; j += 32) dst[j] = src[j];
    if (lane == 0) d_best[chain] = d_best[w];
}

std::mutex g_mutex;
unsigned long long *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, resolved on the
// first call for that device and kept for the life of the process.  A
// cudaDeviceReset unloads the library's device code, so the kept address is
// stale afterwards: the header rules out calls after a reset.
int scratch_address(int dev, unsigned long long **out)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();   // not left behind for a later call's launch check
            rn::set_detached_error("cudaGetSymbolAddress(scratch) on device %d: %s", dev,
                                   cudaGetErrorString(e));
            return RN_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_scratch_ptr[dev];
    return RN_OK;
}

}  // namespace

extern "C" int rn_level_sync_noalloc(int8_t *x_best, int32_t *d_best, int32_t n_chains,
                                     int64_t row_bytes, int32_t n_params, void *stream)
{
    if (!x_best || !d_best) {
        rn::set_detached_error("x_best and d_best must be device pointers");
        return RN_EINVAL;
    }
    if (n_chains < 1 || (int64_t)n_chains > kMaxChains) {
        rn::set_detached_error("n_chains %d outside 1 .. %lld (the fixed scratch holds %d "
                               "partial minima of %d chains)",
                               n_chains, (long long)kMaxChains, kBlocks, kThreads);
        return RN_EINVAL;
    }
    if (n_params < 1 || row_bytes < n_params) {
        rn::set_detached_error("need 1 <= n_params <= row_bytes");
        return RN_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        rn::set_detached_error("no usable current device");
        return RN_ECUDA;
    }
    char why[256];
    if (rn::check_device_span(x_best, (size_t)(n_chains - 1) * (size_t)row_bytes +
                                          (size_t)n_params,
                              dev, "x_best", why, sizeof why) != RN_OK ||
        rn::check_device_span(d_best, (size_t)n_chains * sizeof(int32_t), dev, "d_best", why,
                              sizeof why) != RN_OK) {
        rn::set_detached_error("%s", why);
        return RN_EINVAL;
    }
    unsigned long long *scratch = nullptr;
    const int rc = scratch_address(dev, &scratch);
    if (rc != RN_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int blocks = (int)((n_chains + kThreads - 1) / kThreads);
    partial_min<<<blocks, kThreads, 0, st>>>(d_best, n_chains, scratch);
    final_min<<<1, kThreads, 0, st>>>(blocks, scratch);
    broadcast_rows<<<(n_chains + 7) / 8, 256, 0, st>>>(x_best, d_best, n_chains, row_bytes,
                                                       n_params, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        rn::set_detached_error("level sync kernels: %s", cudaGetErrorString(e));
        return RN_ECUDA;
    }
    return RN_OK;
}
