// rn_umma.cu -- host side of the tcgen05 GEMM: TMA tensor maps (encoded with
// the CUDA driver API's cuTensorMapEncodeTiled, resolved through the runtime so that
// the library needs no link against libcuda) and the persistent launch.
#include <cudaTypedefs.h>

#include "rn_umma.cuh"

namespace rn {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Row-major BF16 matrix [rows][ld] read in boxes of box_rows x 64 elements,
// 128-byte swizzle (the layout the shared-memory descriptors describe).
bool make_map(CUtensorMap *m, const void *ptr, int inner, int rows, int ld, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || (reinterpret_cast<uintptr_t>(ptr) & 15)) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)umma::BK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box,
              es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <int EPI>
cudaError_t launch_t(const CUtensorMap &a, const CUtensorMap &b, const GemmArgs &g, int *err,
                     int grid, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(umma::gemm_tc_kernel<EPI>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)umma::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    umma::gemm_tc_kernel<EPI><<<grid, umma::THREADS, umma::SMEM_BYTES, st>>>(a, b, g, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_hidden(const GemmArgs &g, const HiddenArgs &h, int *err, int sm_count,
                               cudaStream_t st)
{
    if (!gemm_hidden_supported(g, h.K) || !err || !h.rows || !h.A1 || !h.W1b || h.K < 1 ||
        h.n_rows < 0 || h.n_rows > g.M)
        return cudaErrorInvalidValue;
    CUtensorMap b;
    if (!make_map(&b, g.B, g.K, g.N, g.ldb, umma::BN)) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(umma::gemm_hidden_kernel<kBiasReluDot>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)umma::HSMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int tiles = (g.M / umma::BM) * (g.N / umma::BN);
    const int grid = tiles < sm_count ? tiles : sm_count;
    umma::gemm_hidden_kernel<kBiasReluDot><<<grid, umma::HTHREADS, umma::HSMEM_BYTES, st>>>(b, g, h,
                                                                                         err);
    return cudaGetLastError();
}

cudaError_t launch_gemm_tc(int epi, const GemmArgs &g, int *err, int sm_count, cudaStream_t st)
{
    if (!gemm_tc_supported(g) || !err) return cudaErrorInvalidValue;
    CUtensorMap a, b;
    if (!make_map(&a, g.A, g.K, g.M, g.lda, umma::BM) ||
        !make_map(&b, g.B, g.K, g.N, g.ldb, umma::BN))
        return cudaErrorInvalidValue;
    const int tiles = (g.M / umma::BM) * (g.N / umma::BN);
    const int grid = tiles < sm_count ? tiles : sm_count;
    switch (epi) {
    case kStoreF32: return launch_t<kStoreF32>(a, b, g, err, grid, st);
    case kBiasReluBf16: return launch_t<kBiasReluBf16>(a, b, g, err, grid, st);
    case kBiasReluDot: return launch_t<kBiasReluDot>(a, b, g, err, grid, st);
    case kMaskBf16: return launch_t<kMaskBf16>(a, b, g, err, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace rn
