// rn_anneal1.cu -- annealing kernels with 1 node(s) per lane (one translation
// unit per layout so that they compile in parallel).
#include "rn_kernels.cuh"

namespace rn {

cudaError_t launch_anneal_npl1(const DevNet &net, int d0, int d1, const DevChains &ch,
                               const DevSched &sc, int sm_count, cudaStream_t st)
{
#define RN_CASE(NPL_, CG_, A, B)                                                         \
    if (net.cg == CG_ && d0 == A && d1 == B)                                             \
        return launch_anneal_t<NPL_, CG_, A, B>(net, ch, sc, sm_count, st);
    RN_CASE(1, 1, 4, 1) RN_CASE(1, 1, 8, 1) RN_CASE(1, 1, 12, 1) RN_CASE(1, 1, 16, 1)
    RN_CASE(1, 4, 4, 1) RN_CASE(1, 4, 8, 1) RN_CASE(1, 4, 12, 1) RN_CASE(1, 4, 16, 1)
#undef RN_CASE
    return cudaErrorNotSupported;
}

}  // namespace rn
