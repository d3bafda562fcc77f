// rn_anneal4.cu -- annealing kernels with 4 node(s) per lane (one translation
// unit per layout so that they compile in parallel).
#include "rn_kernels.cuh"

namespace rn {

cudaError_t launch_anneal_npl4(const DevNet &net, int d0, int d1, const DevChains &ch,
                               const DevSched &sc, int sm_count, cudaStream_t st)
{
#define RN_CASE(NPL_, CG_, A, B)                                                         \
    if (net.cg == CG_ && d0 == A && d1 == B)                                             \
        return launch_anneal_t<NPL_, CG_, A, B>(net, ch, sc, sm_count, st);
    RN_ANNEAL_PAIRS(RN_CASE, 4, 1)
    RN_ANNEAL_PAIRS(RN_CASE, 4, 4)
#undef RN_CASE
    return cudaErrorNotSupported;
}

}  // namespace rn
