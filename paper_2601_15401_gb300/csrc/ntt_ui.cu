// Instantiations of the inverse uniform-batch NTT phase kernels (ntt_kernel.cuh);
// one translation unit per direction and job source so that they compile in
// parallel.
#include "ntt_kernel.cuh"

namespace ckks {

cudaError_t ntt_dispatch_uniform_inv(bool cols, int logn, const NttPhase &P, const LimbJobs &J, const LoadSpec &L,
                                    const StoreSpec &S, const PhaseLaunch &G) {
    return dispatch_phase<false, false>(cols, logn, P, &J, nullptr, 0, L, S, G);
}

}  // namespace ckks
