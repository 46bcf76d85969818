// Instantiations of the specialised forward uniform-batch NTT phase kernels with the
// modular products for primes = 1 (mod 2^32) (ntt_kernel.cuh); a translation
// unit of its own so that it compiles in parallel with the others.
#include "ntt_kernel.cuh"

namespace ckks {

cudaError_t ntt_dispatch_q1_uniform_fwd(bool cols, int logn, const NttPhase &P, const LimbJobs &J,
                                        const LoadSpec &L, const StoreSpec &S, const PhaseLaunch &G, bool &found) {
    return dispatch_fast<true, false, true>(cols, logn, P, &J, nullptr, 0, L, S, G, found);
}

}  // namespace ckks
