// Instantiations of the specialised inverse table-driven NTT phase kernels with the
// modular products for primes = 1 (mod 2^32) (ntt_kernel.cuh); a translation
// unit of its own so that it compiles in parallel with the others.
#include "ntt_kernel.cuh"

namespace ckks {

cudaError_t ntt_dispatch_q1_table_inv(bool cols, int logn, const NttPhase &P, const NttJob *jobs, int n_jobs,
                                      const LoadSpec &L, const StoreSpec &S, const PhaseLaunch &G, bool &found) {
    return dispatch_fast<false, true, true>(cols, logn, P, nullptr, jobs, n_jobs, L, S, G, found);
}

}  // namespace ckks
