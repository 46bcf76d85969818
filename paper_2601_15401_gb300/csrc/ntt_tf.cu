// Instantiations of the forward table-driven (cross-shape) NTT phase kernels (ntt_kernel.cuh);
// one translation unit per direction and job source so that they compile in
// parallel.
#include "ntt_kernel.cuh"

namespace ckks {

cudaError_t ntt_dispatch_table_fwd(bool cols, int logn, const NttPhase &P, const NttJob *jobs, int n_jobs,
                                  const LoadSpec &L, const StoreSpec &S, const PhaseLaunch &G) {
    return dispatch_phase<true, true>(cols, logn, P, nullptr, jobs, n_jobs, L, S, G);
}

}  // namespace ckks
