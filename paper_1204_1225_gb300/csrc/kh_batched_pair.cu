// Batched persistent migration kernel for FP32 traces staged as SamplePair rows.
#include "kh_migrate_impl.cuh"

namespace kh {
cudaError_t launch_batched_pair(const GeomParams& gm, const BatchJob* jobs, const int4* items, int n_items, int* next,
                                int vel, int weight, int fast, int lg_terms, const WaitCfg& w, int ctas, int* ctas_out,
                                cudaStream_t s)
{
    return launch_batched_dtype<SamplePair>(gm, jobs, items, n_items, next, vel, weight, fast, lg_terms, w, ctas,
                                            ctas_out, s);
}
}  // namespace kh
