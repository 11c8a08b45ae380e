// Migration kernels with operator anti-aliasing for FP32 traces staged as SamplePair rows.
#include "kh_migrate_impl.cuh"

namespace kh {
cudaError_t launch_migrate_aa_pair(const GeomParams& g, const TileShape& t, const TraceSet& tr, const void* traces,
                                   float* image, int vel, int fast, const WaitCfg& w, cudaStream_t s)
{
    return launch_migrate_aa_t<SamplePair>(g, t, tr, traces, image, vel, fast, w, s);
}
}  // namespace kh
