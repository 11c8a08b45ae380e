// FP32-trace instantiations of the migration kernel.
#include "kh_migrate_impl.cuh"

namespace kh {
cudaError_t launch_migrate_f32(const GeomParams& g, const TileShape& t, const TraceSet& tr, const void* traces,
                              float* image, int vel, int fast, const WaitCfg& w, cudaStream_t s)
{
    return launch_migrate_dtype<float>(g, t, tr, traces, image, vel, fast, w, s);
}
}  // namespace kh
