// FP32-trace instantiations of the migration and velocity-gradient kernels.
#include "kh_migrate_impl.cuh"

namespace kh {
cudaError_t launch_dtype_f32(const GeomParams& g, const TileShape& t, const TraceSet& tr, const void* traces,
                             float* image, int vel, int fast, const WaitCfg& w, double* partial,
                             cudaStream_t s)
{
    return launch_dtype<float>(g, t, tr, traces, image, vel, fast, w, partial, s);
}
}  // namespace kh
