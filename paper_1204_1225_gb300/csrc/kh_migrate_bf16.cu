// BF16-trace instantiations of the migration kernel (mixed precision: 16-bit trace storage
// in HBM and shared memory, FP32 interpolation and accumulation).
#include "kh_migrate_impl.cuh"

namespace kh {
cudaError_t launch_migrate_bf16(const GeomParams& g, const TileShape& t, const TraceSet& tr, const void* traces,
                               float* image, int vel, int fast, const WaitCfg& w, cudaStream_t s)
{
    return launch_migrate_dtype<__nv_bfloat16>(g, t, tr, traces, image, vel, fast, w, s);
}
}  // namespace kh
