// Migration kernels with operator anti-aliasing for 16-bit traces (constant velocity).
#include "kh_migrate_impl.cuh"

namespace kh {
cudaError_t launch_migrate_aa_f16(const GeomParams& g, const TileShape& t, const TraceSet& tr, const void* traces,
                                  float* image, int vel, int fast, const WaitCfg& w, cudaStream_t s)
{
    return launch_migrate_aa_t<__half>(g, t, tr, traces, image, vel, fast, w, s);
}

cudaError_t launch_migrate_aa_bf16(const GeomParams& g, const TileShape& t, const TraceSet& tr, const void* traces,
                                   float* image, int vel, int fast, const WaitCfg& w, cudaStream_t s)
{
    return launch_migrate_aa_t<__nv_bfloat16>(g, t, tr, traces, image, vel, fast, w, s);
}
}  // namespace kh
