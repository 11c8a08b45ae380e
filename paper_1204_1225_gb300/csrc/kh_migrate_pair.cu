// Migration kernel instantiations for FP32 traces staged as SamplePair rows (constant and
// linear v(z), time migration, gridded-model tables; radial-table migrations stage plain samples).
#include "kh_migrate_impl.cuh"

namespace kh {
cudaError_t launch_migrate_pair(const GeomParams& g, const TileShape& t, const TraceSet& tr, const void* traces,
                                float* image, int vel, int fast, const WaitCfg& w, cudaStream_t s)
{
    if (g.weight == KH_W_TRUE_AMP) {   // constant velocity only (the plan refuses the others)
        if (vel != VK_CONST) return cudaErrorInvalidValue;
        return fast ? launch_migrate_t<VK_CONST, 2, true, SamplePair>(g, t, tr, traces, image, w, s)
                    : launch_migrate_t<VK_CONST, 2, false, SamplePair>(g, t, tr, traces, image, w, s);
    }
    const int key = vel * 4 + g.weight * 2 + (fast ? 1 : 0);
    switch (key) {
        case 0: return launch_migrate_t<VK_CONST, 0, false, SamplePair>(g, t, tr, traces, image, w, s);
        case 1: return launch_migrate_t<VK_CONST, 0, true, SamplePair>(g, t, tr, traces, image, w, s);
        case 2: return launch_migrate_t<VK_CONST, 1, false, SamplePair>(g, t, tr, traces, image, w, s);
        case 3: return launch_migrate_t<VK_CONST, 1, true, SamplePair>(g, t, tr, traces, image, w, s);
        case 4: return launch_migrate_t<VK_LINEAR, 0, false, SamplePair>(g, t, tr, traces, image, w, s);
        case 5: return launch_migrate_t<VK_LINEAR, 0, true, SamplePair>(g, t, tr, traces, image, w, s);
        case 6: return launch_migrate_t<VK_LINEAR, 1, false, SamplePair>(g, t, tr, traces, image, w, s);
        case 7: return launch_migrate_t<VK_LINEAR, 1, true, SamplePair>(g, t, tr, traces, image, w, s);
        case 12: return launch_migrate_t<VK_PSTM, 0, false, SamplePair>(g, t, tr, traces, image, w, s);
        case 13: return launch_migrate_t<VK_PSTM, 0, true, SamplePair>(g, t, tr, traces, image, w, s);
        case 14: return launch_migrate_t<VK_PSTM, 1, false, SamplePair>(g, t, tr, traces, image, w, s);
        case 15: return launch_migrate_t<VK_PSTM, 1, true, SamplePair>(g, t, tr, traces, image, w, s);
        case 16:
        case 17: return launch_migrate_t<VK_GRID, 0, true, SamplePair>(g, t, tr, traces, image, w, s);
        case 18:
        case 19: return launch_migrate_t<VK_GRID, 1, true, SamplePair>(g, t, tr, traces, image, w, s);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace kh
