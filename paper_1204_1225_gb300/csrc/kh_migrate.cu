// Migration, batched-migration and velocity-gradient launches: dispatch on the trace type to
// the per-type translation units (kh_migrate_<type>.cu, kh_migrate_aa_<type>.cu with operator
// anti-aliasing, kh_batched_<type>.cu), the gradient
// kernels (FP32 traces only, instantiated here) and the gradient's final sum.
#include "kh_migrate_impl.cuh"

namespace kh {

#define KH_MIGRATE_DECL(name)                                                                            \
    cudaError_t name(const GeomParams&, const TileShape&, const TraceSet&, const void*, float*, int, int,     \
                     const WaitCfg&, cudaStream_t);
KH_MIGRATE_DECL(launch_migrate_f32)
KH_MIGRATE_DECL(launch_migrate_pair)
KH_MIGRATE_DECL(launch_migrate_f16)
KH_MIGRATE_DECL(launch_migrate_bf16)
KH_MIGRATE_DECL(launch_migrate_aa_f32)
KH_MIGRATE_DECL(launch_migrate_aa_pair)
KH_MIGRATE_DECL(launch_migrate_aa_f16)
KH_MIGRATE_DECL(launch_migrate_aa_bf16)
#undef KH_MIGRATE_DECL

#define KH_BATCHED_DECL(name)                                                                            \
    cudaError_t name(const GeomParams&, const BatchJob*, const int4*, int, int*, int, int, int, int,          \
                     const WaitCfg&, int, int*, cudaStream_t);
KH_BATCHED_DECL(launch_batched_f32)
KH_BATCHED_DECL(launch_batched_pair)
KH_BATCHED_DECL(launch_batched_f16)
KH_BATCHED_DECL(launch_batched_bf16)
#undef KH_BATCHED_DECL

size_t migrate_smem_bytes(const GeomParams& g) { return mig_smem_bytes(g); }

cudaError_t launch_migrate_batched(const GeomParams& gm, const BatchJob* jobs, const int4* items, int n_items,
                                   int* next, int vel_kind, int weight, int fast, int lg_terms,
                                   int trace_dtype, const WaitCfg& w, int ctas, int* ctas_out,
                                   cudaStream_t s)
{
    switch (trace_dtype) {
        case KH_F32:
            if (gm.pairs)
                return launch_batched_pair(gm, jobs, items, n_items, next, vel_kind, weight, fast, lg_terms, w, ctas,
                                           ctas_out, s);
            return launch_batched_f32(gm, jobs, items, n_items, next, vel_kind, weight, fast, lg_terms, w, ctas,
                                      ctas_out, s);
        case KH_F16:
            return launch_batched_f16(gm, jobs, items, n_items, next, vel_kind, weight, fast, lg_terms, w, ctas,
                                      ctas_out, s);
        case KH_BF16:
            return launch_batched_bf16(gm, jobs, items, n_items, next, vel_kind, weight, fast, lg_terms, w, ctas,
                                       ctas_out, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_migrate(const GeomParams& g, const TileShape& t, const TraceSet& tr,
                           const void* traces, float* image, int vel_kind, int fast_math,
                           const WaitCfg& w, cudaStream_t s)
{
    if (t.cz > MAX_ZG) return cudaErrorInvalidValue;
    if (g.pstm) vel_kind = VK_PSTM;   // time migration has kernels of its own
    if (g.aa_c > 0.f) {   // operator anti-aliasing has kernels of its own
        switch (g.tdtype) {
            case KH_F32:
                return g.pairs ? launch_migrate_aa_pair(g, t, tr, traces, image, vel_kind, fast_math, w, s)
                               : launch_migrate_aa_f32(g, t, tr, traces, image, vel_kind, fast_math, w, s);
            case KH_F16: return launch_migrate_aa_f16(g, t, tr, traces, image, vel_kind, fast_math, w, s);
            case KH_BF16: return launch_migrate_aa_bf16(g, t, tr, traces, image, vel_kind, fast_math, w, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (g.tdtype) {
        case KH_F32:
            return g.pairs ? launch_migrate_pair(g, t, tr, traces, image, vel_kind, fast_math, w, s)
                           : launch_migrate_f32(g, t, tr, traces, image, vel_kind, fast_math, w, s);
        case KH_F16: return launch_migrate_f16(g, t, tr, traces, image, vel_kind, fast_math, w, s);
        case KH_BF16: return launch_migrate_bf16(g, t, tr, traces, image, vel_kind, fast_math, w, s);
        default: return cudaErrorInvalidValue;
    }
}

static cudaError_t launch_vgrad_impl(const GeomParams& g, const TileShape& t, const TraceSet& tr,
                                     const float* traces, const float* image, int vel, int fast, const WaitCfg& w,
                                     double* partial, cudaStream_t s)
{
    const int key = vel * 4 + g.weight * 2 + (fast ? 1 : 0);
    switch (key) {
        case 0: return launch_vgrad_t<VK_CONST, 0, false>(g, t, tr, traces, image, w, partial, s);
        case 1: return launch_vgrad_t<VK_CONST, 0, true>(g, t, tr, traces, image, w, partial, s);
        case 2: return launch_vgrad_t<VK_CONST, 1, false>(g, t, tr, traces, image, w, partial, s);
        case 3: return launch_vgrad_t<VK_CONST, 1, true>(g, t, tr, traces, image, w, partial, s);
        case 4: return launch_vgrad_t<VK_LINEAR, 0, false>(g, t, tr, traces, image, w, partial, s);
        case 5: return launch_vgrad_t<VK_LINEAR, 0, true>(g, t, tr, traces, image, w, partial, s);
        case 6: return launch_vgrad_t<VK_LINEAR, 1, false>(g, t, tr, traces, image, w, partial, s);
        case 7: return launch_vgrad_t<VK_LINEAR, 1, true>(g, t, tr, traces, image, w, partial, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_vgrad(const GeomParams& g, const TileShape& t, const TraceSet& tr,
                         const void* traces, const float* image, int vel_kind, int fast_math,
                         const WaitCfg& w, double* partial, cudaStream_t s)
{
    if (t.cz > MAX_ZG || !partial) return cudaErrorInvalidValue;
    if (g.tdtype != KH_F32 || vel_kind == VK_TABLE || g.weight == KH_W_TRUE_AMP) return cudaErrorInvalidValue;
    return launch_vgrad_impl(g, t, tr, static_cast<const float*>(traces), image, vel_kind, fast_math, w, partial,
                             s);
}

// out[0..1] = (sum of the per-warp partials, in index order) / dt: one CTA, fixed order.
__global__ void k_vgrad_reduce(const double* __restrict__ partial, long long n, double inv_dt,
                               double* __restrict__ out)
{
    __shared__ double s0[256], s1[256];
    double a = 0.0, b = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        a += partial[2 * i];
        b += partial[2 * i + 1];
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s0[threadIdx.x] += s0[threadIdx.x + w];
            s1[threadIdx.x] += s1[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = s0[0] * inv_dt;
        out[1] = s1[0] * inv_dt;
    }
}

cudaError_t launch_vgrad_reduce(const double* partial, long long n, double inv_dt, double* out,
                                cudaStream_t s)
{
    k_vgrad_reduce<<<1, 256, 0, s>>>(partial, n, inv_dt, out);
    return cudaGetLastError();
}

}  // namespace kh
