// kirchhoff_migrate_noalloc: the migration without any device allocation.
//
// Some callers cannot call cudaMalloc: services whose device memory is owned by another
// allocator (a framework's caching pool that has reserved most of HBM), and latency-bound
// services that must not allocate after start-up because cudaMalloc can synchronise the
// device and stall every stream.  The plan path (kirchhoff_create / kirchhoff_migrate)
// allocates its trace-sort workspace; this entry point instead uses one file-scope
// __device__ array of fixed size, so the caller only passes inputs and outputs.
#include <mutex>

#include "kh_plan.h"

namespace {

// Traces one call can bin and sort without allocating.
constexpr int NOALLOC_MAX_TRACES = 65536;
constexpr int NOALLOC_MAX_BINS = 256;
constexpr int NOALLOC_MAX_DEVICES = 64;

// Scratch of the binning pass (2.1 MB).  Every GPU that loads the library holds one copy
// until the process exits; every call on that device reuses it.
struct NoallocScratch {
    int bin[NOALLOC_MAX_TRACES];
    int perm[NOALLOC_MAX_TRACES];
    float4 hdr[NOALLOC_MAX_TRACES];
    float2 mid[NOALLOC_MAX_TRACES];
    int bin_start[NOALLOC_MAX_BINS + 1];
    int status[4];
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

std::mutex g_noalloc_mu;
NoallocScratch* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch on the current device.  In host code the symbol is only a
// host-side stand-in, so the address is looked up once per device, with that device current,
// on the first call made on it.
kh_status noalloc_scratch(NoallocScratch** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return kh::set_cuda_error(e, "kirchhoff_migrate_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return kh::set_error(KH_ERR_UNSUPPORTED, "kirchhoff_migrate_noalloc: device index above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return kh::set_cuda_error(e, "kirchhoff_migrate_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = static_cast<NoallocScratch*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return KH_OK;
}

}  // namespace

extern "C" kh_status kirchhoff_migrate_noalloc(const kh_desc* d, int ntr, const float* sx,
                                               const float* sy, const float* rx, const float* ry,
                                               const void* traces, float* image, int* status,
                                               void* cuda_stream)
{
    using namespace kh;
    if (!d) return set_error(KH_ERR_INVALID_ARG, "kirchhoff_migrate_noalloc: desc is NULL");
    if (ntr < 0 || ntr > NOALLOC_MAX_TRACES)
        return set_error(KH_ERR_INVALID_ARG,
                         "kirchhoff_migrate_noalloc: ntr must be in [0, 65536] (the fixed scratch "
                         "holds 65536 traces); use kirchhoff_migrate for larger surveys");
    if (d->trace_dtype != KH_F32)
        return set_error(KH_ERR_UNSUPPORTED, "kirchhoff_migrate_noalloc: FP32 traces only");
    if (d->vel == KH_VEL_TABLE || d->vel == KH_VEL_GRID)
        return set_error(KH_ERR_UNSUPPORTED, "kirchhoff_migrate_noalloc: analytic traveltimes only "
                                             "(a table needs device workspace)");
    if (!image || (ntr > 0 && (!sx || !rx || !traces)) || (ntr > 0 && d->dim == 3 && (!sy || !ry)))
        return set_error(KH_ERR_INVALID_ARG, "kirchhoff_migrate_noalloc: NULL array");
    if (ntr > 0 && ((reinterpret_cast<uintptr_t>(traces) & 15u) != 0 || (d->nt % 4) != 0))
        return set_error(KH_ERR_INVALID_ARG, "kirchhoff_migrate_noalloc: trace rows must be 16-byte "
                                             "aligned (aligned pointer, nt a multiple of 4)");
    GeomParams g;
    TileShape t;
    kh_status st = noalloc_prepare(d, &g, &t);
    if (st != KH_OK) return st;
    NoallocScratch* sc = nullptr;
    if ((st = noalloc_scratch(&sc)) != KH_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int* stw = status ? status : sc->status;
    cudaError_t e = cudaMemsetAsync(stw, 0, sizeof(int), s);
    if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_migrate_noalloc: status reset");
    if (ntr == 0) {
        e = cudaMemsetAsync(image, 0, sizeof(float) * (size_t)d->n_bins * d->ny * d->nx * d->nz, s);
        return e == cudaSuccess ? KH_OK : set_cuda_error(e, "kirchhoff_migrate_noalloc: cudaMemsetAsync");
    }
    e = noalloc_bin(ntr, sx, sy, rx, ry, *d, sc->bin, sc->perm, sc->bin_start, sc->hdr, sc->mid, s);
    if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_migrate_noalloc: binning kernels");
    g.ld = d->nt;
    TraceSet ts{sc->hdr, sc->mid, sc->perm, sc->bin_start};
    WaitCfg w{stw, 0, WAIT_NS};
    e = launch_migrate(g, t, ts, traces, image, g.k == 0.0 ? VK_CONST : VK_LINEAR, 1, w, s);
    return e == cudaSuccess ? KH_OK : set_cuda_error(e, "kirchhoff_migrate_noalloc: migration kernel");
}
