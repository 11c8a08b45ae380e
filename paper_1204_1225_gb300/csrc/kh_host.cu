// Host-resident migration, pipelined across calls: the headers and traces come from host
// memory and the image goes back to host memory.  Two slots of plan-owned device buffers
// alternate, and two plan-owned copy streams carry the copies (one per direction), so that call
// n's host-to-device copy overlaps call n-1's migration and call n-1's image copy overlaps call
// n's migration.  Events order the reuse of a slot: its inputs are overwritten only after the
// slot's previous migration has read them, and its image only after the previous image copy
// out of it has finished.
#include <algorithm>

#include "kh_plan.h"

namespace kh {

static void host_free_slot(kh_plan_s::HostSlot& k)
{
    cudaFree(k.hdr);
    cudaFree(k.traces);
    cudaFree(k.image);
    if (k.in_done) cudaEventDestroy(k.in_done);
    if (k.mig_done) cudaEventDestroy(k.mig_done);
    if (k.out_done) cudaEventDestroy(k.out_done);
    k = kh_plan_s::HostSlot{};
}

void host_release(kh_plan_s* p)
{
    for (auto& k : p->host) host_free_slot(k);
    if (p->host_in) cudaStreamDestroy(p->host_in);
    if (p->host_out) cudaStreamDestroy(p->host_out);
    p->host_in = p->host_out = nullptr;
    p->host_next = 0;
}

// Device buffers of slot k for ntr traces (the slot's outstanding work is waited for before a
// buffer is replaced), its image and its events.
static kh_status host_slot_ready(kh_plan_s* p, kh_plan_s::HostSlot& k, int ntr, size_t trace_bytes,
                                 size_t image_bytes)
{
    cudaError_t e = cudaSuccess;
    const bool grow_hdr = (size_t)ntr > k.cap_ntr, grow_tr = trace_bytes > k.cap_tr;
    if ((grow_hdr || grow_tr) && k.used) {
        e = cudaEventSynchronize(k.mig_done);
        if (e == cudaSuccess) e = cudaEventSynchronize(k.out_done);
        if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_migrate_host: waiting for a slot");
    }
    if (grow_hdr) {
        cudaFree(k.hdr);
        k.hdr = nullptr;
        k.cap_ntr = 0;
        const size_t n = std::max<size_t>((size_t)ntr + ntr / 4, 256);
        if ((e = cudaMalloc(reinterpret_cast<void**>(&k.hdr), 4 * n * sizeof(float))) != cudaSuccess)
            return set_cuda_error(e, "kirchhoff_migrate_host: header buffers");
        k.cap_ntr = n;
    }
    if (grow_tr) {
        cudaFree(k.traces);
        k.traces = nullptr;
        k.cap_tr = 0;
        const size_t n = std::max<size_t>(trace_bytes + trace_bytes / 4, 256);
        if ((e = cudaMalloc(reinterpret_cast<void**>(&k.traces), n)) != cudaSuccess)
            return set_cuda_error(e, "kirchhoff_migrate_host: trace buffer");
        k.cap_tr = n;
    }
    if (!k.image) {
        if ((e = cudaMalloc(reinterpret_cast<void**>(&k.image), image_bytes)) != cudaSuccess)
            return set_cuda_error(e, "kirchhoff_migrate_host: image buffer");
    }
    for (cudaEvent_t* ev : {&k.in_done, &k.mig_done, &k.out_done}) {
        if (!*ev && (e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
            return set_cuda_error(e, "kirchhoff_migrate_host: events");
    }
    return KH_OK;
}

}  // namespace kh

using namespace kh;

extern "C" kh_status kirchhoff_migrate_host(kh_plan p, int ntr, const float* sx, const float* sy,
                                            const float* rx, const float* ry, const void* traces,
                                            float* image, void* cuda_stream)
{
    if (!p) return set_error(KH_ERR_INVALID_ARG, "plan is NULL");
    if (ntr < 0) return set_error(KH_ERR_INVALID_ARG, "kirchhoff_migrate_host: ntr must be >= 0");
    if (!image) return set_error(KH_ERR_INVALID_ARG, "kirchhoff_migrate_host: image is NULL");
    if (ntr > 0 && (!sx || !rx || !traces || (p->d.dim == 3 && (!sy || !ry))))
        return set_error(KH_ERR_INVALID_ARG, "kirchhoff_migrate_host: NULL header or trace array");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaSuccess;
    if (!p->host_in) {
        if ((e = cudaStreamCreateWithFlags(&p->host_in, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&p->host_out, cudaStreamNonBlocking)) != cudaSuccess)
            return set_cuda_error(e, "kirchhoff_migrate_host: copy streams");
    }
    const size_t hdr_bytes = (size_t)ntr * sizeof(float);
    const size_t tr_bytes = (size_t)ntr * p->d.nt * (p->d.trace_dtype == KH_F32 ? 4 : 2);
    const size_t img_bytes = (size_t)p->d.n_bins * p->d.ny * p->d.nx * p->d.nz * sizeof(float);
    kh_plan_s::HostSlot& k = p->host[p->host_next];
    kh_status st = host_slot_ready(p, k, ntr, tr_bytes, img_bytes);
    if (st != KH_OK) return st;
    float* dh[4] = {k.hdr, k.hdr + k.cap_ntr, k.hdr + 2 * k.cap_ntr, k.hdr + 3 * k.cap_ntr};
    const float* hh[4] = {sx, sy, rx, ry};
    // 1. inputs in, once the slot's previous migration has read them
    if (k.used) e = cudaStreamWaitEvent(p->host_in, k.mig_done, 0);
    for (int a = 0; a < 4 && e == cudaSuccess && ntr > 0; ++a)
        if (hh[a]) e = cudaMemcpyAsync(dh[a], hh[a], hdr_bytes, cudaMemcpyHostToDevice, p->host_in);
    if (e == cudaSuccess && ntr > 0) e = cudaMemcpyAsync(k.traces, traces, tr_bytes, cudaMemcpyHostToDevice, p->host_in);
    if (e == cudaSuccess) e = cudaEventRecord(k.in_done, p->host_in);
    // 2. the migration, after its inputs and after the slot's previous image copy
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, k.in_done, 0);
    if (e == cudaSuccess && k.used) e = cudaStreamWaitEvent(s, k.out_done, 0);
    if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_migrate_host: host-to-device copies");
    st = kirchhoff_migrate(p, ntr, dh[0], sy ? dh[1] : nullptr, dh[2], ry ? dh[3] : nullptr, k.traces, k.image,
                           cuda_stream);
    if (st != KH_OK) return st;
    // 3. the image out, after the migration
    e = cudaEventRecord(k.mig_done, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->host_out, k.mig_done, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(image, k.image, img_bytes, cudaMemcpyDeviceToHost, p->host_out);
    if (e == cudaSuccess) e = cudaEventRecord(k.out_done, p->host_out);
    if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_migrate_host: device-to-host copy");
    k.used = true;
    p->host_next ^= 1;
    return KH_OK;
}

extern "C" kh_status kirchhoff_host_join(kh_plan p, void* cuda_stream)
{
    if (!p) return set_error(KH_ERR_INVALID_ARG, "plan is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    for (auto& k : p->host) {
        if (!k.used) continue;
        cudaError_t e = cudaStreamWaitEvent(s, k.out_done, 0);
        if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_host_join");
    }
    return KH_OK;
}
