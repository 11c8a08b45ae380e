// Batched persistent migration: many independent migrations (each with its own plan, headers,
// traces and image) in one launch of k_migrate_batched.
//
// kirchhoff_batched_prepare does everything that allocates, synchronises or reads back:
// validation, each job's geometry, tile and ln(1 + rho) fit, binning of its headers into the
// batch's own buffers, a per-(tile, bin) count of the traces that survive the aperture cull,
// and the work list of (job, tile, bin) items sorted by estimated cost, longest first.
// kirchhoff_migrate_batched then issues only stream work (row staging: FP32 rows as (sample,
// step) pairs, or 16-bit rows padded where they are not 16-byte aligned; a memset of the work
// counters; and the persistent kernel once per ln(1 + rho) fit length present in the batch),
// so a CUDA graph can capture and replay it.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <numeric>
#include <vector>

#include "kh_plan.h"
#include "kh_tau.cuh"

using namespace kh;

struct kh_batch_s {
    int device = 0;
    int njobs = 0;
    GeomParams g_max{};            // sizes the shared-memory ring (largest nt of the jobs)
    int vel = VK_CONST, weight = 0, fast = 1, tdtype = KH_F32;
    long long wait_polls = 0;
    unsigned char* ws = nullptr;   // one device allocation holding everything below
    BatchJob* d_jobs = nullptr;
    int4* d_items = nullptr;
    int* d_next = nullptr;         // work counters (one per part), zeroed before every run
    int* d_status = nullptr;       // bit 0: a bounded wait ran out
    int n_items = 0;
    int ctas = 0;
    // The sorted work list is cut into parts of one ln(1 + rho) fit length each (shortest
    // first); each part is one launch of the kernel compiled for that length.
    struct Part {
        int lg_terms, first, count, ctas;
    };
    std::vector<Part> parts;
    double work = 0.0;             // estimated contributions: culled traces x points, summed
    long long launches = 0;
    // Rows restaged at every launch: padded to 16-byte rows, or FP32 rows to SamplePair rows
    // (pairs: every job, when the jobs' plans stage pairs and the longest trace allows it).
    struct Pad {
        int ntr, nt;
        long long ld;
        int esize;
        const void* src;
        void* dst;
    };
    std::vector<Pad> pads;
    int pairs = 0;
    // KH_OPT_BATCH_MODE 1: each job's own k_migrate launch, descending cost, round-robin over
    // library streams forked from and joined to the caller's stream
    int mode = 0;
    std::vector<BatchJob> conc;            // jobs in launch order
    std::vector<int> conc_pad;             // index into pads, or -1
    static constexpr int N_STREAMS = 4;
    cudaStream_t st[N_STREAMS] = {};
    cudaEvent_t fork = nullptr, join[N_STREAMS] = {};
};

namespace {

kh_status bfail(kh_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return set_error(s, buf);
}

// Traces of bin `blockIdx.y` whose midpoint passes the producer's aperture cull for the
// column footprint of xy tile `blockIdx.x` (all z tiles share it).
__global__ void k_cull_count(GeomParams g, TileShape ts, const float2* __restrict__ mid,
                             const int* __restrict__ bin_start, int* __restrict__ out)
{
    __shared__ int total;
    const int txy = blockIdx.x, bin = blockIdx.y;
    const int txi = txy % ts.tiles_x, tyi = txy / ts.tiles_x;
    const TileBox box = tile_box(g, txi * ts.cx, tyi * ts.cy, 0, ts.cx, ts.cy, ts.cz * NZ);
    if (threadIdx.x == 0) total = 0;
    __syncthreads();
    int c = 0;
    for (int k = bin_start[bin] + threadIdx.x; k < bin_start[bin + 1]; k += blockDim.x) {
        bool ok = true;
        if (g.use_aperture) {
            const float2 m = mid[k];
            const float ax = fmaxf(fmaxf(box.xlo - m.x, m.x - box.xhi), 0.f);
            const float ay = fmaxf(fmaxf(box.ylo - m.y, m.y - box.yhi), 0.f);
            ok = ax * ax + ay * ay <= g.A2cull;
        }
        c += ok ? 1 : 0;
    }
    atomicAdd(&total, c);   // integer sum: order independent
    __syncthreads();
    if (threadIdx.x == 0) out[(size_t)bin * gridDim.x + txy] = total;
}

// Bump allocator over one device block (256-byte aligned pieces).
struct Layout {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    }
};

int dtype_bytes(kh_dtype t) { return t == KH_F32 ? 4 : 2; }

// Index of a per-leg fit length in LG_TERMS (constant and table jobs fall in the last class).
int lg_class(int terms)
{
    for (int i = 0; i < N_LG_TERMS; ++i)
        if (LG_TERMS[i] == terms) return i;
    return N_LG_TERMS - 1;
}

}  // namespace

extern "C" {

kh_status kirchhoff_batched_prepare(int njobs, const kh_job* jobs, kh_batch* out, void* cuda_stream)
{
    if (!out) return bfail(KH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (njobs < 1 || !jobs) return bfail(KH_ERR_INVALID_ARG, "need njobs >= 1 and a job array");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");

    // ---- validation and per-job geometry
    std::vector<GeomParams> gs(njobs);
    std::vector<TileShape> tss(njobs);
    int vel = -1, weight = -1, fast = -1, tdt = -1, nt_max = 0;
    for (int j = 0; j < njobs; ++j) {
        const kh_job& J = jobs[j];
        const kh_plan_s* p = J.plan;
        if (!p) return bfail(KH_ERR_INVALID_ARG, "job %d: plan is NULL", j);
        if (p->device != dev) return bfail(KH_ERR_INVALID_ARG, "job %d: plan belongs to device %d, current is %d",
                                           j, p->device, dev);
        kh_status st = plan_check_headers(p, J.ntr, J.sx, J.sy, J.rx, J.ry);
        if (st != KH_OK) return st;
        if (!J.image) return bfail(KH_ERR_INVALID_ARG, "job %d: image is NULL", j);
        if (J.ntr > 0 && !J.traces) return bfail(KH_ERR_INVALID_ARG, "job %d: traces is NULL", j);
        if (p->d.weight == KH_W_TRUE_AMP)
            return bfail(KH_ERR_UNSUPPORTED, "job %d: the batched launch takes W = 1 or the obliquity weight", j);
        if (p->d.aa_spacing > 0.0)
            return bfail(KH_ERR_UNSUPPORTED, "job %d: the batched launch has no operator anti-aliasing", j);
        if (p->d.vel == KH_VEL_TABLE || p->d.vel == KH_VEL_PSTM || p->d.vel == KH_VEL_GRID)
            return bfail(KH_ERR_UNSUPPORTED, "job %d: the batched launch takes analytic depth traveltimes "
                                             "(KH_VEL_CONST / KH_VEL_LINEAR_Z)", j);
        if ((st = plan_geometry(p, &gs[j], &tss[j])) != KH_OK) return st;
        if (tss[j].cz > 16 || tss[j].cx * tss[j].cy * tss[j].cz != CONSUMERS)
            return bfail(KH_ERR_INTERNAL, "job %d: tile %dx%dx%d is not a 256-thread tile with cz <= 16", j,
                         tss[j].cx, tss[j].cy, tss[j].cz);
        const int vk = gs[j].k == 0.0 ? VK_CONST : VK_LINEAR;
        if (j == 0) {
            vel = vk;
            weight = (int)p->d.weight;
            fast = p->fast_math ? 1 : 0;
            tdt = (int)p->d.trace_dtype;
        } else if (vk != vel || (int)p->d.weight != weight || (p->fast_math ? 1 : 0) != fast ||
                   (int)p->d.trace_dtype != tdt) {
            return bfail(KH_ERR_UNSUPPORTED, "job %d: all jobs of a batch need the same velocity kind "
                                             "(constant or linear), weight, fast-math option and trace dtype", j);
        }
        nt_max = std::max(nt_max, p->d.nt);
    }

    // ---- device layout
    const bool pairs = jobs[0].plan->sample_pairs && tdt == KH_F32 && nt_max <= PAIR_MAX_NT;
    const int es = pairs ? (int)sizeof(SamplePair) : dtype_bytes((kh_dtype)tdt), ealign = 16 / es;
    Layout L;
    struct Off {
        size_t bin, perm, bs, hdr, mid, pad, cull, key2, perm2, hist, cs;
        long long ld;
        bool padded;
    };
    std::vector<Off> off(njobs);
    std::vector<CellGrid> cgs(njobs);
    size_t n_items = 0, n_cull = 0;
    for (int j = 0; j < njobs; ++j) {
        const kh_job& J = jobs[j];
        const kh_desc& d = J.plan->d;
        const size_t n = (size_t)std::max(J.ntr, 1);
        Off& o = off[j];
        o.bin = L.take(n * sizeof(int));
        o.perm = L.take(n * sizeof(int));
        o.bs = L.take((size_t)(d.n_bins + 1) * sizeof(int));
        // the plan path's binning sort (same trace order, so bit-identical images)
        cgs[j] = cell_grid_of(d, J.plan->spatial_sort != 0);
        o.key2 = L.take(n * sizeof(int));
        o.perm2 = L.take(n * sizeof(int));
        o.hist = L.take((size_t)std::max(sort_hist_entries(J.ntr), 1) * sizeof(int));
        o.cs = L.take(((size_t)d.n_bins * cgs[j].ncx * cgs[j].ncy + 1) * sizeof(int));
        o.hdr = L.take(n * sizeof(float4));
        o.mid = L.take(n * sizeof(float2));
        o.padded = J.ntr > 0 && (pairs || !((reinterpret_cast<uintptr_t>(J.traces) & 15u) == 0 && d.nt % ealign == 0));
        o.ld = o.padded ? (d.nt + ealign - 1) / ealign * ealign : d.nt;
        o.pad = o.padded ? L.take((size_t)J.ntr * o.ld * es) : 0;
        const TileShape& t = tss[j];
        n_items += (size_t)t.tiles_x * t.tiles_y * t.tiles_z * d.n_bins;
        n_cull += (size_t)t.tiles_x * t.tiles_y * d.n_bins;
    }
    if (n_items > (size_t)INT32_MAX) return bfail(KH_ERR_UNSUPPORTED, "more than 2^31 work items");
    const size_t o_jobs = L.take(sizeof(BatchJob) * njobs);
    const size_t o_items = L.take(sizeof(int4) * n_items);
    const size_t o_next = L.take(N_LG_TERMS * sizeof(int));
    const size_t o_status = L.take(sizeof(int));
    const size_t o_cull = L.take(sizeof(int) * std::max<size_t>(n_cull, 1));

    kh_batch_s* b = new kh_batch_s();
    b->device = dev;
    b->njobs = njobs;
    b->vel = vel;
    b->weight = weight;
    b->fast = fast;
    b->tdtype = tdt;
    b->wait_polls = jobs[0].plan->wait_polls;
    b->mode = jobs[0].plan->batch_mode;
    b->n_items = (int)n_items;
    b->pairs = pairs ? 1 : 0;
    e = cudaMalloc(&b->ws, L.off);
    if (e != cudaSuccess) {
        delete b;
        return set_cuda_error(e, "kirchhoff_batched_prepare: workspace");
    }
    auto fail_free = [&](kh_status st) {
        cudaFree(b->ws);
        delete b;
        return st;
    };
    unsigned char* w = b->ws;
    b->d_jobs = reinterpret_cast<BatchJob*>(w + o_jobs);
    b->d_items = reinterpret_cast<int4*>(w + o_items);
    b->d_next = reinterpret_cast<int*>(w + o_next);
    b->d_status = reinterpret_cast<int*>(w + o_status);
    int* d_cull = reinterpret_cast<int*>(w + o_cull);
    if ((e = cudaMemsetAsync(b->d_status, 0, sizeof(int), s)) != cudaSuccess)
        return fail_free(set_cuda_error(e, "kirchhoff_batched_prepare: memset"));

    // ---- per job: binning, staged rows, cull counts
    std::vector<BatchJob> hj(njobs);
    std::vector<int> pad_of(njobs, -1);
    std::vector<size_t> cull_at(njobs);
    size_t cull_off = 0;
    for (int j = 0; j < njobs; ++j) {
        const kh_job& J = jobs[j];
        const kh_desc& d = J.plan->d;
        const Off& o = off[j];
        GeomParams g = gs[j];
        g.ld = o.ld;
        if (pairs) {
            g.pairs = 1;
            g.esize = es;
            g.elem_align = ealign;
        }
        float4* hdr = reinterpret_cast<float4*>(w + o.hdr);
        float2* mid = reinterpret_cast<float2*>(w + o.mid);
        int* bs = reinterpret_cast<int*>(w + o.bs);
        int* cs = reinterpret_cast<int*>(w + o.cs);
        const int* perm = nullptr;
        int nl = 0;
        e = sort_traces(J.ntr, J.sx, J.sy, J.rx, J.ry, d.dim, d.n_bins, d.bin_width, cgs[j],
                        reinterpret_cast<int*>(w + o.bin), reinterpret_cast<int*>(w + o.key2),
                        reinterpret_cast<int*>(w + o.perm), reinterpret_cast<int*>(w + o.perm2),
                        reinterpret_cast<int*>(w + o.hist), cs, bs, &perm, &nl, s);
        if (e == cudaSuccess) e = launch_gather(J.ntr, bs, d.n_bins, perm, J.sx, J.sy, J.rx, J.ry, d.dim, hdr, mid, s);
        if (e != cudaSuccess) return fail_free(set_cuda_error(e, "kirchhoff_batched_prepare: binning"));
        TraceSet tr{hdr, mid, perm, bs};
        if (cgs[j].ncx * cgs[j].ncy > 1) tr.cell_start = cs;
        tr.cg = cgs[j];
        const void* rows = J.traces;
        if (o.padded) {
            rows = w + o.pad;
            pad_of[j] = (int)b->pads.size();
            b->pads.push_back({J.ntr, d.nt, o.ld, es, J.traces, w + o.pad});
        }
        hj[j] = BatchJob{g, tss[j], tr, rows, J.image};
        cull_at[j] = cull_off;
        const TileShape& t = tss[j];
        dim3 grid((unsigned)(t.tiles_x * t.tiles_y), (unsigned)d.n_bins);
        k_cull_count<<<grid, 256, 0, s>>>(g, t, tr.mid, tr.bin_start, d_cull + cull_off);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return fail_free(set_cuda_error(e, "kirchhoff_batched_prepare: cull count"));
        cull_off += (size_t)t.tiles_x * t.tiles_y * d.n_bins;
    }
    std::vector<int> cull(std::max<size_t>(n_cull, 1));
    e = cudaMemcpyAsync(cull.data(), d_cull, sizeof(int) * n_cull, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_free(set_cuda_error(e, "kirchhoff_batched_prepare: cull read-back"));

    // ---- work list: (job, tile, bin), estimated cost = points x (culled traces + 4).  Order:
    // fit-length group (shortest first), then jobs by descending total cost, then bins, then
    // longest item first.  Keeping a job's bin together keeps that bin's trace windows in L2
    // while all CTAs work on it (as a per-job launch does); the smallest jobs form the tail.
    std::vector<int4> items(n_items);
    std::vector<double> cost(n_items);
    std::vector<int> cls(n_items);
    std::vector<double> job_cost(njobs, 0.0);
    size_t k = 0;
    double work = 0.0;
    for (int j = 0; j < njobs; ++j) {
        const kh_desc& d = jobs[j].plan->d;
        const TileShape& t = tss[j];
        const int ntxy = t.tiles_x * t.tiles_y;
        for (int tyi = 0; tyi < t.tiles_y; ++tyi)
            for (int txi = 0; txi < t.tiles_x; ++txi) {
                const int cols = std::min(t.cx, d.nx - txi * t.cx) * std::min(t.cy, d.ny - tyi * t.cy);
                for (int tzi = 0; tzi < t.tiles_z; ++tzi) {
                    const int zs = std::min(t.cz * NZ, d.nz - tzi * t.cz * NZ);
                    const int tile = (tyi * t.tiles_x + txi) * t.tiles_z + tzi;
                    for (int bin = 0; bin < d.n_bins; ++bin) {
                        const int c = cull[cull_at[j] + (size_t)bin * ntxy + tyi * t.tiles_x + txi];
                        items[k] = make_int4(j, tile, bin, 0);
                        cls[k] = lg_class(gs[j].lg_terms);
                        cost[k] = (double)cols * zs * (c + 4);
                        job_cost[j] += cost[k];
                        work += (double)cols * zs * c;
                        ++k;
                    }
                }
            }
    }
    std::vector<int> order(n_items);
    std::iota(order.begin(), order.end(), 0);
    std::vector<int> job_rank(njobs);
    {
        std::vector<int> jo(njobs);
        std::iota(jo.begin(), jo.end(), 0);
        std::stable_sort(jo.begin(), jo.end(), [&](int a, int c) { return job_cost[a] > job_cost[c]; });
        for (int r = 0; r < njobs; ++r) job_rank[jo[r]] = r;
    }
    if (b->mode == 1) {   // concurrent per-job kernels: jobs by descending cost
        std::vector<int> jo(njobs);
        std::iota(jo.begin(), jo.end(), 0);
        std::stable_sort(jo.begin(), jo.end(), [&](int a, int c) { return job_cost[a] > job_cost[c]; });
        for (int j : jo) {
            b->conc.push_back(hj[j]);
            b->conc_pad.push_back(pad_of[j]);
        }
        b->work = work;
        e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (int k = 0; e == cudaSuccess && k < kh_batch_s::N_STREAMS; ++k) {
            e = cudaStreamCreateWithFlags(&b->st[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            kirchhoff_batch_destroy(b);
            return set_cuda_error(e, "kirchhoff_batched_prepare: streams");
        }
        b->ctas = 0;
        *out = b;
        return KH_OK;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        if (cls[a] != cls[c]) return cls[a] < cls[c];
        const int ja = job_rank[items[a].x], jc = job_rank[items[c].x];
        if (ja != jc) return ja < jc;
        if (items[a].z != items[c].z) return items[a].z < items[c].z;
        return cost[a] > cost[c];
    });
    std::vector<int4> sorted(n_items);
    for (size_t i = 0; i < n_items; ++i) sorted[i] = items[order[i]];
    b->work = work;

    e = cudaMemcpyAsync(b->d_jobs, hj.data(), sizeof(BatchJob) * njobs, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n_items)
        e = cudaMemcpyAsync(b->d_items, sorted.data(), sizeof(int4) * n_items, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host vectors go out of scope
    if (e != cudaSuccess) return fail_free(set_cuda_error(e, "kirchhoff_batched_prepare: upload"));

    GeomParams gm = gs[0];
    gm.nt = nt_max;
    gm.esize = es;
    gm.elem_align = ealign;
    gm.pairs = pairs ? 1 : 0;
    gm.table = nullptr;
    b->g_max = gm;
    WaitCfg wc{b->d_status, b->wait_polls, WAIT_NS};
    for (int c = 0, first = 0; c < N_LG_TERMS; ++c) {
        int count = 0;
        for (size_t i = 0; i < n_items; ++i) count += cls[i] == c ? 1 : 0;
        if (count == 0) continue;
        kh_batch_s::Part part{LG_TERMS[c], first, count, 0};
        e = launch_migrate_batched(gm, b->d_jobs, b->d_items + first, count, b->d_next + b->parts.size(), vel,
                                   weight, fast, part.lg_terms, tdt, wc, 0, &part.ctas, s);
        if (e != cudaSuccess) return fail_free(set_cuda_error(e, "kirchhoff_batched_prepare: kernel set-up"));
        b->ctas = std::max(b->ctas, part.ctas);
        b->parts.push_back(part);
        first += count;
    }
    *out = b;
    return KH_OK;
}

kh_status kirchhoff_migrate_batched(kh_batch b, void* cuda_stream)
{
    if (!b) return bfail(KH_ERR_INVALID_ARG, "batch is NULL");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
    if (dev != b->device) return bfail(KH_ERR_INVALID_ARG, "batch belongs to device %d, current is %d", b->device, dev);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (b->mode == 1) {
        WaitCfg wc{b->d_status, b->wait_polls, WAIT_NS};
        if ((e = cudaEventRecord(b->fork, s)) != cudaSuccess) return set_cuda_error(e, "kirchhoff_migrate_batched: fork");
        for (int k = 0; k < kh_batch_s::N_STREAMS; ++k)
            if ((e = cudaStreamWaitEvent(b->st[k], b->fork, 0)) != cudaSuccess)
                return set_cuda_error(e, "kirchhoff_migrate_batched: fork");
        for (size_t i = 0; i < b->conc.size(); ++i) {
            cudaStream_t sk = b->st[i % kh_batch_s::N_STREAMS];
            const BatchJob& J = b->conc[i];
            if (b->conc_pad[i] >= 0) {
                const auto& p = b->pads[b->conc_pad[i]];
                e = b->pairs ? launch_pairs(p.ntr, p.nt, (int)p.ld, p.src, p.dst, sk)
                             : launch_pad(p.ntr, p.nt, p.ld, p.esize, p.src, p.dst, sk);
                if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_migrate_batched: row staging");
                ++b->launches;
            }
            e = launch_migrate(J.g, J.ts, J.tr, J.traces, J.image, b->vel, b->fast, wc, sk);
            ++b->launches;
            if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_migrate_batched: migration kernel");
        }
        for (int k = 0; k < kh_batch_s::N_STREAMS; ++k) {
            if ((e = cudaEventRecord(b->join[k], b->st[k])) != cudaSuccess ||
                (e = cudaStreamWaitEvent(s, b->join[k], 0)) != cudaSuccess)
                return set_cuda_error(e, "kirchhoff_migrate_batched: join");
        }
        return KH_OK;
    }
    for (const auto& p : b->pads) {
        e = b->pairs ? launch_pairs(p.ntr, p.nt, (int)p.ld, p.src, p.dst, s)
                     : launch_pad(p.ntr, p.nt, p.ld, p.esize, p.src, p.dst, s);
        if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_migrate_batched: row staging");
        ++b->launches;
    }
    if (b->n_items == 0) return KH_OK;
    if ((e = cudaMemsetAsync(b->d_next, 0, N_LG_TERMS * sizeof(int), s)) != cudaSuccess)
        return set_cuda_error(e, "kirchhoff_migrate_batched: counter reset");
    WaitCfg wc{b->d_status, b->wait_polls, WAIT_NS};
    for (size_t i = 0; i < b->parts.size(); ++i) {
        const kh_batch_s::Part& part = b->parts[i];
        e = launch_migrate_batched(b->g_max, b->d_jobs, b->d_items + part.first, part.count, b->d_next + i, b->vel,
                                   b->weight, b->fast, part.lg_terms, b->tdtype, wc, part.ctas, nullptr, s);
        ++b->launches;
        if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_migrate_batched: persistent kernel");
    }
    return KH_OK;
}

kh_status kirchhoff_batch_sync(kh_batch b, void* cuda_stream)
{
    if (!b) return bfail(KH_ERR_INVALID_ARG, "batch is NULL");
    int h = 0;
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
    if (e == cudaSuccess) e = cudaMemcpy(&h, b->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_batch_sync");
    if (h != 0) {
        cudaMemset(b->d_status, 0, sizeof(int));
        return bfail(KH_ERR_TIMEOUT, "a bounded in-kernel wait ran out (status 0x%x); results are invalid", h);
    }
    return KH_OK;
}

kh_status kirchhoff_batch_info(kh_batch b, long long* n_items, int* n_ctas, double* est_contributions,
                               long long* launches)
{
    if (!b) return bfail(KH_ERR_INVALID_ARG, "batch is NULL");
    if (n_items) *n_items = b->n_items;
    if (n_ctas) *n_ctas = b->ctas;
    if (est_contributions) *est_contributions = b->work;
    if (launches) *launches = b->launches;
    return KH_OK;
}

kh_status kirchhoff_batch_destroy(kh_batch b)
{
    if (!b) return KH_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    for (int k = 0; k < kh_batch_s::N_STREAMS; ++k) {
        if (b->st[k]) cudaStreamDestroy(b->st[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    cudaFree(b->ws);
    if (prev != b->device) cudaSetDevice(prev);
    delete b;
    return KH_OK;
}

}  // extern "C"
