// Migration kernel (Eq. 1, Sec. 3): output-stationary gather over an image tile and one
// offset bin.
//
// CTA = 8 consumer warps + 1 producer warp.  Each consumer thread owns NZ = 16 consecutive
// z samples of one image column and keeps their FP32 accumulators in registers for the
// whole kernel; nothing is accumulated in global memory.  The producer warp walks the
// bin's traces (sorted by bin), culls those whose midpoint is outside the aperture of the
// tile footprint, bounds the two-way time over the tile box to a sample window, and stages
// each window into a 3-deep shared-memory ring with one cp.async.bulk per trace (16-byte
// aligned, no multicast) completing on the stage's mbarrier.  Consumers read the staged
// samples at tau = (T_s + T_r - t0)/dt, interpolate linearly, weight and accumulate.
// All mbarrier waits are bounded; a wait that runs out sets the plan's status word.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kh_device.cuh"

namespace kh {

template <typename TT>
__device__ __forceinline__ float to_f32(TT v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

struct __align__(16) MigSmem {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    int cnt[STAGES];
    int last[STAGES];
    float4 hdr[STAGES][BMAX];   // sx, sy, rx, ry
    float2 mid[STAGES][BMAX];   // FP32 midpoint
    int4 win[STAGES][BMAX];     // cb = -MAGIC_BITS - lo, sb = smem index of sample lo, lim = hi - lo
    float zero[4];
};

__host__ __device__ constexpr size_t mig_static_bytes() { return (sizeof(MigSmem) + 127) / 128 * 128; }

// Elements of one stage's sample area: a full trace always fits, so every trace is stageable.
__host__ __device__ inline int mig_cap(int nt, int ealign)
{
    const int need = (nt + 2 * ealign + ealign - 1) / ealign * ealign;
    const int base = 24576 / 4;   // 24 KB of FP32 (48 KB worth of 16-bit samples is the same count)
    return need > base ? need : base;
}

size_t migrate_smem_bytes(const GeomParams& g)
{
    return mig_static_bytes() + (size_t)STAGES * mig_cap(g.nt, g.elem_align) * g.esize;
}

// Smallest and largest one-way time from a surface point at horizontal distance [hmin, hmax]
// from the tile footprint to any depth in [zlo, zhi].  T grows with h at fixed z; at fixed h,
// q(z) = (h^2 + z^2)/(v0 (v0 + k z)) has its only interior stationary point (a minimum) at
// z* = k h^2 / (v0 + sqrt(v0^2 + k^2 h^2)).
__device__ __forceinline__ void leg_bounds(float hmin, float hmax, float zlo, float zhi, int vel,
                                           float v0, float k, float& tmin, float& tmax)
{
    const float kk = (vel == VK_CONST) ? 0.f : k;
    float zs = kk * hmin * hmin / (v0 + sqrtf(v0 * v0 + kk * kk * hmin * hmin));
    zs = fminf(fmaxf(zs, zlo), zhi);
    tmin = fminf(fminf(tt_bound(hmin, zlo, vel, v0, kk), tt_bound(hmin, zhi, vel, v0, kk)),
                 tt_bound(hmin, zs, vel, v0, kk));
    tmax = fmaxf(tt_bound(hmax, zlo, vel, v0, kk), tt_bound(hmax, zhi, vel, v0, kk));
}

__device__ __forceinline__ void rect_dist(float px, float py, float xlo, float xhi, float ylo,
                                          float yhi, float& dmin, float& dmax)
{
    const float ax = fmaxf(fmaxf(xlo - px, px - xhi), 0.f);
    const float ay = fmaxf(fmaxf(ylo - py, py - yhi), 0.f);
    dmin = sqrtf(ax * ax + ay * ay);
    const float bx = fmaxf(fabsf(px - xlo), fabsf(px - xhi));
    const float by = fmaxf(fabsf(py - ylo), fabsf(py - yhi));
    dmax = sqrtf(bx * bx + by * by);
}

// ------------------------------------------------------------------ producer warp
template <typename TT>
__device__ void mig_producer(MigSmem& S, TT* data, int cap, const GeomParams& g,
                             const TraceSet& tr, const TT* __restrict__ traces, int tb, int te,
                             float xlo, float xhi, float ylo, float yhi, float zlo, float zhi,
                             int vel, const WaitCfg& wc)
{
    const int lane = threadIdx.x & 31;
    const float v0 = (float)g.v0, kf = (float)g.k;
    const float inv_dt = 1.f / g.dt;
    int cur = tb;
    int n = 0;
    bool failed = false;
    while (true) {
        const int s = n % STAGES;
        if (n >= STAGES) {
            if (!warp_wait(&S.empty[s], ((n / STAGES) - 1) & 1, wc.polls, wc.ns, wc.status)) {
                failed = true;
                break;
            }
        }
        int cnt = 0, used = 0;
        bool full = false;
        while (cur < te && !full) {
            const int k = cur + lane;
            bool ok = false;
            int lo = 0, hi = 0, lo_al = 0, len_al = 0;
            float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 m = make_float2(0.f, 0.f);
            if (k < te) {
                h = tr.hdr[k];
                m = tr.mid[k];
                ok = true;
                if (g.use_aperture) {
                    const float ax = fmaxf(fmaxf(xlo - m.x, m.x - xhi), 0.f);
                    const float ay = fmaxf(fmaxf(ylo - m.y, m.y - yhi), 0.f);
                    ok = ax * ax + ay * ay <= g.A2cull;
                }
                if (ok) {
                    float hs0, hs1, hr0, hr1, ts0, ts1, tr0, tr1;
                    rect_dist(h.x, h.y, xlo, xhi, ylo, yhi, hs0, hs1);
                    rect_dist(h.z, h.w, xlo, xhi, ylo, yhi, hr0, hr1);
                    leg_bounds(hs0, hs1, zlo, zhi, vel, v0, kf, ts0, ts1);
                    leg_bounds(hr0, hr1, zlo, zhi, vel, v0, kf, tr0, tr1);
                    const float tlo = (ts0 + tr0 - g.t0) * inv_dt;
                    const float thi = (ts1 + tr1 - g.t0) * inv_dt;
                    const float slo = 2.f + 2e-4f * fabsf(tlo), shi = 2.f + 2e-4f * fabsf(thi);
                    const float flo = floorf(tlo - slo), fhi = ceilf(thi + shi) + 1.f;
                    if (!(fhi >= 1.f && flo <= (float)(g.nt - 2))) {
                        ok = false;   // no sample of this trace can reach the tile (also NaN)
                    } else {
                        lo = flo < 0.f ? 0 : (int)flo;
                        hi = fhi > (float)(g.nt - 1) ? g.nt - 1 : (int)fhi;
                        ok = hi > lo;
                        lo_al = lo & ~(g.elem_align - 1);
                        len_al = (hi + 1 - lo_al + g.elem_align - 1) & ~(g.elem_align - 1);
                    }
                }
            }
            const unsigned okm = __ballot_sync(0xffffffffu, ok);
            // exclusive prefix of window lengths over accepted lanes
            int pre = ok ? len_al : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, pre, o);
                if (lane >= o) pre += v;
            }
            const int excl = pre - (ok ? len_al : 0);
            const int rank = __popc(okm & ((1u << lane) - 1u));
            const bool fits = ok && (cnt + rank < BMAX) && (used + excl + len_al <= cap);
            const unsigned fm = __ballot_sync(0xffffffffu, fits);
            const unsigned nofit = okm & ~fm;
            const int consumed = nofit ? (__ffs(nofit) - 1) : min(32, te - cur);
            const int nfit = __popc(fm);
            // bytes staged by the fitting lanes
            int bytes = fits ? len_al * g.esize : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
            int used_add = fits ? len_al : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) used_add += __shfl_xor_sync(0xffffffffu, used_add, o);
            if (fits) {
                const int slot = cnt + rank;
                const int dst = s * cap + used + excl;
                S.hdr[s][slot] = h;
                S.mid[s][slot] = m;
                S.win[s][slot] = make_int4(-MAGIC_BITS - lo, dst + (lo - lo_al), hi - lo, 0);
            }
            if (lane == 0 && bytes > 0) mbar_expect_tx(&S.full[s], (uint32_t)bytes);
            __syncwarp();
            if (fits) {
                const int j = tr.perm[k];
                const TT* src = traces + (long long)j * g.ld + lo_al;
                bulk_g2s(data + s * cap + used + excl, src, (uint32_t)(len_al * g.esize), &S.full[s]);
            }
            cnt += nfit;
            used += used_add;
            cur += consumed;
            full = (nofit != 0u) || cnt >= BMAX;
        }
        __syncwarp();
        if (lane == 0) {
            S.cnt[s] = cnt;
            S.last[s] = (cur >= te) ? 1 : 0;
            mbar_arrive(&S.full[s]);
        }
        __syncwarp();
        ++n;
        if (cur >= te) break;
    }
    if (failed) {
        if (lane == 0) atomicOr(wc.status, 1);
        // let every copy already issued land before the CTA can exit
        const int first = n > STAGES ? n - STAGES : 0;
        for (int f = first; f < n; ++f)
            mbar_wait_bounded(&S.full[f % STAGES], (f / STAGES) & 1, 0, WAIT_NS, nullptr);
    }
}

// ------------------------------------------------------------------ consumer warps
template <int VEL, int WGT, bool FAST>
__device__ __forceinline__ float tau_half(float dhs2, float dhr2, float z2, float a, float az2,
                                          float b, float wz, const GeomParams& g, float& W)
{
    // returns tau - 1/2; W is the weight of this contribution
    if constexpr (VEL == VK_CONST) {
        const float Rs = hsqrt<FAST>(dhs2 + z2);
        const float Rr = hsqrt<FAST>(dhr2 + z2);
        const float S = Rs + Rr;
        if constexpr (WGT == 1) W = wz * S; else W = 1.f;
        return fmaf(S, g.C1, g.C0h);
    } else {
        float xs, xr;
        if constexpr (WGT == 1) {
            const float Rs = hsqrt<FAST>(dhs2 + z2);
            const float Rr = hsqrt<FAST>(dhr2 + z2);
            const float ss = b * Rs, sr = b * Rr;            // sqrt(q)
            const float qs = ss * ss, qr = sr * sr;
            xs = fmaf(ss, hsqrt<FAST>(qs + 2.f), qs);       // e^{|k| T} - 1
            xr = fmaf(sr, hsqrt<FAST>(qr + 2.f), qr);
            W = wz * (Rs + Rr);
        } else {
            const float qs = fmaf(dhs2, a, az2), qr = fmaf(dhr2, a, az2);
            xs = qs + hsqrt<FAST>(qs * (qs + 2.f));
            xr = qr + hsqrt<FAST>(qr * (qr + 2.f));
            W = 1.f;
        }
        const float y = fmaf(xs, xr, xs + xr);              // (1+xs)(1+xr) - 1
        const float L = hlog2<FAST>(1.f + y);               // |k| (T_s + T_r) / ln 2
        return fmaf(L, g.C1, g.C0h);
    }
}

template <int VEL, int WGT, bool FAST, typename TT>
__device__ void mig_consumer(MigSmem& S, const TT* data, const GeomParams& g, const TileShape& ts,
                             int x0, int y0, int z0, int bin, float* __restrict__ image,
                             const WaitCfg& wc)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tid % ts.cx, ty = (tid / ts.cx) % ts.cy, tzg = tid / (ts.cx * ts.cy);
    const int ix = x0 + tx, iy = y0 + ty, izb = z0 + tzg * NZ;
    const bool col_ok = ix < g.nx && iy < g.ny;
    const float cxf = col_coord(g.ox, ix, g.dx);
    const float cyf = (g.dim == 3) ? col_coord(g.oy, iy, g.dy) : 0.f;

    float z2[NZ], ca[NZ], cb[NZ], wz[NZ], acc[NZ];
#pragma unroll
    for (int i = 0; i < NZ; ++i) {
        const double zd = __dadd_rn(g.oz, __dmul_rn((double)(izb + i), g.dz));
        z2[i] = (float)(zd * zd);
        const double vz = g.v0 + g.k * zd;
        const double alpha = (VEL == VK_LINEAR) ? g.kabs * g.kabs / (2.0 * g.v0 * vz) : 0.0;
        ca[i] = (float)alpha;                               // q = a R^2
        cb[i] = (float)((WGT == 1) ? sqrt(fmax(alpha, 0.0)) : alpha * zd * zd);
        wz[i] = (WGT == 1 && fabs(zd) >= 1e-6 * fabs(g.dz)) ? (float)(zd * g.wscale) : 0.f;
        acc[i] = 0.f;
    }
    const int zero_off = (int)(((const char*)S.zero - (const char*)data) / (int)sizeof(TT));

    bool failed = false;
    int n = 0;
    while (true) {
        const int s = n % STAGES;
        if (!warp_wait(&S.full[s], (n / STAGES) & 1, wc.polls, wc.ns, wc.status)) {
            failed = true;
            break;
        }
        const int cnt = S.cnt[s];
        const int last = S.last[s];
        for (int t = 0; t < cnt; ++t) {
            const float4 h = S.hdr[s][t];
            const int4 w = S.win[s][t];
            unsigned lim = col_ok ? (unsigned)w.z : 0u;
            if (g.use_aperture) {
                const float2 m = S.mid[s][t];
                if (!in_aperture(cxf, cyf, m.x, m.y, g.A2)) lim = 0u;
            }
            if (!__any_sync(0xffffffffu, lim != 0u)) continue;
            const float dxs = cxf - h.x, dys = cyf - h.y;
            const float dxr = cxf - h.z, dyr = cyf - h.w;
            const float dhs2 = fmaf(dxs, dxs, dys * dys);
            const float dhr2 = fmaf(dxr, dxr, dyr * dyr);
#pragma unroll
            for (int i = 0; i < NZ; ++i) {
                float W;
                const float th = tau_half<VEL, WGT, FAST>(dhs2, dhr2, z2[i], ca[i], cb[i], cb[i],
                                                          wz[i], g, W);
                const float tm = __fadd_rn(th, MAGIC);
                const float r = __fadd_rn(tm, -MAGIC);
                const float f = __fadd_rn(__fadd_rn(th, -r), 0.5f);
                const int idx = __float_as_int(tm) + w.x;   // i - lo
                const int off = ((unsigned)idx < lim) ? idx + w.y : zero_off;
                const float d0 = to_f32<TT>(data[off]);
                const float d1 = to_f32<TT>(data[off + 1]);
                const float val = fmaf(f, d1 - d0, d0);
                if constexpr (WGT == 1) acc[i] = fmaf(W, val, acc[i]);
                else acc[i] += val;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[s]);
        ++n;
        if (last) break;
    }
    (void)warp;
    if (failed) {
        if (lane == 0) atomicOr(wc.status, 1);
        return;
    }
    if (!col_ok) return;
    float* out = image + (((long long)bin * g.ny + iy) * g.nx + ix) * (long long)g.nz + izb;
    const bool vec = ((g.nz & 3) == 0) && (izb + NZ <= g.nz) &&
                     ((reinterpret_cast<uintptr_t>(image) & 15) == 0);
    if (vec) {
#pragma unroll
        for (int i = 0; i < NZ; i += 4)
            *reinterpret_cast<float4*>(out + i) = make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < NZ; ++i)
            if (izb + i < g.nz) out[i] = acc[i];
    }
}

template <int VEL, int WGT, bool FAST, typename TT>
__global__ void __launch_bounds__(THREADS, 2)
    k_migrate(GeomParams g, TileShape ts, TraceSet tr, const TT* __restrict__ traces,
              float* __restrict__ image, int cap, WaitCfg wc)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MigSmem& S = *reinterpret_cast<MigSmem*>(smem_raw);
    TT* data = reinterpret_cast<TT*>(smem_raw + mig_static_bytes());
    const int bin = blockIdx.y;
    int t = blockIdx.x;
    const int tzi = t % ts.tiles_z;
    t /= ts.tiles_z;
    const int txi = t % ts.tiles_x, tyi = t / ts.tiles_x;
    const int x0 = txi * ts.cx, y0 = tyi * ts.cy, z0 = tzi * ts.cz * NZ;

    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        // a wait in another CTA of this plan already ran out: results are invalid anyway
        s_abort = *reinterpret_cast<const volatile int*>(wc.status);
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], CONSUMER_WARPS);
        }
        S.zero[0] = S.zero[1] = S.zero[2] = S.zero[3] = 0.f;
        fence_barrier_init();
    }
    __syncthreads();
    if (s_abort) return;
    if (threadIdx.x >= CONSUMERS) {
        const int xe = min(x0 + ts.cx, g.nx) - 1, ye = min(y0 + ts.cy, g.ny) - 1;
        const int ze = min(z0 + ts.cz * NZ, g.nz) - 1;
        const float xlo = col_coord(g.ox, x0, g.dx), xhi = col_coord(g.ox, xe, g.dx);
        const float ylo = g.dim == 3 ? col_coord(g.oy, y0, g.dy) : 0.f;
        const float yhi = g.dim == 3 ? col_coord(g.oy, ye, g.dy) : 0.f;
        const float zlo = (float)(g.oz + z0 * g.dz), zhi = (float)(g.oz + ze * g.dz);
        mig_producer<TT>(S, data, cap, g, tr, traces, tr.bin_start[bin], tr.bin_start[bin + 1],
                         fminf(xlo, xhi), fmaxf(xlo, xhi), fminf(ylo, yhi), fmaxf(ylo, yhi),
                         fminf(zlo, zhi), fmaxf(zlo, zhi), VEL, wc);
    } else {
        mig_consumer<VEL, WGT, FAST, TT>(S, data, g, ts, x0, y0, z0, bin, image, wc);
    }
}

template <int VEL, int WGT, bool FAST, typename TT>
static cudaError_t launch_t(const GeomParams& g, const TileShape& t, const TraceSet& tr,
                            const void* traces, float* image, const WaitCfg& w, cudaStream_t s)
{
    auto kern = k_migrate<VEL, WGT, FAST, TT>;
    const size_t smem = migrate_smem_bytes(g);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(t.tiles_x * t.tiles_y * t.tiles_z), (unsigned)g.n_bins);
    kern<<<grid, THREADS, smem, s>>>(g, t, tr, static_cast<const TT*>(traces), image,
                                     mig_cap(g.nt, g.elem_align), w);
    return cudaGetLastError();
}

template <typename TT>
static cudaError_t launch_dtype(const GeomParams& g, const TileShape& t, const TraceSet& tr,
                                const void* traces, float* image, int vel, int fast,
                                const WaitCfg& w, cudaStream_t s)
{
    const int key = vel * 4 + g.weight * 2 + (fast ? 1 : 0);
    switch (key) {
        case 0: return launch_t<VK_CONST, 0, false, TT>(g, t, tr, traces, image, w, s);
        case 1: return launch_t<VK_CONST, 0, true, TT>(g, t, tr, traces, image, w, s);
        case 2: return launch_t<VK_CONST, 1, false, TT>(g, t, tr, traces, image, w, s);
        case 3: return launch_t<VK_CONST, 1, true, TT>(g, t, tr, traces, image, w, s);
        case 4: return launch_t<VK_LINEAR, 0, false, TT>(g, t, tr, traces, image, w, s);
        case 5: return launch_t<VK_LINEAR, 0, true, TT>(g, t, tr, traces, image, w, s);
        case 6: return launch_t<VK_LINEAR, 1, false, TT>(g, t, tr, traces, image, w, s);
        case 7: return launch_t<VK_LINEAR, 1, true, TT>(g, t, tr, traces, image, w, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_migrate(const GeomParams& g, const TileShape& t, const TraceSet& tr,
                           const void* traces, float* image, int vel_kind, int fast_math,
                           const WaitCfg& w, cudaStream_t s)
{
    switch (g.esize) {
        case 4: return launch_dtype<float>(g, t, tr, traces, image, vel_kind, fast_math, w, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace kh
