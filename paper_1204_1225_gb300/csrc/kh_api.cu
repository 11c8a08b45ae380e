// C ABI (include/kirchhoff.h): plan creation, argument validation, the trace binning pass
// (offset bin per trace and a stable counting sort by bin), the Eq. 2 work count, the
// traveltime evaluator and the dispatch to the migration / demigration / gradient kernels.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#define _USE_MATH_DEFINES
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kh_device.cuh"
#include "kh_plan.h"

namespace {

thread_local std::string g_err;

kh_status fail(kh_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

kh_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(e == cudaErrorMemoryAllocation ? KH_ERR_OOM : KH_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

}  // namespace

namespace kh {

kh_status set_error(kh_status s, const char* msg)
{
    g_err = msg;
    return s;
}

kh_status set_cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }

// ------------------------------------------------------------------ binning kernels

__global__ void k_bin(int ntr, const float* __restrict__ sx, const float* __restrict__ sy,
                      const float* __restrict__ rx, const float* __restrict__ ry, int dim,
                      int n_bins, double w, int* __restrict__ bin)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ntr) return;
    const float ys = (dim == 3 && sy) ? sy[j] : 0.f, yr = (dim == 3 && ry) ? ry[j] : 0.f;
    bin[j] = offset_bin(sx[j], ys, rx[j], yr, n_bins, w);
}

// Stable counting sort of the traces by bin in one CTA of 1024 threads.  Traces without a
// bin are dropped.  bin_start[b] .. bin_start[b+1] is the range of bin b in perm.
constexpr int SORT_THREADS = 1024;
constexpr int MAX_BINS = 256;

__global__ void __launch_bounds__(SORT_THREADS)
    k_sort(int ntr, int n_bins, const int* __restrict__ bin, int* __restrict__ perm,
           int* __restrict__ bin_start)
{
    __shared__ int cnt[MAX_BINS + 1];
    __shared__ int wc[SORT_THREADS / 32][MAX_BINS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int b = tid; b <= n_bins; b += SORT_THREADS) cnt[b] = 0;
    __syncthreads();
    for (int j = tid; j < ntr; j += SORT_THREADS) {
        const int b = bin[j];
        if (b >= 0) atomicAdd(&cnt[b], 1);
    }
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int b = 0; b < n_bins; ++b) {
            const int c = cnt[b];
            cnt[b] = run;
            bin_start[b] = run;
            run += c;
        }
        bin_start[n_bins] = run;
    }
    __syncthreads();
    // cnt[b] is now the running insertion offset of bin b
    for (int base = 0; base < ntr; base += SORT_THREADS) {
        for (int i = tid; i < (SORT_THREADS / 32) * n_bins; i += SORT_THREADS) (&wc[0][0])[(i / n_bins) * MAX_BINS + i % n_bins] = 0;
        __syncthreads();
        const int j = base + tid;
        const int b = (j < ntr) ? bin[j] : -1;
        const unsigned same = __match_any_sync(0xffffffffu, b);
        const int rank = __popc(same & ((1u << lane) - 1u));
        if (b >= 0 && rank == 0) wc[warp][b] = __popc(same);
        __syncthreads();
        for (int bb = tid; bb < n_bins; bb += SORT_THREADS) {
            int run = cnt[bb];
            for (int w = 0; w < SORT_THREADS / 32; ++w) {
                const int c = wc[w][bb];
                wc[w][bb] = run;
                run += c;
            }
            cnt[bb] = run;
        }
        __syncthreads();
        if (b >= 0) perm[wc[warp][b] + rank] = j;
        __syncthreads();
    }
}

__global__ void k_gather(const int* __restrict__ bin_start, int n_bins,
                         const int* __restrict__ perm, const float* __restrict__ sx,
                         const float* __restrict__ sy, const float* __restrict__ rx,
                         const float* __restrict__ ry, int dim, float4* __restrict__ hdr,
                         float2* __restrict__ mid)
{
    const int n = bin_start[n_bins];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int j = perm[k];
        const float a = sx[j], c = rx[j];
        const float b = (dim == 3 && sy) ? sy[j] : 0.f, d = (dim == 3 && ry) ? ry[j] : 0.f;
        hdr[k] = make_float4(a, b, c, d);
        mid[k] = make_float2(__fmul_rn(__fadd_rn(a, c), 0.5f), __fmul_rn(__fadd_rn(b, d), 0.5f));
    }
}

// Rows of `nt` samples copied to rows of `ld` (a multiple of 16 bytes) for the bulk copies.
template <typename T>
__global__ void k_pad(int ntr, int nt, long long ld, const T* __restrict__ src, T* __restrict__ dst)
{
    const long long total = (long long)ntr * ld;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long j = i / ld, t = i - j * ld;
        dst[i] = (t < nt) ? src[j * nt + t] : T(0);
    }
}

// FP32 rows of `nt` samples to SamplePair rows of `ld` pairs: (d[i], d[i + 1] - d[i]) with
// d[nt] = 0, zero pairs from nt to ld.  The step is the IEEE difference the interpolation would
// form from the two samples, so the migration result does not depend on the staging layout.
__global__ void k_pairs(int ntr, int nt, int ld, const float* __restrict__ src, SamplePair* __restrict__ dst)
{
    for (int j = blockIdx.x; j < ntr; j += gridDim.x) {
        const float* row = src + (long long)j * nt;
        SamplePair* out = dst + (long long)j * ld;
        for (int t = threadIdx.x; t < ld; t += blockDim.x) {
            const float v = t < nt ? row[t] : 0.f;
            const float n = t + 1 < nt ? row[t + 1] : 0.f;
            SamplePair q;
            q.v = v;
            q.d = __fsub_rn(n, v);
            out[t] = q;
        }
    }
}

// FP32 rows of `nt` samples to slope rows of `ld`: d[i + 1] - d[i] with d[nt] = 0 (the IEEE
// difference the gradient kernel would form from the two samples), zeros from nt to ld.
__global__ void k_slopes(int ntr, int nt, int ld, const float* __restrict__ src, float* __restrict__ dst)
{
    for (int j = blockIdx.x; j < ntr; j += gridDim.x) {
        const float* row = src + (long long)j * nt;
        float* out = dst + (long long)j * ld;
        for (int t = threadIdx.x; t < ld; t += blockDim.x) {
            const float v = t < nt ? row[t] : 0.f;
            const float n = t + 1 < nt ? row[t + 1] : 0.f;
            out[t] = __fsub_rn(n, v);
        }
    }
}

// Eq. 2 work count: per trace (one CTA each), the in-aperture columns times nz.
__global__ void k_count(int ntr, const float* __restrict__ sx, const float* __restrict__ sy,
                        const float* __restrict__ rx, const float* __restrict__ ry, GeomParams g,
                        double bin_width, long long* __restrict__ out)
{
    __shared__ long long part[32];
    const int j = blockIdx.x;
    const float a = sx[j], c = rx[j];
    const float b = (g.dim == 3 && sy) ? sy[j] : 0.f, d = (g.dim == 3 && ry) ? ry[j] : 0.f;
    const int bin = offset_bin(a, b, c, d, g.n_bins, bin_width);
    long long n = 0;
    if (bin >= 0) {
        if (!g.use_aperture) {
            n = (threadIdx.x == 0) ? (long long)g.nx * g.ny : 0;
        } else {
            const float mx = __fmul_rn(__fadd_rn(a, c), 0.5f), my = __fmul_rn(__fadd_rn(b, d), 0.5f);
            for (long long col = threadIdx.x; col < (long long)g.nx * g.ny; col += blockDim.x) {
                const int iy = (int)(col / g.nx), ix = (int)(col % g.nx);
                const float cx = col_coord(g.ox, ix, g.dx);
                const float cy = g.dim == 3 ? col_coord(g.oy, iy, g.dy) : 0.f;
                n += in_aperture(cx, cy, mx, my, g.A2) ? 1 : 0;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
        out[j] = s * g.nz;
    }
}

// Traveltime of the plan's model in FP64, rounded to FP32 (a utility, not the hot loop).
// Velocity kind of the traveltime utility for time migration (the double-square-root leg).
constexpr int VK_PSTM_UTIL = 7;

__device__ double tt_exact(double R, double z, int vel, double v0, double k)
{
    if (vel == VK_CONST || k == 0.0) return R / v0;
    const double vz = v0 + k * z;
    const double g = sqrt(v0 * vz);
    const double s = fabs(k) * R / (2.0 * g);
    if (s < 1e-4) return R / g * (1.0 - s * s / 6.0 + 3.0 * s * s * s * s / 40.0);
    return 2.0 * asinh(s) / fabs(k);
}

__global__ void k_traveltime(int n, const float* __restrict__ px, const float* __restrict__ py,
                             const float* __restrict__ pz, const float* __restrict__ lx,
                             const float* __restrict__ ly, int vel, double v0, double k,
                             float* __restrict__ T)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ex = (double)px[i] - lx[i];
    const double ey = (py && ly) ? (double)py[i] - ly[i] : 0.0;
    const double z = pz[i];
    if (vel == VK_PSTM_UTIL) {   // time migration: z is the two-way vertical time t0
        const double h2 = ex * ex + ey * ey;
        T[i] = (float)sqrt(0.25 * z * z + h2 / vrms2_of(v0, k, z));
        return;
    }
    T[i] = (float)tt_exact(sqrt(ex * ex + ey * ey + z * z), z, vel, v0, k);
}

}  // namespace kh

using namespace kh;

// ------------------------------------------------------------------ plan helpers

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static int dtype_size(kh_dtype t) { return t == KH_F32 ? 4 : 2; }

static kh_status validate_desc(const kh_desc* d)
{
    if (!d) return fail(KH_ERR_INVALID_ARG, "desc is NULL");
    if (d->dim != 2 && d->dim != 3) return fail(KH_ERR_INVALID_ARG, "dim must be 2 or 3 (got %d)", d->dim);
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(KH_ERR_INVALID_ARG, "image sizes must be >= 1");
    if (d->dim == 2 && d->ny != 1) return fail(KH_ERR_INVALID_ARG, "ny must be 1 for dim 2");
    if (!(d->dx > 0) || !(d->dz > 0) || (d->dim == 3 && !(d->dy > 0)))
        return fail(KH_ERR_INVALID_ARG, "image spacing must be > 0");
    if ((long long)d->nx * d->ny * d->nz * (long long)d->n_bins > (1LL << 40))
        return fail(KH_ERR_INVALID_ARG, "image too large");
    if (d->n_bins < 1 || d->n_bins > kh::MAX_BINS)
        return fail(KH_ERR_INVALID_ARG, "n_bins must be in [1, %d]", kh::MAX_BINS);
    if (!(d->bin_width > 0)) return fail(KH_ERR_INVALID_ARG, "bin_width must be > 0");
    if (d->vel != KH_VEL_CONST && d->vel != KH_VEL_LINEAR_Z && d->vel != KH_VEL_TABLE && d->vel != KH_VEL_PSTM &&
        d->vel != KH_VEL_GRID)
        return fail(KH_ERR_INVALID_ARG, "bad velocity kind %d", (int)d->vel);
    if (d->vel == KH_VEL_GRID && d->dim != 2)
        return fail(KH_ERR_UNSUPPORTED, "KH_VEL_GRID (gridded v(x, z)) is 2D only");
    if (d->vel == KH_VEL_PSTM && !(std::min(d->oz, d->oz + (d->nz - 1) * d->dz) >= 0.0))
        return fail(KH_ERR_INVALID_ARG, "time migration: the image's vertical axis is two-way time, t0 >= 0");
    if (d->vel != KH_VEL_GRID && (!(d->v0 > 0) || !std::isfinite(d->v0)))
        return fail(KH_ERR_INVALID_ARG, "v0 must be > 0");
    if (d->vel != KH_VEL_GRID && !std::isfinite(d->k)) return fail(KH_ERR_INVALID_ARG, "k must be finite");
    if (d->weight != KH_W_ONE && d->weight != KH_W_OBLIQ_SPREAD && d->weight != KH_W_TRUE_AMP)
        return fail(KH_ERR_INVALID_ARG, "bad weight kind %d", (int)d->weight);
    if (d->weight == KH_W_TRUE_AMP && d->vel != KH_VEL_CONST)
        return fail(KH_ERR_UNSUPPORTED, "the true-amplitude weight is built for constant velocity only");
    if (d->weight == KH_W_OBLIQ_SPREAD && !(d->r0 > 0)) return fail(KH_ERR_INVALID_ARG, "r0 must be > 0");
    if (d->nt < 2) return fail(KH_ERR_UNSUPPORTED, "nt must be >= 2 (got %d)", d->nt);
    if (!(d->dt > 0) || !std::isfinite(d->t0)) return fail(KH_ERR_INVALID_ARG, "dt must be > 0, t0 finite");
    if (d->trace_dtype != KH_F32 && d->trace_dtype != KH_F16 && d->trace_dtype != KH_BF16)
        return fail(KH_ERR_INVALID_ARG, "bad trace dtype");
    if (d->vel != KH_VEL_CONST && d->vel != KH_VEL_PSTM && d->vel != KH_VEL_GRID) {
        const double zlo = std::min(0.0, std::min(d->oz, d->oz + (d->nz - 1) * d->dz));
        const double zhi = std::max(d->oz, d->oz + (d->nz - 1) * d->dz);
        if (!(d->v0 + d->k * zlo > 0) || !(d->v0 + d->k * zhi > 0))
            return fail(KH_ERR_UNSUPPORTED, "v(z) = v0 + k z must stay > 0 over the image depths");
    }
    if (d->vel == KH_VEL_TABLE) {
        if (!(d->table_spacing > 0) || !std::isfinite(d->table_spacing))
            return fail(KH_ERR_INVALID_ARG, "table_spacing must be > 0");
        if (d->table_dtype != KH_F32 && d->table_dtype != KH_F16 && d->table_dtype != KH_U16)
            return fail(KH_ERR_INVALID_ARG, "table_dtype must be KH_F32, KH_F16 or KH_U16");
    }
    if (d->trace_dtype == KH_U16) return fail(KH_ERR_INVALID_ARG, "traces cannot be KH_U16");
    if (!(d->taper >= 0.0 && d->taper < 1.0)) return fail(KH_ERR_INVALID_ARG, "taper must be in [0, 1)");
    if (!(d->aa_spacing >= 0.0) || !std::isfinite(d->aa_spacing))
        return fail(KH_ERR_INVALID_ARG, "aa_spacing must be finite and >= 0");
    if (d->aa_spacing > 0.0 && d->vel != KH_VEL_CONST && d->vel != KH_VEL_LINEAR_Z)
        return fail(KH_ERR_UNSUPPORTED, "operator anti-aliasing is built for KH_VEL_CONST and KH_VEL_LINEAR_Z");
    if (d->aa_spacing > 0.0 && d->vel == KH_VEL_LINEAR_Z && d->k != 0.0 && d->trace_dtype != KH_F32)
        return fail(KH_ERR_UNSUPPORTED, "operator anti-aliasing with v0 + k z takes FP32 traces");
    const int ealign = 16 / dtype_size(d->trace_dtype);
    const int cap = std::max((d->nt + 3 * ealign) / ealign * ealign, 16384 / 4);
    if ((size_t)kh::STAGES * cap * dtype_size(d->trace_dtype) > 160u * 1024u)
        return fail(KH_ERR_UNSUPPORTED, "nt = %d too long for the shared-memory trace ring", d->nt);
    return KH_OK;
}

static GeomParams geom_of(const kh_desc& d)
{
    GeomParams g;
    std::memset(&g, 0, sizeof g);
    g.dim = d.dim;
    g.nx = d.nx;
    g.ny = d.ny;
    g.nz = d.nz;
    g.n_bins = d.n_bins;
    g.ox = d.ox;
    g.oy = d.oy;
    g.oz = d.oz;
    g.dx = d.dx;
    g.dy = d.dy;
    g.dz = d.dz;
    g.fdz = (float)d.dz;
    const bool lin = d.vel != KH_VEL_CONST && d.vel != KH_VEL_PSTM && d.vel != KH_VEL_GRID && d.k != 0.0;
    g.pstm = d.vel == KH_VEL_PSTM ? 1 : 0;
    g.pk = d.vel == KH_VEL_PSTM ? d.k : 0.0;
    g.v0 = d.v0;
    g.k = lin ? d.k : 0.0;
    g.kabs = std::fabs(g.k);
    g.t0 = (float)d.t0;
    g.dt = (float)d.dt;
    g.t0d = d.t0;
    g.dtd = d.dt;
    g.a = lin ? g.k * g.k / (2.0 * d.v0) : 0.0;
    const double c1 = lin ? 1.0 / (g.kabs * d.dt) : 1.0 / (d.v0 * d.dt);
    g.C1 = (float)c1;
    g.C1lo = (float)(c1 - (double)g.C1);
    g.c0 = -d.t0 / d.dt - 0.5;
    g.weight = (int)d.weight;   // 0 one, 1 obliquity x spreading, 2 true amplitude
    g.wscale = 1.0 / (2.0 * d.r0 * d.r0);
    g.use_aperture = d.aperture > 0 ? 1 : 0;
    g.A2 = (float)(d.aperture * d.aperture);
    g.use_taper = (d.aperture > 0 && d.taper > 0) ? 1 : 0;
    g.ap_core = g.use_taper ? (float)((1.0 - d.taper) * d.aperture) : 0.f;
    g.ap_core2 = g.use_taper ? (float)((1.0 - d.taper) * d.aperture * (1.0 - d.taper) * d.aperture) : 0.f;
    g.ap_invband = g.use_taper ? (float)(1.0 / (d.taper * d.aperture)) : 0.f;
    g.A2cull = (float)((d.aperture * (1.0 + 1e-5) + 1.0) * (d.aperture * (1.0 + 1e-5) + 1.0));
    // anti-aliasing: the constant-velocity kernels take p = sum (x - a)_h / R_a scaled by 1 / (v0 dt),
    // the v0 + k z kernels p = sum (x - a)_h f_a with each leg's slowness factor f_a, scaled by 1 / dt
    const bool aa = (d.vel == KH_VEL_CONST || d.vel == KH_VEL_LINEAR_Z) && d.aa_spacing > 0.0;
    g.aa_c = !aa ? 0.f : (g.k == 0.0 ? (float)(d.aa_spacing / (d.v0 * d.dt)) : (float)(d.aa_spacing / d.dt));
    g.aa_v0sq = (float)(d.v0 * d.v0);
    g.aa_v0k = (float)(d.v0 * g.k);
    g.aa_kq = (float)(0.25 * g.k * g.k);
    g.nt = d.nt;
    g.esize = dtype_size(d.trace_dtype);
    g.tdtype = (int)d.trace_dtype;
    g.elem_align = 16 / g.esize;
    g.ld = d.nt;
    return g;
}

// Fits ln(1 + x) = x (1 + x Q) on [lo, hi], Q a polynomial in t = (x - m)/h (m, h: centre
// and half-width), by interpolation at the Chebyshev nodes of [-1, 1] (well conditioned in
// t); then checks the FP32-coefficient evaluation against log1p in double on a dense grid.
// Returns false if the interval is too wide for the term count.
static bool cheb_q(double lo, double hi, int terms, double* cq, double& m, double& h)
{
    const int n = terms - 1;
    m = 0.5 * (lo + hi);
    h = 0.5 * (hi - lo);
    double A[LP_LONG][LP_LONG + 1];
    for (int i = 0; i < n; ++i) {
        const double t = std::cos((2.0 * i + 1.0) * M_PI / (2.0 * n));
        const double x = m + h * t;
        double q;
        if (std::fabs(x) < 1e-4) {
            q = -0.5 + x / 3.0 - x * x / 4.0 + x * x * x / 5.0 - x * x * x * x / 6.0;
        } else {
            q = (std::log1p(x) / x - 1.0) / x;
        }
        double pw = 1.0;
        for (int j = 0; j < n; ++j) {
            A[i][j] = pw;
            pw *= t;
        }
        A[i][n] = q;
    }
    for (int c = 0; c < n; ++c) {   // Gaussian elimination, partial pivoting
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return false;
        if (piv != c)
            for (int j = 0; j <= n; ++j) std::swap(A[c][j], A[piv][j]);
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int j = c; j <= n; ++j) A[r][j] -= f * A[c][j];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double v = A[r][n];
        for (int j = r + 1; j < n; ++j) v -= A[r][j] * cq[j];
        cq[r] = v / A[r][r];
    }
    return true;
}

static bool fit_log1p(double lo, double hi, int terms, float* coef, float* scale, float* offset,
                      double tol = 2e-9)
{
    const int n = terms - 1;
    double cq[LP_LONG], m, h;
    if (!cheb_q(lo, hi, terms, cq, m, h)) return false;
    coef[0] = 1.f;
    for (int j = 0; j < n; ++j) coef[j + 1] = (float)cq[j];
    for (int j = terms; j < LP_LONG; ++j) coef[j] = 0.f;   // kernels of a longer length read zeros
    *scale = (float)(1.0 / h);
    *offset = (float)(-m / h);
    double worst = 0.0;
    for (int i = 0; i <= 4000; ++i) {
        const double x = lo + (hi - lo) * i / 4000.0;
        const double t = (double)*scale * x + (double)*offset;
        double p = coef[terms - 1];
        for (int j = terms - 2; j >= 1; --j) p = p * t + coef[j];
        worst = std::max(worst, std::fabs(x * (1.0 + x * p) - std::log1p(x)));
    }
    return worst <= tol;
}

// The per-leg fit of the migration kernel on [expm1(-b), expm1(b)], scaled by c1 (coefc[0] = c1,
// coefc[j + 1] = c1 Q_j, zero beyond `terms`).  Up to LG_MONO terms, Q is re-expanded in x itself,
// t^j = ((x - m)/h)^j = sum_k C(j, k) x^k (-m)^(j - k) / h^j, and the budget check evaluates Q
// by FP32 Horner steps in x as the kernel does (*s = 1, *o = 0); longer fits keep fit_log1p's
// shifted variable.
static bool fit_leg_log(double b, int terms, double c1, float* coefc, float* s, float* o, double tol)
{
    const double lo = std::expm1(-b), hi = std::expm1(b);
    const int n = terms - 1;
    if (terms > LG_MONO) {
        float lp[LP_LONG];
        if (!fit_log1p(lo, hi, terms, lp, s, o, tol)) return false;
        for (int j = 0; j < LP_LONG; ++j) coefc[j] = (float)(c1 * lp[j]);
        return true;
    }
    double cq[LP_LONG], m, h;
    if (!cheb_q(lo, hi, terms, cq, m, h)) return false;
    double d[LP_LONG] = {0.0};
    for (int j = 0; j < n; ++j) {
        double binom = 1.0;   // C(j, k)
        for (int k = 0; k <= j; ++k) {
            d[k] += cq[j] * binom * std::pow(-m, j - k) / std::pow(h, j);
            binom = binom * (j - k) / (k + 1);
        }
    }
    float q[LP_LONG];
    for (int k = 0; k < n; ++k) q[k] = (float)d[k];
    double worst = 0.0;
    for (int i = 0; i <= 4000; ++i) {
        const float x = (float)(lo + (hi - lo) * i / 4000.0);
        float p = q[n - 1];
        for (int k = n - 2; k >= 0; --k) p = std::fma(p, x, q[k]);
        worst = std::max(worst, std::fabs((double)x * (1.0 + (double)x * p) - std::log1p((double)x)));
    }
    if (worst > tol) return false;
    coefc[0] = (float)c1;
    for (int j = 1; j < LP_LONG; ++j) coefc[j] = j <= n ? (float)(c1 * d[j - 1]) : 0.f;
    *s = 1.f;
    *o = 0.f;
    return true;
}

// Linear v(z): the bound on rho = U/U_c - 1 over a tile (|dT| <= distance / v_min along the
// straight segment from the tile centre, per leg).
static double rho_bound(const kh_desc& d, const GeomParams& g, int cx, int cy, int cz)
{
    const double ex = (cx - 1) * d.dx, ey = (d.dim == 3 ? (cy - 1) * d.dy : 0.0);
    const double ez = (cz * NZ - 1) * d.dz;
    const double half = 0.5 * std::sqrt(ex * ex + ey * ey + ez * ez);
    const double zlo = std::min(d.oz, d.oz + (d.nz - 1) * d.dz), zhi = std::max(d.oz, d.oz + (d.nz - 1) * d.dz);
    const double vmin = std::min(d.v0 + d.k * zlo, d.v0 + d.k * zhi);
    return 2.0 * g.kabs * half / vmin * 1.02 + 1e-6;
}

// The ln(1 + rho) fit for the tile: the shortest length of LP_TERMS that meets the budget,
// else unsupported.
static kh_status prepare_linear(const kh_desc& d, const TileShape& t, GeomParams& g)
{
    g.lp_terms = LP_SHORT;
    g.lg_terms = LP_SHORT;
    if (g.k == 0.0 || d.vel == KH_VEL_TABLE) return KH_OK;
    const double b = rho_bound(d, g, t.cx, t.cy, t.cz);
    g.rho_max = (float)std::expm1(b);
    // ln-error budget: 5e-6 of a sample in tau, i.e. 5e-6 |k| dt in ln U
    const double tol = std::max(5e-6 * g.kabs * d.dt, 1e-12);
    for (int i = 0; i < N_LP_TERMS; ++i) {
        g.lp_terms = LP_TERMS[i];
        if (fit_log1p(std::expm1(-b), std::expm1(b), g.lp_terms, g.lp, &g.lp_s, &g.lp_o, tol)) {
            const double c1 = (double)g.C1 + (double)g.C1lo;
            for (int j = 0; j < LP_LONG; ++j) g.lpc[j] = (float)(c1 * g.lp[j]);
            // per-leg fit of the migration kernel: each leg's |ln(1 + rho)| is bounded by half
            // of the two-leg bound, and each leg takes half of the budget
            const double bl = 0.5 * (b - 1e-6) + 1e-6;
            for (int k = 0; k < N_LG_TERMS; ++k) {
                g.lg_terms = LG_TERMS[k];
                if (fit_leg_log(bl, g.lg_terms, c1, g.lgc, &g.lg_s, &g.lg_o, 0.5 * tol)) return KH_OK;
            }
            break;
        }
    }
    return fail(KH_ERR_UNSUPPORTED, "tile too large for the v(z) delta evaluation (rho up to %.3f); "
                                    "choose a smaller tile with KH_OPT_TILE", std::expm1(b));
}

static TileShape shape(const kh_desc& d, int cx, int cy, int cz)
{
    TileShape t;
    t.cx = cx;
    t.cy = cy;
    t.cz = cz;
    t.tiles_x = (d.nx + cx - 1) / cx;
    t.tiles_y = (d.ny + cy - 1) / cy;
    t.tiles_z = (d.nz + cz * NZ - 1) / (cz * NZ);
    return t;
}

// The CTA tile: the caller's choice, else the most compact candidate whose v(z) rho range the
// short polynomial covers (any candidate for constant velocity).
static TileShape tile_of(const kh_plan_s* p)
{
    const kh_desc& d = p->d;
    if (p->tile_code)
        return shape(d, (int)(p->tile_code & 0x3ff), (int)((p->tile_code >> 10) & 0x3ff),
                     (int)((p->tile_code >> 20) & 0x3ff));
    static const int c3[][3] = {{16, 16, 1}, {32, 8, 1}, {8, 8, 4}, {16, 8, 2}};
    static const int c2[][3] = {{64, 1, 4}, {32, 1, 8}, {128, 1, 2}, {16, 1, 16}};
    const int(*c)[3] = d.dim == 3 ? c3 : c2;
    const int nc = 4;
    GeomParams g = geom_of(d);
    if (g.k == 0.0 || d.vel == KH_VEL_TABLE) return shape(d, c[0][0], c[0][1], c[0][2]);
    int best = 0;
    double bb = 1e30;
    for (int i = 0; i < nc; ++i) {
        // prefer shapes the short fit covers; among the rest the smallest rho bound
        const double b = rho_bound(d, g, c[i][0], c[i][1], c[i][2]);
        float tmp[LP_LONG], ts, to;
        if (fit_log1p(std::expm1(-b), std::expm1(b), LP_SHORT, tmp, &ts, &to,
                      std::max(5e-6 * g.kabs * d.dt, 1e-12)))
            return shape(d, c[i][0], c[i][1], c[i][2]);
        if (b < bb) {
            bb = b;
            best = i;
        }
    }
    return shape(d, c[best][0], c[best][1], c[best][2]);
}

template <typename T>
static cudaError_t grow(T*& ptr, size_t& cap, size_t n)
{
    if (n <= cap && ptr) return cudaSuccess;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    size_t want = std::max<size_t>(n + n / 4, 256);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&ptr), want * sizeof(T));
    if (e == cudaSuccess) cap = want;
    return e;
}

namespace kh {

static cudaEvent_t take_event(kh_plan_s* p)
{
    if (!p->ev_pool.empty()) {
        cudaEvent_t e = p->ev_pool.back();
        p->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(kh_plan_s* p, cudaStream_t s)
{
    if (!p->profiling) return;
    cudaEvent_t a = take_event(p);
    cudaEventRecord(a, s);
    p->ev_open.push_back({a, nullptr});
}

void prof_end(kh_plan_s* p, cudaStream_t s)
{
    if (!p->profiling || p->ev_open.empty() || p->ev_open.back().second) return;
    cudaEvent_t b = take_event(p);
    cudaEventRecord(b, s);
    p->ev_open.back().second = b;
}

kh_status ensure_traces_ws(kh_plan_s* p, int ntr)
{
    cudaError_t e;
    if ((e = grow(p->ws_bin, p->cap_bin, (size_t)ntr)) != cudaSuccess) return cuda_fail(e, "workspace (bins)");
    if ((e = grow(p->ws_perm, p->cap_perm, (size_t)ntr)) != cudaSuccess) return cuda_fail(e, "workspace (perm)");
    if ((e = grow(p->ws_hdr, p->cap_hdr, (size_t)ntr)) != cudaSuccess) return cuda_fail(e, "workspace (headers)");
    if ((e = grow(p->ws_mid, p->cap_mid, (size_t)ntr)) != cudaSuccess) return cuda_fail(e, "workspace (midpoints)");
    return KH_OK;
}

CellGrid cell_grid_of(const kh_desc& d, bool spatial)
{
    CellGrid cg;
    if (!(d.aperture > 0)) return cg;
    const double margin = d.aperture * (1.0 + 1e-5) + 2.0;   // the staging cull radius + 1 m
    const double xmin = std::min(d.ox, d.ox + (d.nx - 1) * d.dx), xmax = std::max(d.ox, d.ox + (d.nx - 1) * d.dx);
    const double ymin = d.dim == 3 ? std::min(d.oy, d.oy + (d.ny - 1) * d.dy) : 0.0;
    const double ymax = d.dim == 3 ? std::max(d.oy, d.oy + (d.ny - 1) * d.dy) : 0.0;
    const double ex = xmax - xmin + 2.0 * margin, ey = d.dim == 3 ? ymax - ymin + 2.0 * margin : 0.0;
    const double ext = std::max(ex, ey);
    double cs = std::max(0.5 * d.aperture, ext / MAX_CELLS_PER_AXIS);
    if (spatial) {
        // cells pay only if a default tile's aperture disc spans at most half of them; otherwise
        // every CTA would examine most of its bin anyway, and the bin's original (shot) order
        // keeps the source-leg cache warmer
        const int nx = std::max(1, (int)std::ceil(ex / cs)), ny = d.dim == 3 ? std::max(1, (int)std::ceil(ey / cs)) : 1;
        const double foot = (d.dim == 3 ? 16.0 : 64.0) * std::max(d.dx, d.dim == 3 ? d.dy : 0.0);
        const int span = (int)std::ceil((foot + 2.0 * margin) / cs) + 1;
        const double covered = (double)std::min(nx, span) * (d.dim == 3 ? std::min(ny, span) : 1);
        if (covered > 0.5 * nx * ny) spatial = false;
    }
    if (!spatial) cs = ext * (1.0 + 1e-9) + 1.0;
    cg.ncx = std::min(MAX_CELL_ROWS, std::max(1, (int)std::ceil(ex / cs)));
    cg.ncy = d.dim == 3 ? std::min(MAX_CELL_ROWS, std::max(1, (int)std::ceil(ey / cs))) : 1;
    cg.gx0 = xmin - margin;
    cg.gy0 = ymin - margin;
    cg.inv_cs = 1.0 / cs;
    cg.margin = margin;
    return cg;
}

kh_status bin_traces(kh_plan_s* p, int ntr, const float* sx, const float* sy, const float* rx,
                     const float* ry, cudaStream_t s, bool spatial)
{
    kh_status st = ensure_traces_ws(p, ntr);
    if (st != KH_OK) return st;
    const CellGrid cg = cell_grid_of(p->d, spatial && p->spatial_sort);
    const size_t nkeys = (size_t)p->d.n_bins * cg.ncx * cg.ncy;
    cudaError_t e;
    if ((e = grow(p->ws_key2, p->cap_key2, (size_t)ntr)) != cudaSuccess) return cuda_fail(e, "workspace (sort keys)");
    if ((e = grow(p->ws_perm2, p->cap_perm2, (size_t)ntr)) != cudaSuccess) return cuda_fail(e, "workspace (sort values)");
    if ((e = grow(p->ws_hist, p->cap_hist, (size_t)sort_hist_entries(ntr))) != cudaSuccess)
        return cuda_fail(e, "workspace (sort counts)");
    if ((e = grow(p->ws_cell_start, p->cap_cell_start, nkeys + 1)) != cudaSuccess)
        return cuda_fail(e, "workspace (cell starts)");
    int launches = 0;
    e = sort_traces(ntr, sx, sy, rx, ry, p->d.dim, p->d.n_bins, p->d.bin_width, cg, p->ws_bin, p->ws_key2,
                    p->ws_perm, p->ws_perm2, p->ws_hist, p->ws_cell_start, p->ws_bin_start, &p->cur_perm,
                    &launches, s);
    p->launches += launches;
    if (e != cudaSuccess) return cuda_fail(e, "binning sort");
    p->cur_cg = cg;
    k_gather<<<std::max(1, std::min((ntr + 255) / 256, 4096)), 256, 0, s>>>(
        p->ws_bin_start, p->d.n_bins, p->cur_perm, sx, sy, rx, ry, p->d.dim, p->ws_hdr, p->ws_mid);
    ++p->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "binning kernels");
    return KH_OK;
}

TraceSet plan_traces(const kh_plan_s* p)
{
    TraceSet ts{p->ws_hdr, p->ws_mid, p->cur_perm, p->ws_bin_start};
    if (p->cur_cg.ncx * p->cur_cg.ncy > 1) ts.cell_start = p->ws_cell_start;
    ts.cg = p->cur_cg;
    return ts;
}

// Traces as the kernels read them: rows 16-byte aligned.  Returns the pointer and row stride.
kh_status staged_traces(kh_plan_s* p, int ntr, const void* traces, cudaStream_t s,
                        const void** out, long long* ld)
{
    const int es = dtype_size(p->d.trace_dtype);
    const int ealign = 16 / es;
    if (aligned16(traces) && (p->d.nt % ealign) == 0) {
        *out = traces;
        *ld = p->d.nt;
        return KH_OK;
    }
    const long long L = (p->d.nt + ealign - 1) / ealign * ealign;
    const size_t bytes = (size_t)ntr * L * es;
    cudaError_t e = grow(p->ws_pad, p->cap_pad, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "workspace (padded traces)");
    const int blocks = (int)std::min<long long>(((long long)ntr * L + 255) / 256, 65535);
    if (es == 4)
        k_pad<float><<<std::max(blocks, 1), 256, 0, s>>>(ntr, p->d.nt, L, (const float*)traces,
                                                          (float*)p->ws_pad);
    else
        k_pad<unsigned short><<<std::max(blocks, 1), 256, 0, s>>>(
            ntr, p->d.nt, L, (const unsigned short*)traces, (unsigned short*)p->ws_pad);
    ++p->launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "trace padding kernel");
    *out = p->ws_pad;
    *ld = L;
    return KH_OK;
}

// Whether a migration stages its FP32 traces as SamplePair rows.
static bool use_pairs(const kh_plan_s* p)
{
    return p->sample_pairs && p->d.trace_dtype == KH_F32 && p->d.vel != KH_VEL_TABLE && p->d.nt <= PAIR_MAX_NT;
}

// FP32 traces as SamplePair rows of 16-byte multiples in plan workspace; sets the staging
// fields of g (pairs, esize, elem_align, ld).
static kh_status paired_traces(kh_plan_s* p, int ntr, const void* traces, cudaStream_t s, const void** out,
                               GeomParams& g)
{
    const int L = (p->d.nt + 1) / 2 * 2;
    cudaError_t e = grow(p->ws_pad, p->cap_pad, (size_t)ntr * L * sizeof(SamplePair));
    if (e != cudaSuccess) return cuda_fail(e, "workspace (trace pairs)");
    ++p->launches;
    if ((e = launch_pairs(ntr, p->d.nt, L, traces, p->ws_pad, s)) != cudaSuccess)
        return cuda_fail(e, "trace pair kernel");
    *out = p->ws_pad;
    g.pairs = 1;
    g.esize = (int)sizeof(SamplePair);
    g.elem_align = 16 / (int)sizeof(SamplePair);
    g.ld = L;
    return KH_OK;
}

}  // namespace kh

static kh_status check_headers(const kh_plan_s* p, int ntr, const float* sx, const float* sy,
                               const float* rx, const float* ry)
{
    if (ntr < 0) return fail(KH_ERR_INVALID_ARG, "ntr must be >= 0");
    if (ntr > 0 && (!sx || !rx)) return fail(KH_ERR_INVALID_ARG, "sx/rx must not be NULL");
    if (ntr > 0 && p->d.dim == 3 && (!sy || !ry)) return fail(KH_ERR_INVALID_ARG, "sy/ry must not be NULL for dim 3");
    return KH_OK;
}

// ------------------------------------------------------------------ radial traveltime table

// Largest horizontal distance from any source or receiver to the image footprint (a max is
// order independent, so the atomic keeps the result deterministic).
__global__ void k_hmax(int ntr, const float* __restrict__ sx, const float* __restrict__ sy,
                       const float* __restrict__ rx, const float* __restrict__ ry, int dim, float xlo,
                       float xhi, float ylo, float yhi, unsigned* __restrict__ out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.f;
    if (j < ntr) {
        const float px[2] = {sx[j], rx[j]};
        const float py[2] = {(dim == 3 && sy) ? sy[j] : 0.f, (dim == 3 && ry) ? ry[j] : 0.f};
        for (int a = 0; a < 2; ++a) {
            const float bx = fmaxf(fabsf(px[a] - xlo), fabsf(px[a] - xhi));
            const float by = fmaxf(fabsf(py[a] - ylo), fabsf(py[a] - yhi));
            m = fmaxf(m, sqrtf(bx * bx + by * by));
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// FP64 closed-form node values T(i D, z_a + j D), nodes [nh][nz] with z fastest.
__global__ void k_table_nodes(int nh, int nz, double D, double za, double Dz, int vel, double v0, double k,
                              double* __restrict__ T)
{
    const long long n = (long long)nh * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double h = (double)(i / nz) * D, z = za + (double)(i % nz) * Dz;
        T[i] = tt_exact(sqrt(h * h + z * z), z, vel, v0, k);
    }
}

__global__ void k_table_minmax(long long n, const double* __restrict__ T, double* __restrict__ mm)
{
    __shared__ double lo[256], hi[256];
    double a = 1e300, b = -1e300;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        a = fmin(a, T[i]);
        b = fmax(b, T[i]);
    }
    lo[threadIdx.x] = a;
    hi[threadIdx.x] = b;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            lo[threadIdx.x] = fmin(lo[threadIdx.x], lo[threadIdx.x + w]);
            hi[threadIdx.x] = fmax(hi[threadIdx.x], hi[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mm[0] = lo[0];
        mm[1] = hi[0];
    }
}

// KH_F16: per h row, the least-squares quadratic c0 + c1 u + c2 u^2 in the normalised node depth
// u = j / (nz - 1) (FP64 normal equations, coefficients rounded to FP32).  One thread per row.
__global__ void k_table_rowfit(int nh, int nz, const double* __restrict__ T, float4* __restrict__ coef)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nh) return;
    double m[5] = {0, 0, 0, 0, 0}, b[3] = {0, 0, 0};
    for (int j = 0; j < nz; ++j) {
        const double u = (double)j / (nz - 1), t = T[(long long)r * nz + j];
        double pw = 1.0;
        for (int q = 0; q < 5; ++q) {
            m[q] += pw;
            if (q < 3) b[q] += pw * t;
            pw *= u;
        }
    }
    // [m0 m1 m2; m1 m2 m3; m2 m3 m4] c = b by Cramer's rule (well conditioned on [0, 1])
    const double a00 = m[0], a01 = m[1], a02 = m[2], a11 = m[2], a12 = m[3], a22 = m[4];
    const double det = a00 * (a11 * a22 - a12 * a12) - a01 * (a01 * a22 - a12 * a02) + a02 * (a01 * a12 - a11 * a02);
    const double c0 = (b[0] * (a11 * a22 - a12 * a12) - a01 * (b[1] * a22 - a12 * b[2]) + a02 * (b[1] * a12 - a11 * b[2])) / det;
    const double c1 = (a00 * (b[1] * a22 - a12 * b[2]) - b[0] * (a01 * a22 - a12 * a02) + a02 * (a01 * b[2] - b[1] * a02)) / det;
    const double c2 = (a00 * (a11 * b[2] - b[1] * a12) - a01 * (a01 * b[2] - b[1] * a02) + b[0] * (a01 * a12 - a11 * a02)) / det;
    coef[r] = make_float4((float)c0, (float)c1, (float)c2, 0.f);
}

// Stored values: F32 seconds; F16 T minus the row's reference polynomial (FP32 coefficients,
// evaluated in FP64); U16 round((T - T_min) / scale).
__global__ void k_table_store(long long n, int nz, const double* __restrict__ T, int dt, double tmin,
                              double scale, const float4* __restrict__ coef, void* __restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (dt == KH_F32) {
            static_cast<float*>(out)[i] = (float)T[i];
        } else if (dt == KH_F16) {
            const float4 c = coef[i / nz];
            const double u = (double)(i % nz) / (nz - 1);
            const double ref = (double)c.x + u * ((double)c.y + u * (double)c.z);
            static_cast<__half*>(out)[i] = __double2half(T[i] - ref);
        } else {
            const double u = rint((T[i] - tmin) / scale);
            static_cast<unsigned short*>(out)[i] = (unsigned short)fmin(fmax(u, 0.0), 65535.0);
        }
    }
}

// Builds (or reuses) the radial table for this call's traces and fills the table fields of
// g, including the scale and offset folded into C1 and c0.  Synchronises the stream.
// The radial table of the plan's v(z) model: nodes at h = i D and at image depths
// z = z_min + j m dz (m the largest power of two <= min(4, D / dz)), enough of them for every
// depth of every tile (the padded depth range tiles_z * cz * 16), built in FP64 and stored as
// F32, FP16 of T - T_min or U16 fixed point.  The h extent comes from the headers (one
// synchronisation), so a table migrate call synchronises the stream.
static kh_status ensure_table(kh_plan_s* p, int ntr, const float* sx, const float* sy, const float* rx,
                              const float* ry, cudaStream_t s, const TileShape& tile, GeomParams& g)
{
    const kh_desc& d = p->d;
    cudaError_t e = cudaSuccess;
    if (!p->ws_hmax) e = cudaMalloc(reinterpret_cast<void**>(&p->ws_hmax), sizeof(unsigned));
    if (e == cudaSuccess && !p->ws_tmm) e = cudaMalloc(reinterpret_cast<void**>(&p->ws_tmm), 2 * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e, "workspace (table)");
    const double x0 = d.ox, x1 = d.ox + (d.nx - 1) * d.dx;
    const double y0 = d.dim == 3 ? d.oy : 0.0, y1 = d.dim == 3 ? d.oy + (d.ny - 1) * d.dy : 0.0;
    e = cudaMemsetAsync(p->ws_hmax, 0, sizeof(unsigned), s);
    if (e == cudaSuccess && ntr > 0) {
        k_hmax<<<(ntr + 255) / 256, 256, 0, s>>>(ntr, sx, sy, rx, ry, d.dim, (float)std::min(x0, x1),
                                                 (float)std::max(x0, x1), (float)std::min(y0, y1),
                                                 (float)std::max(y0, y1), p->ws_hmax);
        ++p->launches;
        e = cudaGetLastError();
    }
    unsigned hb = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, p->ws_hmax, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "table extent");
    float hmax;
    std::memcpy(&hmax, &hb, sizeof hmax);
    const double D = d.table_spacing;
    const double zmin = std::min(d.oz, d.oz + (d.nz - 1) * d.dz), zmax = std::max(d.oz, d.oz + (d.nz - 1) * d.dz);
    int m = 1;
    while (m < 4 && 2.0 * m <= D / d.dz) m *= 2;
    const double za = d.oz, Dz = m * d.dz;
    const int nh = (int)std::floor(hmax * (1.0 + 1e-6) / D) + 3;
    const int nz = tile.tiles_z * tile.cz * NZ / m + 2;
    const size_t es = d.table_dtype == KH_F32 ? 4 : 2;
    const size_t node_bytes = ((size_t)nh * nz * es + 15) / 16 * 16;
    const size_t bytes = node_bytes + (d.table_dtype == KH_F16 ? (size_t)nh * sizeof(float4) : 0);
    if (bytes > 96u * 1024u)
        return fail(KH_ERR_UNSUPPORTED, "traveltime table of %d x %d nodes (%zu bytes) exceeds the 96 KB "
                                        "shared-memory budget; use a larger table_spacing", nh, nz, bytes);
    if (p->tab_nh < nh || p->tab_nz != nz) {
        const long long n = (long long)nh * nz;
        if ((e = grow(p->ws_tab64, p->cap_tab64, (size_t)n)) != cudaSuccess) return cuda_fail(e, "workspace (table)");
        if ((e = grow(p->ws_tab, p->cap_tab, bytes)) != cudaSuccess) return cuda_fail(e, "workspace (table)");
        const int vel = d.k == 0.0 ? VK_CONST : VK_LINEAR;
        const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
        k_table_nodes<<<blocks, 256, 0, s>>>(nh, nz, D, za, Dz, vel, d.v0, d.k, p->ws_tab64);
        k_table_minmax<<<1, 256, 0, s>>>(n, p->ws_tab64, p->ws_tmm);
        p->launches += 2;
        double mm[2] = {0.0, 0.0};
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(mm, p->ws_tmm, sizeof mm, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "table build");
        const double tmin = d.table_dtype == KH_U16 ? mm[0] : 0.0;
        const double scale = d.table_dtype == KH_U16 ? std::max(mm[1] - mm[0], 1e-30) / 65535.0 : 1.0;
        float4* coef = reinterpret_cast<float4*>(p->ws_tab + node_bytes);
        e = cudaMemsetAsync(p->ws_tab, 0, bytes, s);
        if (e == cudaSuccess && d.table_dtype == KH_F16) {
            k_table_rowfit<<<(nh + 127) / 128, 128, 0, s>>>(nh, nz, p->ws_tab64, coef);
            ++p->launches;
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            k_table_store<<<blocks, 256, 0, s>>>(n, nz, p->ws_tab64, (int)d.table_dtype, tmin, scale, coef,
                                                 p->ws_tab);
            ++p->launches;
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return cuda_fail(e, "table store");
        p->tab_nh = nh;
        p->tab_nz = nz;
        p->tab_tmin = tmin;
        p->tab_scale = scale;
    }
    g.table = p->ws_tab;
    g.tnh = p->tab_nh;
    g.tnz = p->tab_nz;
    g.tdt = (int)d.table_dtype;
    g.tinv = (float)(1.0 / D);
    g.tunz = (float)(1.0 / (g.tnz - 1));
    g.thmax = (float)(g.tnh - 1) - 1e-3f;
    g.tza = za;
    g.tsp = D;
    g.tm = m;
    // Window slack for the interpolation: an interpolated leg time is a convex combination of
    // node times, each node within sqrt(D^2 + Dz^2) of the point, and T is Lipschitz with
    // 1/v_min over the depths the segments cross (image and node depths); two legs, plus two
    // samples for the FP16 / U16 storage error.
    const double zn1 = za + (nz - 1) * Dz;
    const double zlo_all = std::min({0.0, zmin, za}), zhi_all = std::max({0.0, zmax, zn1});
    const double vmin = std::min(d.v0 + d.k * zlo_all, d.v0 + d.k * zhi_all);
    g.tslack = (float)(2.0 * std::sqrt(D * D + Dz * Dz) / (vmin * d.dt) + 2.0);
    const double c1 = p->tab_scale / d.dt;
    g.C1 = (float)c1;
    g.C1lo = (float)(c1 - (double)g.C1);
    g.c0 = (2.0 * p->tab_tmin - d.t0) / d.dt - 0.5;
    return KH_OK;
}

// Demigration tile: the first candidate whose sample window fits the kernel's 96 window rows
// (|dT| <= diagonal / v_min per leg, plus the window slack) and, for v(z), whose rho range the
// ln(1 + rho) fit covers; P image parts so that about six waves of warp tasks run.
static kh_status demigrate_tile(const kh_desc& d, GeomParams& g, int ntr, DmTile& dt)
{
    static const int c3[][3] = {{8, 8, 16}, {8, 8, 8}, {4, 4, 8}, {4, 4, 4}, {2, 2, 4}, {2, 2, 2}};
    static const int c2[][3] = {{32, 1, 32}, {16, 1, 16}, {8, 1, 8}, {4, 1, 4}, {2, 1, 2}};
    const int(*c)[3] = d.dim == 3 ? c3 : c2;
    const int nc = d.dim == 3 ? 6 : 5;
    const double zlo = std::min(0.0, std::min(d.oz, d.oz + (d.nz - 1) * d.dz));
    const double zhi = std::max(0.0, std::max(d.oz, d.oz + (d.nz - 1) * d.dz));
    const double vmin = (d.vel == KH_VEL_CONST) ? d.v0 : std::min(d.v0 + d.k * zlo, d.v0 + d.k * zhi);
    const double slack = 2.0 * (2.0 + 2e-4 * d.nt) + 4.0;
    for (int i = 0; i < nc; ++i) {
        const double ex = (c[i][0] - 1) * d.dx, ey = d.dim == 3 ? (c[i][1] - 1) * d.dy : 0.0;
        const double ez = (c[i][2] - 1) * d.dz;
        const double diag = std::sqrt(ex * ex + ey * ey + ez * ez);
        if (2.0 * diag / (vmin * d.dt) + slack > DM_ROWS_HOST) continue;
        TileShape probe = shape(d, c[i][0], c[i][1], 1);
        probe.cz = 1;
        GeomParams gt = g;
        if (g.k != 0.0) {
            // rho range over this tile (reuses the migration fit with the tile's extent)
            const double half = 0.5 * diag;
            const double b = 2.0 * g.kabs * half / vmin * 1.02 + 1e-6;
            const double tol = std::max(5e-6 * g.kabs * d.dt, 1e-12);
            bool fitted = false;   // the shortest length of LP_TERMS that meets the budget
            for (int q = 0; q < N_LP_TERMS && !fitted; ++q) {
                gt.lp_terms = LP_TERMS[q];
                fitted = fit_log1p(std::expm1(-b), std::expm1(b), gt.lp_terms, gt.lp, &gt.lp_s, &gt.lp_o, tol);
            }
            if (!fitted) continue;
            const double c1 = (double)gt.C1 + (double)gt.C1lo;
            for (int q = 0; q < LP_LONG; ++q) gt.lpc[q] = (float)(c1 * gt.lp[q]);
            gt.rho_max = (float)std::expm1(b);
            // the per-leg fit the kernel evaluates (half the interval, half the budget per leg)
            const double bl = 0.5 * (b - 1e-6) + 1e-6;
            bool leg_fitted = false;
            for (int q = 0; q < N_LG_TERMS && !leg_fitted; ++q) {
                gt.lg_terms = LG_TERMS[q];
                leg_fitted = fit_leg_log(bl, gt.lg_terms, c1, gt.lgc, &gt.lg_s, &gt.lg_o, 0.5 * tol);
            }
            if (!leg_fitted) continue;
        }
        (void)probe;
        g = gt;
        dt.tx = c[i][0];
        dt.ty = c[i][1];
        dt.tz = c[i][2];
        dt.tiles_x = (d.nx + dt.tx - 1) / dt.tx;
        dt.tiles_y = (d.ny + dt.ty - 1) / dt.ty;
        dt.tiles_z = (d.nz + dt.tz - 1) / dt.tz;
        const long long warp_tasks = std::max(1, (ntr + 31) / 32);
        long long P = (6LL * 152 * 16 + warp_tasks - 1) / warp_tasks;
        const long long mem_cap = std::max(1LL, (long long)(8e9 / (4.0 * ntr * (double)d.nt)));
        const long long n_tiles = (long long)dt.tiles_x * dt.tiles_y * dt.tiles_z;
        P = std::max(1LL, std::min(std::min(P, 32LL), std::min(mem_cap, n_tiles)));
        dt.parts = (int)P;
        return KH_OK;
    }
    return fail(KH_ERR_UNSUPPORTED, "no demigration tile keeps the time window within %d samples "
                                    "(velocity too low for the sampling)", DM_ROWS_HOST);
}

// ------------------------------------------------------------------ C ABI

extern "C" {

kh_status kirchhoff_create(const kh_desc* d, kh_plan* out)
{
    if (!out) return fail(KH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    kh_status st = validate_desc(d);
    if (st != KH_OK) return st;
    kh_plan_s* p = new (std::nothrow) kh_plan_s();
    if (!p) return fail(KH_ERR_OOM, "host allocation failed");
    p->d = *d;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->ws_status), 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->ws_status, 0, 2 * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void**>(&p->ws_bin_start), (MAX_BINS + 1) * sizeof(int));
    if (e != cudaSuccess) {
        kirchhoff_destroy(p);
        return cuda_fail(e, "kirchhoff_create");
    }
    *out = p;
    return KH_OK;
}

kh_status kirchhoff_destroy(kh_plan p)
{
    if (!p) return KH_OK;
    cudaDeviceSynchronize();
    cudaFree(p->ws_status);
    cudaFree(p->ws_bin_start);
    cudaFree(p->ws_bin);
    cudaFree(p->ws_perm);
    cudaFree(p->ws_hdr);
    cudaFree(p->ws_mid);
    cudaFree(p->ws_key2);
    cudaFree(p->ws_perm2);
    cudaFree(p->ws_hist);
    cudaFree(p->ws_cell_start);
    cudaFree(p->ws_stats);
    cudaFree(p->ws_semb);
    cudaFree(p->ws_pad);
    cudaFree(p->ws_count);
    cudaFree(p->ws_partial);
    cudaFree(p->ws_dm);
    cudaFree(p->ws_tab);
    cudaFree(p->ws_tab64);
    cudaFree(p->ws_tmm);
    cudaFree(p->ws_hmax);
    cudaFree(p->ws_gtab);
    cudaFree(p->ws_gloc);
    cudaFree(p->ws_grounds);
    cudaFree(p->ws_gslow);
    cudaFree(p->ws_gbnd);
    for (auto& pr : p->ev_open) {
        if (pr.first) cudaEventDestroy(pr.first);
        if (pr.second) cudaEventDestroy(pr.second);
    }
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    host_release(p);
    delete p;
    return KH_OK;
}

kh_status kirchhoff_set_option(kh_plan p, kh_option opt, long long value)
{
    if (!p) return fail(KH_ERR_INVALID_ARG, "plan is NULL");
    switch (opt) {
        case KH_OPT_WAIT_POLLS:
            if (value < 0) return fail(KH_ERR_INVALID_ARG, "wait polls must be >= 0");
            p->wait_polls = value;
            return KH_OK;
        case KH_OPT_FAST_MATH:
            p->fast_math = value ? 1 : 0;
            return KH_OK;
        case KH_OPT_TILE: {
            if (value == 0) {
                p->tile_code = 0;
                return KH_OK;
            }
            const int cx = (int)(value & 0x3ff), cy = (int)((value >> 10) & 0x3ff), cz = (int)((value >> 20) & 0x3ff);
            if (cx < 1 || cy < 1 || cz < 1 || cx * cy * cz != CONSUMERS || (value >> 30) != 0)
                return fail(KH_ERR_INVALID_ARG, "tile cx*cy*cz must equal %d", CONSUMERS);
            if (cz > 16) return fail(KH_ERR_INVALID_ARG, "tile cz must be <= 16");
            if (p->d.dim == 2 && cy != 1) return fail(KH_ERR_INVALID_ARG, "tile cy must be 1 for dim 2");
            p->tile_code = value;
            return KH_OK;
        }
        case KH_OPT_BATCH_MODE:
            if (value != 0 && value != 1) return fail(KH_ERR_INVALID_ARG, "batch mode must be 0 or 1");
            p->batch_mode = (int)value;
            return KH_OK;
        case KH_OPT_SAMPLE_PAIRS:
            p->sample_pairs = value ? 1 : 0;
            return KH_OK;
        case KH_OPT_SPATIAL_SORT:
            p->spatial_sort = value ? 1 : 0;
            return KH_OK;
        default:
            return fail(KH_ERR_INVALID_ARG, "unknown option %d", (int)opt);
    }
}

kh_status kirchhoff_migrate(kh_plan p, int ntr, const float* sx, const float* sy, const float* rx,
                            const float* ry, const void* traces, float* image, void* cuda_stream)
{
    if (!p) return fail(KH_ERR_INVALID_ARG, "plan is NULL");
    kh_status st = check_headers(p, ntr, sx, sy, rx, ry);
    if (st != KH_OK) return st;
    if (!image) return fail(KH_ERR_INVALID_ARG, "image is NULL");
    if (ntr > 0 && !traces) return fail(KH_ERR_INVALID_ARG, "traces is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const size_t img_bytes = (size_t)p->d.n_bins * p->d.ny * p->d.nx * p->d.nz * sizeof(float);
    if (ntr == 0) {
        cudaError_t e = cudaMemsetAsync(image, 0, img_bytes, s);
        return e == cudaSuccess ? KH_OK : cuda_fail(e, "cudaMemsetAsync");
    }
    if ((st = bin_traces(p, ntr, sx, sy, rx, ry, s)) != KH_OK) return st;
    const void* tr_ptr = nullptr;
    GeomParams g = geom_of(p->d);
    st = use_pairs(p) ? paired_traces(p, ntr, traces, s, &tr_ptr, g) : staged_traces(p, ntr, traces, s, &tr_ptr, &g.ld);
    if (st != KH_OK) return st;
    const TileShape tile = tile_of(p);
    if ((st = prepare_linear(p->d, tile, g)) != KH_OK) return st;
    int vk = (g.k == 0.0) ? VK_CONST : VK_LINEAR;
    if (p->d.vel == KH_VEL_TABLE) {
        if ((st = ensure_table(p, ntr, sx, sy, rx, ry, s, tile, g)) != KH_OK) return st;
        vk = VK_TABLE;
    } else if (p->d.vel == KH_VEL_GRID) {
        if ((st = grid_prepare(p, tile, g, s)) != KH_OK) return st;
        vk = VK_GRID;
    }
    TraceSet ts = plan_traces(p);
    WaitCfg w{p->ws_status, p->wait_polls, WAIT_NS};
    if (p->profiling) w.stats = p->ws_stats;
    prof_begin(p, s);
    cudaError_t e = launch_migrate(g, tile, ts, tr_ptr, image, vk, p->fast_math, w, s);
    prof_end(p, s);
    ++p->launches;
    if (e != cudaSuccess) return cuda_fail(e, "migration kernel");
    return KH_OK;
}

kh_status kirchhoff_demigrate(kh_plan p, int ntr, const float* sx, const float* sy,
                              const float* rx, const float* ry, const float* image,
                              float* traces_out, void* cuda_stream)
{
    if (!p) return fail(KH_ERR_INVALID_ARG, "plan is NULL");
    kh_status st = check_headers(p, ntr, sx, sy, rx, ry);
    if (st != KH_OK) return st;
    if (ntr > 0 && (!image || !traces_out)) return fail(KH_ERR_INVALID_ARG, "image/traces_out is NULL");
    if (p->d.vel == KH_VEL_TABLE || p->d.vel == KH_VEL_PSTM || p->d.vel == KH_VEL_GRID)
        return fail(KH_ERR_UNSUPPORTED, "demigration uses the analytic depth traveltimes; "
                                        "create the plan with KH_VEL_CONST or KH_VEL_LINEAR_Z");
    if (ntr == 0) return KH_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const kh_desc& d = p->d;
    GeomParams g = geom_of(d);
    DmTile dt;
    if ((st = demigrate_tile(d, g, ntr, dt)) != KH_OK) return st;
    // bin order alone: the adjoint's warps share source legs when their traces come shot by shot
    if ((st = bin_traces(p, ntr, sx, sy, rx, ry, s, false)) != KH_OK) return st;
    const size_t per_part = (size_t)ntr * d.nt;
    cudaError_t e = grow(p->ws_dm, p->cap_dm, per_part * dt.parts);
    if (e != cudaSuccess) return cuda_fail(e, "workspace (demigration partial traces)");
    e = cudaMemsetAsync(p->ws_dm, 0, sizeof(float) * per_part * dt.parts, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(traces_out, 0, sizeof(float) * per_part, s);
    if (e != cudaSuccess) return cuda_fail(e, "kirchhoff_demigrate: memset");
    TraceSet ts = plan_traces(p);
    const int vk = (g.k == 0.0) ? VK_CONST : VK_LINEAR;
    const int max_chunks = (ntr + 127) / 128;
    prof_begin(p, s);
    e = launch_demigrate(g, dt, ts, image, p->ws_dm, p->ws_status, max_chunks, vk, p->fast_math, s);
    prof_end(p, s);
    ++p->launches;
    if (e == cudaSuccess) e = launch_dm_reduce(ts, d.n_bins, p->ws_dm, dt.parts, d.nt, traces_out, ntr, s);
    ++p->launches;
    if (e != cudaSuccess) return cuda_fail(e, "demigration kernels");
    return KH_OK;
}

kh_status kirchhoff_velocity_grad(kh_plan p, int ntr, const float* sx, const float* sy,
                                  const float* rx, const float* ry, const float* image,
                                  const float* traces, double* out_dv0_dk, void* cuda_stream)
{
    if (!p) return fail(KH_ERR_INVALID_ARG, "plan is NULL");
    kh_status st = check_headers(p, ntr, sx, sy, rx, ry);
    if (st != KH_OK) return st;
    if (!out_dv0_dk) return fail(KH_ERR_INVALID_ARG, "out_dv0_dk is NULL");
    if (ntr > 0 && (!image || !traces)) return fail(KH_ERR_INVALID_ARG, "image/traces is NULL");
    if (p->d.vel == KH_VEL_TABLE || p->d.vel == KH_VEL_PSTM || p->d.vel == KH_VEL_GRID)
        return fail(KH_ERR_UNSUPPORTED, "no velocity gradient for table traveltimes or time migration");
    if (p->d.weight == KH_W_TRUE_AMP || p->d.aa_spacing > 0.0)
        return fail(KH_ERR_UNSUPPORTED, "no velocity gradient with the true-amplitude weight or anti-aliasing");
    if (p->d.trace_dtype != KH_F32) return fail(KH_ERR_UNSUPPORTED, "velocity gradient takes FP32 traces");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemsetAsync(out_dv0_dk, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (ntr == 0) return KH_OK;
    if ((st = bin_traces(p, ntr, sx, sy, rx, ry, s)) != KH_OK) return st;
    GeomParams g = geom_of(p->d);
    g.grad = 1;
    // slope rows, 16-byte multiples, in plan workspace
    const int L = (p->d.nt + 3) / 4 * 4;
    if ((e = grow(p->ws_pad, p->cap_pad, (size_t)ntr * L * sizeof(float))) != cudaSuccess)
        return cuda_fail(e, "workspace (slope rows)");
    k_slopes<<<std::min(ntr, 1 << 20), 256, 0, s>>>(ntr, p->d.nt, L, traces, reinterpret_cast<float*>(p->ws_pad));
    ++p->launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "slope kernel");
    const void* tr_ptr = p->ws_pad;
    g.ld = L;
    const TileShape tile = tile_of(p);
    if ((st = prepare_linear(p->d, tile, g)) != KH_OK) return st;
    const long long nwarps = (long long)tile.tiles_x * tile.tiles_y * tile.tiles_z * p->d.n_bins * CONSUMER_WARPS;
    if ((e = grow(p->ws_partial, p->cap_partial, (size_t)(2 * nwarps))) != cudaSuccess)
        return cuda_fail(e, "workspace (gradient partials)");
    TraceSet ts = plan_traces(p);
    WaitCfg w{p->ws_status, p->wait_polls, WAIT_NS};
    if (p->profiling) w.stats = p->ws_stats;
    const int vk = (g.k == 0.0) ? VK_CONST : VK_LINEAR;
    prof_begin(p, s);
    e = launch_vgrad(g, tile, ts, tr_ptr, image, vk, p->fast_math, w, p->ws_partial, s);
    prof_end(p, s);
    ++p->launches;
    if (e == cudaSuccess) e = launch_vgrad_reduce(p->ws_partial, nwarps, 1.0 / p->d.dt, out_dv0_dk, s);
    ++p->launches;
    if (e != cudaSuccess) return cuda_fail(e, "velocity-gradient kernels");
    return KH_OK;
}

kh_status kirchhoff_count(kh_plan p, int ntr, const float* sx, const float* sy, const float* rx,
                          const float* ry, int64_t* out_count, void* cuda_stream)
{
    if (!p || !out_count) return fail(KH_ERR_INVALID_ARG, "plan/out_count is NULL");
    kh_status st = check_headers(p, ntr, sx, sy, rx, ry);
    if (st != KH_OK) return st;
    *out_count = 0;
    if (ntr == 0) return KH_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = grow(p->ws_count, p->cap_count, (size_t)ntr);
    if (e != cudaSuccess) return cuda_fail(e, "workspace (count)");
    GeomParams g = geom_of(p->d);
    k_count<<<ntr, 256, 0, s>>>(ntr, sx, sy, rx, ry, g, p->d.bin_width, p->ws_count);
    ++p->launches;
    std::vector<long long> h((size_t)ntr);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), p->ws_count, sizeof(long long) * ntr, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "kirchhoff_count");
    long long total = 0;
    for (long long v : h) total += v;
    *out_count = total;
    return KH_OK;
}

kh_status kirchhoff_traveltime(kh_plan p, int n, const float* px, const float* py, const float* pz,
                               const float* lx, const float* ly, float* T, void* cuda_stream)
{
    if (!p) return fail(KH_ERR_INVALID_ARG, "plan is NULL");
    if (n < 0) return fail(KH_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return KH_OK;
    if (!px || !pz || !lx || !T) return fail(KH_ERR_INVALID_ARG, "NULL array");
    if (p->d.vel == KH_VEL_GRID)
        return fail(KH_ERR_UNSUPPORTED, "KH_VEL_GRID: read the tables with kirchhoff_grid_read");
    const bool pstm = p->d.vel == KH_VEL_PSTM;
    const bool lin = !pstm && p->d.vel != KH_VEL_CONST && p->d.k != 0.0;
    k_traveltime<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
        n, px, p->d.dim == 3 ? py : nullptr, pz, lx, p->d.dim == 3 ? ly : nullptr,
        pstm ? VK_PSTM_UTIL : (lin ? VK_LINEAR : VK_CONST), p->d.v0, (lin || pstm) ? p->d.k : 0.0, T);
    ++p->launches;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KH_OK : cuda_fail(e, "traveltime kernel");
}

kh_status kirchhoff_fit_report(const kh_desc* d, int cx, int cy, int cz, int* two_leg_terms, int* leg_terms,
                               double* leg_bound, float* coef, float* scale, float* offset, double* c1)
{
    kh_status st = validate_desc(d);
    if (st != KH_OK) return st;
    if (d->vel != KH_VEL_LINEAR_Z || d->k == 0.0)
        return fail(KH_ERR_INVALID_ARG, "the fit report is for linear v(z) descriptors with k != 0");
    if (cx < 1 || cy < 1 || cz < 1 || cz > 16 || cx * cy * cz != CONSUMERS || (d->dim == 2 && cy != 1))
        return fail(KH_ERR_INVALID_ARG, "tile cx*cy*cz must equal %d with cz <= 16 (cy = 1 for dim 2)", CONSUMERS);
    const TileShape t = shape(*d, cx, cy, cz);
    GeomParams g = geom_of(*d);
    if ((st = prepare_linear(*d, t, g)) != KH_OK) return st;
    const double b = rho_bound(*d, g, cx, cy, cz);
    if (two_leg_terms) *two_leg_terms = g.lp_terms;
    if (leg_terms) *leg_terms = g.lg_terms;
    if (leg_bound) *leg_bound = 0.5 * (b - 1e-6) + 1e-6;
    if (coef)
        for (int j = 0; j < LP_LONG; ++j) coef[j] = g.lgc[j];
    if (scale) *scale = g.lg_s;
    if (offset) *offset = g.lg_o;
    if (c1) *c1 = (double)g.C1 + (double)g.C1lo;
    return KH_OK;
}

kh_status kirchhoff_sync(kh_plan p, void* cuda_stream)
{
    if (!p) return fail(KH_ERR_INVALID_ARG, "plan is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int h = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&h, p->ws_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "kirchhoff_sync");
    if (h != 0) {
        cudaMemset(p->ws_status, 0, sizeof(int));
        if (h & 1)
            return fail(KH_ERR_TIMEOUT, "a bounded in-kernel wait ran out (status 0x%x); results are invalid", h);
        if (h == STATUS_NO_TABLE)
            return fail(KH_ERR_INVALID_ARG, "a trace's source or receiver position is not one of the locations "
                                            "of the KH_VEL_GRID tables; those traces were skipped");
        return fail(KH_ERR_INTERNAL, "a kernel reported an internal sizing error (status 0x%x); "
                                     "results are invalid", h);
    }
    return KH_OK;
}

kh_status kirchhoff_profile(kh_plan p, int enable)
{
    if (!p) return fail(KH_ERR_INVALID_ARG, "plan is NULL");
    if (enable && !p->ws_stats) {
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p->ws_stats), 3 * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemset(p->ws_stats, 0, 3 * sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_fail(e, "kirchhoff_profile (staging counters)");
    }
    p->profiling = enable ? 1 : 0;
    return KH_OK;
}

kh_status kirchhoff_cell_grid(const kh_desc* d, int spatial, int* ncx, int* ncy, double* gx0, double* gy0,
                              double* inv_cell)
{
    kh_status st = validate_desc(d);
    if (st != KH_OK) return st;
    const CellGrid cg = cell_grid_of(*d, spatial != 0);
    if (ncx) *ncx = cg.ncx;
    if (ncy) *ncy = cg.ncy;
    if (gx0) *gx0 = cg.gx0;
    if (gy0) *gy0 = cg.gy0;
    if (inv_cell) *inv_cell = cg.inv_cs;
    return KH_OK;
}

kh_status kirchhoff_bin_sort(kh_plan p, int ntr, const float* sx, const float* sy, const float* rx,
                             const float* ry, int* perm_out, int* key_start_out, void* cuda_stream)
{
    if (!p) return fail(KH_ERR_INVALID_ARG, "plan is NULL");
    kh_status st = check_headers(p, ntr, sx, sy, rx, ry);
    if (st != KH_OK) return st;
    if ((ntr > 0 && !perm_out) || !key_start_out) return fail(KH_ERR_INVALID_ARG, "perm/key_start is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if ((st = bin_traces(p, ntr, sx, sy, rx, ry, s)) != KH_OK) return st;
    const size_t nkeys = (size_t)p->d.n_bins * p->cur_cg.ncx * p->cur_cg.ncy;
    cudaError_t e = cudaSuccess;
    if (ntr > 0)
        e = cudaMemcpyAsync(perm_out, p->cur_perm, sizeof(int) * (size_t)ntr, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(key_start_out, p->ws_cell_start, sizeof(int) * (nkeys + 1), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "kirchhoff_bin_sort: copies");
    return KH_OK;
}

kh_status kirchhoff_staging_stats(kh_plan p, void* cuda_stream, unsigned long long* examined,
                                  unsigned long long* staged, unsigned long long* ctas)
{
    if (!p || !examined || !staged || !ctas) return fail(KH_ERR_INVALID_ARG, "NULL argument");
    *examined = *staged = *ctas = 0;
    if (!p->ws_stats) return KH_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned long long h[3] = {0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(h, p->ws_stats, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->ws_stats, 0, sizeof h, s);
    if (e != cudaSuccess) return cuda_fail(e, "kirchhoff_staging_stats");
    *examined = h[0];
    *staged = h[1];
    *ctas = h[2];
    return KH_OK;
}

kh_status kirchhoff_profile_read(kh_plan p, double* kernel_ms, long long* timed_launches)
{
    if (!p || !kernel_ms || !timed_launches) return fail(KH_ERR_INVALID_ARG, "NULL argument");
    double total = 0.0;
    long long n = 0;
    for (auto& pr : p->ev_open) {
        if (pr.second) {
            cudaError_t e = cudaEventSynchronize(pr.second);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pr.first, pr.second);
            if (e != cudaSuccess) return cuda_fail(e, "kirchhoff_profile_read");
            total += ms;
            ++n;
            p->ev_pool.push_back(pr.second);
        }
        p->ev_pool.push_back(pr.first);
    }
    p->ev_open.clear();
    *kernel_ms = total;
    *timed_launches = n;
    return KH_OK;
}

long long kirchhoff_launch_count(kh_plan p) { return p ? p->launches : 0; }

const char* kirchhoff_last_error(void) { return g_err.c_str(); }

const char* kirchhoff_version(void) { return "kirchhoff-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// ------------------------------------------------------------------ helpers for the
// allocation-free entry point (kh_noalloc.cu) and the batched launch (kh_batch.cu): the same
// validation, geometry, tile choice, padding and binning launches as the plan path, writing
// into caller-supplied device buffers.
namespace kh {

kh_status noalloc_prepare(const kh_desc* d, GeomParams* g, TileShape* t)
{
    kh_status st = validate_desc(d);
    if (st != KH_OK) return st;
    *g = geom_of(*d);
    kh_plan_s tmp;   // host-only view for the tile choice; owns no device memory
    tmp.d = *d;
    *t = tile_of(&tmp);
    return prepare_linear(*d, *t, *g);
}

kh_status plan_geometry(const kh_plan_s* p, GeomParams* g, TileShape* t)
{
    *g = geom_of(p->d);
    *t = tile_of(p);
    return prepare_linear(p->d, *t, *g);
}

kh_status plan_check_headers(const kh_plan_s* p, int ntr, const float* sx, const float* sy,
                             const float* rx, const float* ry)
{
    return check_headers(p, ntr, sx, sy, rx, ry);
}

cudaError_t launch_pad(int ntr, int nt, long long ld, int esize, const void* src, void* dst, cudaStream_t s)
{
    const int blocks = (int)std::min<long long>(((long long)ntr * ld + 255) / 256, 65535);
    if (esize == 4)
        k_pad<float><<<std::max(blocks, 1), 256, 0, s>>>(ntr, nt, ld, (const float*)src, (float*)dst);
    else
        k_pad<unsigned short><<<std::max(blocks, 1), 256, 0, s>>>(ntr, nt, ld, (const unsigned short*)src,
                                                                 (unsigned short*)dst);
    return cudaGetLastError();
}

cudaError_t launch_pairs(int ntr, int nt, int ld, const void* src, void* dst, cudaStream_t s)
{
    if (ntr > 0)
        k_pairs<<<std::min(ntr, 1 << 20), 256, 0, s>>>(ntr, nt, ld, static_cast<const float*>(src),
                                                         static_cast<SamplePair*>(dst));
    return cudaGetLastError();
}

cudaError_t launch_gather(int ntr, const int* bin_start, int n_bins, const int* perm, const float* sx,
                          const float* sy, const float* rx, const float* ry, int dim, float4* hdr, float2* mid,
                          cudaStream_t s)
{
    k_gather<<<std::max(1, std::min((ntr + 255) / 256, 4096)), 256, 0, s>>>(bin_start, n_bins, perm, sx, sy, rx,
                                                                            ry, dim, hdr, mid);
    return cudaGetLastError();
}

cudaError_t noalloc_bin(int ntr, const float* sx, const float* sy, const float* rx, const float* ry,
                        const kh_desc& d, int* bin, int* perm, int* bin_start, float4* hdr,
                        float2* mid, cudaStream_t s)
{
    if (ntr > 0)
        k_bin<<<(ntr + 255) / 256, 256, 0, s>>>(ntr, sx, sy, rx, ry, d.dim, d.n_bins, d.bin_width, bin);
    k_sort<<<1, SORT_THREADS, 0, s>>>(ntr, d.n_bins, bin, perm, bin_start);
    k_gather<<<std::max(1, std::min((ntr + 255) / 256, 4096)), 256, 0, s>>>(bin_start, d.n_bins, perm,
                                                                            sx, sy, rx, ry, d.dim, hdr, mid);
    return cudaGetLastError();
}

}  // namespace kh
