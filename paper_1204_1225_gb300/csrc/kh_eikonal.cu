// Gridded model v(x, z) (KH_VEL_GRID): first-arrival traveltime tables per surface location and
// what the migration needs to read them.
//
// Sec. 3 takes the traveltimes of Eq. (1) from the high-frequency limit of ray theory, one path
// per source and image point: the first-arrival time, the solution of |grad T| = s (slowness
// s = 1/v) with T = 0 at the surface location.  Per location x_s, one CTA solves it on the node
// grid (ox + i h, j h) held in shared memory:
//   T = T0 + tau, T0 = s0 |x - x_s| (the exact time of the source's own slowness s0), so the
//   point-source singularity leaves the unknown tau (additive factorisation, Luo and Qian 2012);
//   Godunov upwind node equation with shifted neighbours c = tau_neighbour -/+ h dT0/dx, closed-form
//   solve; fast sweeping (Zhao 2005): four Gauss-Seidel orderings per round, rounds until the
//   largest decrease of a round is at most EK_TOL.
// Precision: tau, its neighbour values, the node equation and the round's decrease are FP64 (tau
// accumulates along every ray path); the shift h grad T0 = h s0 (x - x_s) / |x - x_s| is a
// geometric factor evaluated per update in FP32 from the FP64 offset (relative error a few
// 1e-7, i.e. a few 1e-9 s per node on a 20 m grid), and the node equation's square root is an
// FP32 estimate refined by one FP64 Newton step (relative error about 1e-15): the GPU's FP64
// pipe, a sixty-fourth of its FP32 rate, is kept for the accumulation.  Unreached nodes hold a
// large finite value, so an update from unreached neighbours needs no test: it cannot decrease.
// A pass sweeps anti-diagonals i' + j' = d (i', j' the indices in the pass's directions): a node
// depends on its upwind neighbours, which lie on diagonal d - 1, and reads its downwind ones from
// diagonal d + 1, not yet swept, exactly as in the sequential raster pass, so the nodes of one
// diagonal update in parallel with a barrier between diagonals and the result is the sequential
// one.  A node is recomputed only when one of its neighbours changed since it was last computed
// (one dirty bit per node): with unchanged neighbours its update would return the same value.
// The FP64 operations are single IEEE operations (explicit rounding intrinsics, no contraction).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "kh_device.cuh"
#include "kh_plan.h"

namespace kh {

constexpr int EK_THREADS = 256;
constexpr int EK_MAX_ROUNDS = 64;
// A round whose largest decrease is at most EK_TOL seconds ends the sweeps: later rounds would
// change the times by about 1 % of that, below the FP32 resolution of a stored time.
constexpr double EK_TOL = 1e-7;

static kh_status errf(kh_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return set_error(st, buf);
}

template <typename T>
static cudaError_t grow_ws(T*& ptr, size_t& cap, size_t n)
{
    if (n <= cap && ptr) return cudaSuccess;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    const size_t want = n + n / 4 + 16;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&ptr), want * sizeof(T));
    if (e == cudaSuccess) cap = want;
    return e;
}

constexpr double EK_UNREACHED = 1e30;   // seconds; ulp(1e30) dwarfs any shift or h s

// s = 1 / v, f h = h s and 2 (f h)^2 per node (FP64).
__global__ void k_grid_slowness(long long n, const float* __restrict__ v, double h, double* __restrict__ s,
                                double2* __restrict__ fh)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const double sq = __ddiv_rn(1.0, (double)v[q]);
        const double f = __dmul_rn(h, sq);
        s[q] = sq;
        fh[q] = make_double2(f, __dmul_rn(2.0, __dmul_rn(f, f)));
    }
}

// Upwind update of a node from its shifted neighbours a (x) and b (z); fh = (h s, 2 (h s)^2).
// Two-sided case: |a - b| < h s, so the discriminant lies in ((h s)^2, 2 (h s)^2] and its root is
// well conditioned: FP32 estimate y = rsqrt, r = disc y, then one Newton step in FP64.
__device__ __forceinline__ double ek_update(double a, double b, double2 fh)
{
    const double d = a - b;
    if (fabs(d) >= fh.x) return fmin(a, b) + fh.x;
    const double disc = fma(-d, d, fh.y);
    const float y = rsqrtf((float)disc);
    const double r0 = (double)((float)disc * y);
    const double r = fma(fma(-r0, r0, disc), (double)(0.5f * y), r0);
    return 0.5 * ((a + b) + r);
}

// One CTA per location: tau [nx][nz] FP64 and one dirty bit per node in shared memory.
__global__ void __launch_bounds__(EK_THREADS)
    k_eikonal(int nx, int nz, double ox, double h, const double* __restrict__ slow, const double2* __restrict__ fhs,
              const float* __restrict__ loc_x, int max_rounds, double tol, float* __restrict__ tables,
              int* __restrict__ rounds_out)
{
    extern __shared__ __align__(16) unsigned char ek_smem[];
    __shared__ double red[EK_THREADS / 32];
    const int n = nx * nz;
    double* tau = reinterpret_cast<double*>(ek_smem);
    unsigned* dirty = reinterpret_cast<unsigned*>(tau + n);
    float* dxf = reinterpret_cast<float*>(dirty + (n + 31) / 32);   // [nx]: x_i - x_s, FP64 rounded to FP32
    const int tid = threadIdx.x;
    const double xs = (double)loc_x[blockIdx.x];
    // s0: the surface row's slowness, linear between the two nodes around x_s
    const double u = __ddiv_rn(__dsub_rn(xs, ox), h);
    int i0 = (int)floor(u);
    i0 = i0 < 0 ? 0 : (i0 > nx - 2 ? nx - 2 : i0);
    const double f = __dsub_rn(u, (double)i0);
    const double sa = slow[(long long)i0 * nz], sb = slow[(long long)(i0 + 1) * nz];
    const double s0 = __dadd_rn(sa, __dmul_rn(f, __dsub_rn(sb, sa)));
    const double h2 = __dmul_rn(2.0, h);
    const float hs0f = (float)__dmul_rn(h, s0), hf = (float)h;
    for (int i = tid; i < nx; i += EK_THREADS) dxf[i] = (float)__dsub_rn(__dadd_rn(ox, __dmul_rn((double)i, h)), xs);
    // the columns of the source box, |x_i - x_s| <= 2 h (rows 0..2)
    const int ib0 = max(0, (int)floor(__ddiv_rn(__dsub_rn(xs, h2) - ox, h)) - 1);
    int bx0 = nx, bx1 = -1;
    for (int i = ib0; i < nx && i <= ib0 + 6; ++i)
        if (fabs(__dsub_rn(__dadd_rn(ox, __dmul_rn((double)i, h)), xs)) <= h2) {
            bx0 = min(bx0, i);
            bx1 = max(bx1, i);
        }
    // source box: straight ray with the trapezoid slowness, T = s0 dist + tau = dist (s0 + s) / 2
    for (int q = tid; q < n; q += EK_THREADS) {
        const int i = q / nz, j = q - i * nz;
        const double dx = __dsub_rn(__dadd_rn(ox, __dmul_rn((double)i, h)), xs);
        double t = EK_UNREACHED;
        if (i >= bx0 && i <= bx1 && j <= 2) {
            const double zj = __dmul_rn((double)j, h);
            const double dist = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(zj, zj)));
            t = __dmul_rn(dist, __dmul_rn(0.5, __dsub_rn(slow[q], s0)));
        }
        tau[q] = t;
    }
    for (int w = tid; w < (n + 31) / 32; w += EK_THREADS) dirty[w] = 0xffffffffu;
    __syncthreads();

    int rounds = -1;
    for (int r = 0; r < max_rounds; ++r) {
        double most = 0.0;
        for (int pass = 0; pass < 4; ++pass) {
            const bool iup = (pass == 0 || pass == 3), jup = pass < 2;
            for (int d = 0; d <= nx + nz - 2; ++d) {
                const int lo = d - (nz - 1) > 0 ? d - (nz - 1) : 0, hi = d < nx - 1 ? d : nx - 1;
                for (int ii = lo + tid; ii <= hi; ii += EK_THREADS) {
                    const int jj = d - ii;
                    const int i = iup ? ii : nx - 1 - ii, j = jup ? jj : nz - 1 - jj;
                    const int q = i * nz + j;
                    const unsigned bit = 1u << (q & 31);
                    if (!(dirty[q >> 5] & bit)) continue;
                    atomicAnd(&dirty[q >> 5], ~bit);
                    if (j <= 2 && i >= bx0 && i <= bx1) continue;   // the source box is fixed
                    // h grad T0 = h s0 (dx, z) / r in FP32
                    const float xf = dxf[i], zf = (float)j * hf;
                    const float gf = hs0f * rsqrtf(fmaf(xf, xf, zf * zf));
                    const double gx = (double)(gf * xf), gz = (double)(gf * zf);
                    const double cl = i > 0 ? tau[q - nz] - gx : EK_UNREACHED;
                    const double cr = i < nx - 1 ? tau[q + nz] + gx : EK_UNREACHED;
                    const double cu = j > 0 ? tau[q - 1] - gz : EK_UNREACHED;
                    const double cd = j < nz - 1 ? tau[q + 1] + gz : EK_UNREACHED;
                    const double t = ek_update(fmin(cl, cr), fmin(cu, cd), fhs[q]);
                    const double old = tau[q];
                    if (t < old) {
                        most = fmax(most, old - t);
                        tau[q] = t;
                        if (i > 0) atomicOr(&dirty[(q - nz) >> 5], 1u << ((q - nz) & 31));
                        if (i < nx - 1) atomicOr(&dirty[(q + nz) >> 5], 1u << ((q + nz) & 31));
                        if (j > 0) atomicOr(&dirty[(q - 1) >> 5], 1u << ((q - 1) & 31));
                        if (j < nz - 1) atomicOr(&dirty[(q + 1) >> 5], 1u << ((q + 1) & 31));
                    }
                }
                __syncthreads();
            }
        }
        // the round's largest decrease (a max: the same in any order)
        for (int o = 16; o > 0; o >>= 1) most = fmax(most, __shfl_xor_sync(0xffffffffu, most, o));
        if ((tid & 31) == 0) red[tid >> 5] = most;
        __syncthreads();
        double m = red[0];
        for (int w = 1; w < EK_THREADS / 32; ++w) m = fmax(m, red[w]);
        __syncthreads();
        if (m <= tol) {
            rounds = r + 1;
            break;
        }
    }
    // tables [row][column] (x fastest): the migration's warps read consecutive nodes of a row
    float* out = tables + (long long)blockIdx.x * n;
    for (int e = tid; e < n; e += EK_THREADS) {
        const int j = e / nx, i = e - j * nx, q = i * nz + j;
        const double dx = __dsub_rn(__dadd_rn(ox, __dmul_rn((double)i, h)), xs);
        const double zj = __dmul_rn((double)j, h);
        const double r0 = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(zj, zj)));
        out[e] = __double2float_rn(__dadd_rn(__dmul_rn(s0, r0), tau[q]));
    }
    if (tid == 0) rounds_out[blockIdx.x] = rounds;
}

// Location index of each sorted trace's source and receiver (exact match in the increasing
// list), written over the y and receiver-y slots of the 2D headers as int bits; -1 and the
// plan's status bit when a position has no table.
__device__ __forceinline__ int find_loc(const float* __restrict__ loc, int nloc, float x)
{
    int lo = 0, hi = nloc - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const float v = loc[mid];
        if (v == x) return mid;
        if (v < x) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

__global__ void k_grid_locs(const int* __restrict__ bin_start, int n_bins, float4* __restrict__ hdr,
                            const float* __restrict__ loc, int nloc, int* __restrict__ status)
{
    const int n = bin_start[n_bins];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        float4 h = hdr[k];
        const int ls = find_loc(loc, nloc, h.x), lr = find_loc(loc, nloc, h.z);
        if (ls < 0 || lr < 0) atomicOr(status, STATUS_NO_TABLE);
        h.y = __int_as_float(ls);
        h.w = __int_as_float(lr);
        hdr[k] = h;
    }
}

// Per (location, tile of the launch): the smallest and largest node value over the node columns
// and rows the tile's image points interpolate between (every interpolated time of the tile lies
// between them).  One warp per pair.
__global__ void k_grid_bounds(GeomParams g, TileShape ts, int nloc, float2* __restrict__ bnd)
{
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int ntiles = ts.tiles_x * ts.tiles_y * ts.tiles_z;
    if (wid >= (long long)nloc * ntiles) return;
    const int l = (int)(wid / ntiles);
    int t = (int)(wid - (long long)l * ntiles);
    const int tzi = t % ts.tiles_z;
    t /= ts.tiles_z;
    const int txi = t % ts.tiles_x;
    const int x0 = txi * ts.cx, z0 = tzi * ts.cz * NZ;
    const int xe = min(x0 + ts.cx, g.nx) - 1, ze = min(z0 + ts.cz * NZ, g.nz) - 1;
    float lo = __int_as_float(0x7f800000), hi = -lo;
    if (x0 <= xe && z0 <= ze) {
        const int ca = grid_col(g, x0, nullptr), cb = grid_col(g, xe, nullptr) + 1;
        const int ra = g.gzoff + z0 / g.tm, rb = min(g.gzoff + ze / g.tm + 1, g.gnz - 1);
        const int nr = rb - ra + 1, cnt = (cb - ca + 1) * nr;
        const float* T = g.gtab + (long long)l * g.gstride;
        for (int e = lane; e < cnt; e += 32) {
            const float v = T[(long long)(ra + e % nr) * g.gnx + ca + e / nr];
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) bnd[wid] = make_float2(lo, hi);
}

// Shared memory of the solver's CTA: tau (FP64), one dirty bit per node, and the FP32 column offsets.
static size_t grid_smem_bytes(int nx, int nz)
{
    const size_t n = (size_t)nx * nz;
    return n * sizeof(double) + (n + 31) / 32 * sizeof(unsigned) + (size_t)nx * sizeof(float);
}
constexpr size_t EK_SMEM_MAX = 227 * 1024 - 256;   // dynamic shared memory of one CTA, with room for the static part

// Node grid rules of a descriptor: m from h, the node row of the first image depth, and the rows
// a migration needs.  Returns KH_OK or an error with its message set.
static kh_status grid_rules(const kh_desc& d, const kh_grid& G, int* m_out, int* zoff_out)
{
    if (d.vel != KH_VEL_GRID || d.dim != 2) return errf(KH_ERR_INVALID_ARG, "the plan is not a 2D KH_VEL_GRID plan");
    if (G.nx < 2 || G.nz < 2) return errf(KH_ERR_INVALID_ARG, "grid needs nx, nz >= 2 (got %d x %d)", G.nx, G.nz);
    if ((long long)G.nx * G.nz > MAX_GRID_NODES || grid_smem_bytes(G.nx, G.nz) > EK_SMEM_MAX)
        return errf(KH_ERR_INVALID_ARG, "grid of %d x %d nodes exceeds %d nodes (one CTA's shared memory); "
                    "use a coarser h", G.nx, G.nz, MAX_GRID_NODES);
    if (!(G.h > 0) || !std::isfinite(G.h) || !std::isfinite(G.ox)) return errf(KH_ERR_INVALID_ARG, "grid h must be > 0");
    const double r = G.h / d.dz;
    const int m = (int)std::lround(r);
    if ((m != 1 && m != 2 && m != 4) || std::fabs(G.h - m * d.dz) > 1e-9 * G.h)
        return errf(KH_ERR_INVALID_ARG, "grid h = %g must be 1, 2 or 4 times the image dz = %g", G.h, d.dz);
    const double zr = d.oz / G.h;
    const long long zoff = std::llround(zr);
    if (zoff < 0 || std::fabs(zr - (double)zoff) > 1e-9 * std::max(1.0, std::fabs(zr)))
        return errf(KH_ERR_INVALID_ARG, "image oz = %g must be a non-negative multiple of the grid h = %g", d.oz, G.h);
    const long long need = zoff + (long long)((d.nz + NZ - 1) / NZ) * NZ / m + 1;
    if (G.nz < need) return errf(KH_ERR_INVALID_ARG, "grid needs at least %lld rows for the image depths (got %d)", need, G.nz);
    const double x_last = d.ox + (d.nx - 1) * d.dx, g_last = G.ox + (G.nx - 1) * G.h;
    if (G.ox > d.ox || g_last < x_last)
        return errf(KH_ERR_INVALID_ARG, "grid columns [%g, %g] do not cover the image columns [%g, %g]", G.ox, g_last,
                    d.ox, x_last);
    *m_out = m;
    *zoff_out = (int)zoff;
    return KH_OK;
}

kh_status grid_prepare(kh_plan_s* p, const TileShape& t, GeomParams& g, cudaStream_t s)
{
    if (p->grid_nloc <= 0 || !p->ws_gtab)
        return errf(KH_ERR_INVALID_ARG, "KH_VEL_GRID plan has no traveltime tables: call kirchhoff_grid_tables first");
    const int ntiles = t.tiles_x * t.tiles_y * t.tiles_z;
    cudaError_t e = grow_ws(p->ws_gbnd, p->cap_gbnd, (size_t)p->grid_nloc * ntiles);
    if (e != cudaSuccess) return set_cuda_error(e, "workspace (table bounds)");
    g.gtab = p->ws_gtab;
    g.gnx = p->grid.nx;
    g.gnz = p->grid.nz;
    g.gstride = (long long)p->grid.nx * p->grid.nz;
    g.gox = p->grid.ox;
    g.gh = p->grid.h;
    g.gzoff = p->grid_zoff;
    g.tm = p->grid_m;
    g.gbnd = p->ws_gbnd;
    g.gtiles = ntiles;
    g.tslack = 0.f;
    g.C1 = (float)(1.0 / p->d.dt);
    g.C1lo = 0.f;
    g.c0 = -p->d.t0 / p->d.dt - 0.5;
    k_grid_locs<<<2 * 152, 256, 0, s>>>(p->ws_bin_start, p->d.n_bins, p->ws_hdr, p->ws_gloc, p->grid_nloc,
                                         p->ws_status);
    const long long warps = (long long)p->grid_nloc * ntiles;
    k_grid_bounds<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(g, t, p->grid_nloc, p->ws_gbnd);
    p->launches += 2;
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e, "grid table kernels");
    return KH_OK;
}

}  // namespace kh

using namespace kh;

extern "C" {

kh_status kirchhoff_grid_layout(const kh_desc* d, int m, double xmin, double xmax, int margin, kh_grid* out)
{
    if (!d || !out) return errf(KH_ERR_INVALID_ARG, "desc/out is NULL");
    if (m != 1 && m != 2 && m != 4) return errf(KH_ERR_INVALID_ARG, "m must be 1, 2 or 4");
    if (margin < 0 || !std::isfinite(xmin) || !std::isfinite(xmax) || xmin > xmax)
        return errf(KH_ERR_INVALID_ARG, "need margin >= 0 and finite xmin <= xmax");
    if (!(d->dz > 0) || !(d->dx > 0) || d->nx < 1 || d->nz < 1) return errf(KH_ERR_INVALID_ARG, "bad image grid");
    const double h = m * d->dz;
    const double lo = std::min(xmin, d->ox), hi = std::max(xmax, d->ox + (d->nx - 1) * d->dx);
    const long long i0 = (long long)std::floor(lo / h) - margin, i1 = (long long)std::ceil(hi / h) + margin;
    const long long zoff = std::llround(d->oz / h);
    kh_grid G;
    G.nx = (int)(i1 - i0 + 1);
    G.nz = (int)(zoff + (long long)((d->nz + NZ - 1) / NZ) * NZ / m + 1);
    G.ox = (double)i0 * h;
    G.h = h;
    int mm, zz;
    const kh_status st = grid_rules(*d, G, &mm, &zz);
    if (st != KH_OK) return st;
    *out = G;
    return KH_OK;
}

kh_status kirchhoff_grid_tables(kh_plan p, const kh_grid* grid, const float* v, int nloc, const float* loc_x,
                                void* cuda_stream)
{
    if (!p || !grid || !v || !loc_x) return errf(KH_ERR_INVALID_ARG, "plan/grid/v/loc_x is NULL");
    if (nloc < 1) return errf(KH_ERR_INVALID_ARG, "nloc must be >= 1");
    int m = 0, zoff = 0;
    kh_status st = grid_rules(p->d, *grid, &m, &zoff);
    if (st != KH_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const kh_grid G = *grid;
    const long long n = (long long)G.nx * G.nz;
    // host checks of the model and the locations (a setup call: one copy each)
    std::vector<float> hv((size_t)n), hl((size_t)nloc);
    cudaError_t e = cudaMemcpyAsync(hv.data(), v, n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hl.data(), loc_x, nloc * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_grid_tables (inputs)");
    for (long long q = 0; q < n; ++q)
        if (!(hv[q] > 0.f) || !std::isfinite(hv[q]))
            return errf(KH_ERR_INVALID_ARG, "v must be finite and > 0 (node %lld: %g)", q, (double)hv[q]);
    const double g_last = G.ox + (G.nx - 1) * G.h;
    for (int l = 0; l < nloc; ++l) {
        if (!std::isfinite(hl[l]) || (double)hl[l] < G.ox || (double)hl[l] > g_last)
            return errf(KH_ERR_INVALID_ARG, "location %d (x = %g) is outside the grid columns [%g, %g]", l, (double)hl[l],
                        G.ox, g_last);
        if (l > 0 && !(hl[l] > hl[l - 1])) return errf(KH_ERR_INVALID_ARG, "loc_x must be strictly increasing");
    }
    if ((e = grow_ws(p->ws_gtab, p->cap_gtab, (size_t)nloc * n)) != cudaSuccess ||
        (e = grow_ws(p->ws_gloc, p->cap_gloc, (size_t)nloc)) != cudaSuccess ||
        (e = grow_ws(p->ws_grounds, p->cap_grounds, (size_t)nloc)) != cudaSuccess ||
        (e = grow_ws(p->ws_gslow, p->cap_gslow, (size_t)(3 * n + 2))) != cudaSuccess)
        return set_cuda_error(e, "workspace (traveltime tables)");
    p->grid_nloc = 0;
    e = cudaMemcpyAsync(p->ws_gloc, loc_x, nloc * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_grid_tables (locations)");
    // (h s, 2 (h s)^2) per node after s, at an even offset (16-byte aligned double2)
    double2* fhs = reinterpret_cast<double2*>(p->ws_gslow + (n + 1) / 2 * 2);
    k_grid_slowness<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(n, v, G.h, p->ws_gslow, fhs);
    const size_t smem = grid_smem_bytes(G.nx, G.nz);
    e = cudaFuncSetAttribute(k_eikonal, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        k_eikonal<<<nloc, EK_THREADS, smem, s>>>(G.nx, G.nz, G.ox, G.h, p->ws_gslow, fhs, p->ws_gloc, EK_MAX_ROUNDS, EK_TOL,
                                                  p->ws_gtab, p->ws_grounds);
        e = cudaGetLastError();
    }
    p->launches += 2;
    std::vector<int> rounds((size_t)nloc);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rounds.data(), p->ws_grounds, nloc * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_cuda_error(e, "eikonal solver");
    for (int l = 0; l < nloc; ++l)
        if (rounds[l] < 0)
            return errf(KH_ERR_UNSUPPORTED, "location %d (x = %g) did not settle in %d rounds of sweeps", l, (double)hl[l],
                        EK_MAX_ROUNDS);
    p->grid = G;
    p->grid_nloc = nloc;
    p->grid_m = m;
    p->grid_zoff = zoff;
    return KH_OK;
}

kh_status kirchhoff_grid_read(kh_plan p, float* tables, int* rounds, int* nloc, void* cuda_stream)
{
    if (!p) return errf(KH_ERR_INVALID_ARG, "plan is NULL");
    if (p->grid_nloc <= 0) return errf(KH_ERR_INVALID_ARG, "the plan has no traveltime tables");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const size_t n = (size_t)p->grid.nx * p->grid.nz * p->grid_nloc;
    cudaError_t e = cudaSuccess;
    if (tables) e = cudaMemcpyAsync(tables, p->ws_gtab, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && rounds)
        e = cudaMemcpyAsync(rounds, p->ws_grounds, p->grid_nloc * sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_grid_read");
    if (nloc) *nloc = p->grid_nloc;
    return KH_OK;
}

}  // extern "C"
