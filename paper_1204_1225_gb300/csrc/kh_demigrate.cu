// Demigration (the transpose of Eq. 1: each image value is spread back onto the traces at
// the two samples around t = T_s + T_r, Sec. 3 read from the data side).
//
// Trace-stationary: one thread owns one trace; a CTA owns 128 consecutive traces of one
// offset bin and a 1/P share of the image tiles (tiles i with i % P == part).  For each tile
// the CTA stages the tile's image values and per-z constants in shared memory; every lane
// evaluates tau for its own trace at every image point of the tile (the same FP64-reference
// + FP32-delta evaluation as the migration) and adds W (1-f) m and W f m into its own column
// of a lane-interleaved window buffer [row][lane] (bank = lane: no conflicts, no atomics).
// The sample index is floor(tau - lo) (adding 1.5 * 2^23 rounded down), as in the migration.
// After the tile the lane adds its window into its own row of the part's partial-trace
// buffer.  A second kernel sums the P partial buffers in a fixed order into the output.
//
// Linear v(z): tau - lo adds per-leg logarithms (as the migration), and lanes whose traces share
// a source position share the source leg of every image point.  When a warp's traces come from
// at most two source positions (shot-ordered traces), the lanes first evaluate each group's
// source leg at 32 depths of the column cooperatively into shared memory, then every lane
// evaluates only its receiver leg per point; otherwise each lane evaluates both legs.
#include "kh_tau.cuh"

namespace kh {

constexpr int DM_WARPS = 4;
constexpr int DM_THREADS = DM_WARPS * 32;
constexpr int DM_ROWS = 96;     // window rows per lane (the host sizes tiles to fit)
constexpr int DM_TILE = 1024;   // image samples per tile
constexpr int DM_MAXZ = 64;     // depth samples per tile

// The depth loops read the next depth's inputs one depth ahead, past the last depth on the last
// one (the value is not used): each per-depth array has one entry to spare.
struct __align__(16) DmSmem {
    float buf[DM_WARPS][DM_ROWS][32];
    float mt[DM_TILE + 1];
    float4 zc[DM_MAXZ + 1];
    float z2[DM_MAXZ + 1];
    float2 src[DM_WARPS][2][33];   // per warp and source group: (C1 ln(1 + rho_s), sqrt(q_s))
};

static_assert(DM_ROWS == DM_ROWS_HOST, "window rows");

template <int VEL, int WGT, bool FAST, int LPT>
__global__ void __launch_bounds__(DM_THREADS, 4)
    k_demigrate(GeomParams g, DmTile dt, TraceSet tr, const float* __restrict__ image,
                float* __restrict__ partial, int* status)
{
    constexpr int WB = WGT & 3;                 // the weight (KH_W_*)
    constexpr bool AA = (WGT & W_AA) != 0;      // operator anti-aliasing compiled in
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DmSmem& S = *reinterpret_cast<DmSmem*>(smem_raw);
    const int b = blockIdx.y, part = blockIdx.z;
    const int nvalid = tr.bin_start[g.n_bins];
    const int tb = tr.bin_start[b] + blockIdx.x * DM_THREADS;
    const int te = tr.bin_start[b + 1];
    if (tb >= te) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = tb + threadIdx.x;
    const bool has = k < te;
    float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 mid = make_float2(0.f, 0.f);
    if (has) {
        h = tr.hdr[k];
        mid = tr.mid[k];
    }
    float* prow = partial + ((long long)part * nvalid + (has ? k : 0)) * g.nt;
    const double inv_kdt = (VEL == VK_LINEAR) ? 1.0 / (g.kabs * g.dtd) : 0.0;
    const int n_tiles = dt.tiles_x * dt.tiles_y * dt.tiles_z;
    // the warp's source groups: lane 0's source (A) and the first other one (B); lanes without a
    // trace count as A
    const unsigned FULL = 0xffffffffu;
    const unsigned s0x = __shfl_sync(FULL, __float_as_uint(h.x), 0), s0y = __shfl_sync(FULL, __float_as_uint(h.y), 0);
    const unsigned kx = has ? __float_as_uint(h.x) : s0x, ky = has ? __float_as_uint(h.y) : s0y;
    const bool inA = kx == s0x && ky == s0y;
    const unsigned notA = __ballot_sync(FULL, !inA);
    const int lb = notA ? __ffs(notA) - 1 : 0;
    const unsigned s1x = __shfl_sync(FULL, kx, lb), s1y = __shfl_sync(FULL, ky, lb);
    const bool grouped = __all_sync(FULL, inA || (kx == s1x && ky == s1y));
    const int my_group = inA ? 0 : 1, ngroups = notA ? 2 : 1;
    const int ncol = dt.tx * dt.ty;

    for (int ti = part; ti < n_tiles; ti += dt.parts) {
        int t = ti;
        const int tzi = t % dt.tiles_z;
        t /= dt.tiles_z;
        const int txi = t % dt.tiles_x, tyi = t / dt.tiles_x;
        const int x0 = txi * dt.tx, y0 = tyi * dt.ty, z0 = tzi * dt.tz;
        const TileBox box = tile_box(g, x0, y0, z0, dt.tx, dt.ty, dt.tz);

        // this lane's window and FP64 reference for the tile
        bool ok = has;
        if (ok && g.use_aperture) {
            const float ax = fmaxf(fmaxf(box.xlo - mid.x, mid.x - box.xhi), 0.f);
            const float ay = fmaxf(fmaxf(box.ylo - mid.y, mid.y - box.yhi), 0.f);
            ok = ax * ax + ay * ay <= g.A2cull;
        }
        int lo = 0, hi = 0;
        if (ok) ok = trace_window(h, box, VEL, g, lo, hi);
        const int rows = hi - lo + 2;
        if (ok && rows > DM_ROWS) {   // the host sizes tiles so this cannot happen
            atomicOr(status, 2);
            ok = false;
        }
        if (!__syncthreads_or(ok)) continue;

        // per-lane FP64 reference: (R_c^2, (q_c + 2)/u_c, w_c, 1/u_c) per leg, as the migration
        float4 rs = make_float4(0.f, 0.f, 0.f, 0.f), rr = rs;
        float4 ah = h;
        double tau_ref = -g.t0d / g.dtd;
        if constexpr (VEL == VK_LINEAR) {
            // every lane with a trace (not only those the tile keeps): a source group takes its
            // source leg's reference from its first lane
            if (has) {
                LegRef ls_, lr_;
                float qis = 0.f, qir = 0.f;
                const double ls = leg_reference(box.cx, box.cy, box.cz, h.x, h.y, g, ls_, &qis);
                const double lr = leg_reference(box.cx, box.cy, box.cz, h.z, h.w, g, lr_, &qir);
                rs = make_float4(ls_.Rc2, qis, ls_.wc, ls_.iuc);
                rr = make_float4(lr_.Rc2, qir, lr_.wc, lr_.iuc);
                tau_ref = __dadd_rn(tau_ref, __dmul_rn(__dadd_rn(ls, lr), inv_kdt));
                ah = make_float4((float)(box.cx - 2.0 * h.x), (float)(box.cy - 2.0 * h.y),
                                 (float)(box.cx - 2.0 * h.z), (float)(box.cy - 2.0 * h.w));
            }
        }
        // window-relative time th = tau - lo; valid iff 0 <= th <= hi - lo
        const float c0rel = (float)(tau_ref - (double)lo);
        // anti-aliasing with v0 + k z: the tile's first depth and the depth step
        const float aa_z0 = (float)grid_coord(g.oz, z0, g.dz), aa_dz = (float)g.dz;
        const float lim = (float)(hi - lo);
        const float cmid = 0.5f * lim, chalf = 0.5f * lim + EDGE_EPS;

        // stage the tile's image values (zero outside the grid) and per-z constants
        for (int p = threadIdx.x; p < ncol * dt.tz; p += DM_THREADS) {
            const int iz = p % dt.tz, c = p / dt.tz;
            const int ix = x0 + c % dt.tx, iy = y0 + c / dt.tx, zz = z0 + iz;
            float v = 0.f;
            if (ix < g.nx && iy < g.ny && zz < g.nz)
                v = image[(((long long)b * g.ny + iy) * g.nx + ix) * g.nz + zz];
            S.mt[p] = v;
        }
        for (int i = threadIdx.x; i < dt.tz; i += DM_THREADS) {
            const double z = grid_coord(g.oz, z0 + i, g.dz);
            if constexpr (VEL == VK_LINEAR) {
                float gamma;
                S.zc[i] = z_constants_m(z, box.cz, g, gamma);
                S.z2[i] = gamma;
            } else {
                const float wz = (g.weight == 1 && fabs(z) >= 1e-6 * fabs(g.dz)) ? (float)(z * g.wscale) : 0.f;
                S.zc[i] = make_float4((float)(z * z), wz, (float)z, fabs(z) >= 1e-6 * fabs(g.dz) ? 1.f : 0.f);
            }
        }
        // clear this warp's rows in use
        const int wrows = __reduce_max_sync(0xffffffffu, ok ? rows : 0);
        for (int r = 0; r < wrows; ++r) S.buf[warp][r][lane] = 0.f;
        __syncthreads();

        if (__any_sync(0xffffffffu, ok)) {
            float* col0 = &S.buf[warp][0][lane];
            for (int c = 0; c < ncol; ++c) {
                const int ix = x0 + c % dt.tx, iy = y0 + c / dt.tx;
                bool inside = ok && ix < g.nx && iy < g.ny;
                const float cxf = col_coord(g.ox, ix, g.dx);
                const float cyf = (g.dim == 3) ? col_coord(g.oy, iy, g.dy) : 0.f;
                if (inside && g.use_aperture) inside = in_aperture(cxf, cyf, mid.x, mid.y, g.A2);
                const float tp = (inside && g.use_taper) ? aperture_taper(cxf, cyf, mid.x, mid.y, g) : 1.f;
                const float chc = inside ? chalf : -1.f;
                const float* mcol = &S.mt[c * dt.tz];
                if constexpr (VEL == VK_CONST) {
                    const float dxs = cxf - h.x, dys = cyf - h.y;
                    const float dxr = cxf - h.z, dyr = cyf - h.w;
                    const float dhs2 = fmaf(dxs, dxs, dys * dys);
                    const float dhr2 = fmaf(dxr, dxr, dyr * dyr);
                    // the next depth's inputs read ahead of this depth's window stores (as below)
                    float4 zc = S.zc[0];   // (z^2, w_z, z, 1 off the surface row)
                    float mz = mcol[0];
#pragma unroll 4
                    for (int iz = 0; iz < dt.tz; ++iz) {
                        const float Rs = hsqrt<FAST>(dhs2 + zc.x);
                        const float Rr = hsqrt<FAST>(dhr2 + zc.x);
                        const float Ssum = Rs + Rr;
                        const float th = fmaf(Ssum, g.C1, fmaf(Ssum, g.C1lo, c0rel));
                        const float tc = fmaxf(th, 0.f);   // within EDGE_EPS below 0: the first row
                        const float tm = __fadd_rd(tc, MAGIC);                 // MAGIC + floor(tc)
                        const float f = __fsub_rn(tc, __fsub_rn(tm, MAGIC));
                        const bool v = fabsf(th - cmid) <= chc;
                        float W = (WB == 1) ? zc.y * Ssum
                                  : (WB == 2) ? (zc.w != 0.f ? ta_weight<FAST>(zc.z, Rs, Rr, g.dim == 3) : 0.f)
                                               : 1.f;
                        if constexpr (AA) W *= aa_weight<FAST>(g.aa_c, dxs, dys, dxr, dyr, Rs, Rr);
                        const float wm = v ? tp * W * mz : 0.f;
                        const int row = v ? __float_as_int(tm) - MAGIC_BITS : 0;
                        const float a1 = wm * f;
                        zc = S.zc[iz + 1];
                        mz = mcol[iz + 1];
                        col0[row * 32] += wm - a1;
                        col0[row * 32 + 32] += a1;
                    }
                } else {
                    const float dxc = (float)((g.ox + ix * g.dx) - box.cx);
                    const float dyc = (g.dim == 3) ? (float)((g.oy + iy * g.dy) - box.cy) : 0.f;
                    const float dPr = fmaf(dxc, cxf + ah.z, dyc * (cyf + ah.w));
                    const float exr = cxf - h.z, eyr = cyf - h.w;
                    const float dhr2 = fmaf(exr, exr, eyr * eyr);
                    if (grouped) {
                        for (int hz = 0; hz < dt.tz; hz += 32) {
                            // each group's source leg at depths hz + lane (group data is uniform:
                            // taken from the group's first lane)
                            for (int gi = 0; gi < ngroups; ++gi) {
                                const int src_lane = gi ? lb : 0;
                                const float4 rsg = make_float4(__shfl_sync(FULL, rs.x, src_lane), __shfl_sync(FULL, rs.y, src_lane),
                                                               __shfl_sync(FULL, rs.z, src_lane), __shfl_sync(FULL, rs.w, src_lane));
                                const float ahx = __shfl_sync(FULL, ah.x, src_lane), ahy = __shfl_sync(FULL, ah.y, src_lane);
                                const float sgx = __shfl_sync(FULL, h.x, src_lane), sgy = __shfl_sync(FULL, h.y, src_lane);
                                const int izc = hz + lane;
                                if (izc < dt.tz) {
                                    const float dPs = fmaf(dxc, cxf + ahx, dyc * (cyf + ahy));
                                    const float exs = cxf - sgx, eys = cyf - sgy;
                                    const float dhs2 = fmaf(exs, exs, eys * eys);
                                    float sqs = 0.f;
                                    const float rho_s = leg_delta_m<WB, FAST>(dPs, dhs2, S.zc[izc], rsg, sqs);
                                    S.src[warp][gi][lane] = make_float2(leg_log<LPT>(rho_s, g, 0.f), sqs);
                                }
                            }
                            __syncwarp();
                            const float2* sl = &S.src[warp][my_group][0];
                            const int nzh = min(32, dt.tz - hz);
                            // the next depth's shared-memory inputs are read before this depth's
                            // window stores (which the compiler cannot reorder them past), so that
                            // its arithmetic overlaps the read-modify-write of this one
                            float4 zk = S.zc[hz];   // (alpha, alpha kappa, alpha dz2, alpha z^2)
                            float2 sv = sl[0];      // (C1 ln(1 + rho_s), sqrt(q_s))
                            float mz = mcol[hz], wz = S.z2[hz];
#pragma unroll 4
                            for (int j = 0; j < nzh; ++j) {
                                float sqr = 0.f;
                                const float rho_r = leg_delta_m<WB, FAST>(dPr, dhr2, zk, rr, sqr);
                                const float th = leg_log<LPT>(rho_r, g, c0rel + sv.x);
                                const float tc = fmaxf(th, 0.f);   // within EDGE_EPS below 0: the first row
                                const float tm = __fadd_rd(tc, MAGIC);                 // MAGIC + floor(tc)
                                const float f = __fsub_rn(tc, __fsub_rn(tm, MAGIC));
                                const bool v = fabsf(th - cmid) <= chc;
                                float W = (WB == 1) ? wz * (sv.y + sqr) : 1.f;
                                if constexpr (AA) {   // anti-aliasing: both legs' slowness factors at this depth
                                    const float zi = fmaf((float)(hz + j), aa_dz, aa_z0);
                                    const float vv = fmaf(g.aa_v0k, zi, g.aa_v0sq);
                                    const float exs = cxf - h.x, eys = cyf - h.y;
                                    const float fs = aa_leg_lin(fmaf(zi, zi, fmaf(exs, exs, eys * eys)), vv, g.aa_kq);
                                    const float fr = aa_leg_lin(fmaf(zi, zi, dhr2), vv, g.aa_kq);
                                    W *= aa_weight_r(g.aa_c, exs, eys, exr, eyr, fs, fr);
                                }
                                const float wm = v ? tp * W * mz : 0.f;
                                const int row = v ? __float_as_int(tm) - MAGIC_BITS : 0;
                                const float a1 = wm * f;
                                zk = S.zc[hz + j + 1];
                                sv = sl[j + 1];
                                mz = mcol[hz + j + 1];
                                wz = S.z2[hz + j + 1];
                                col0[row * 32] += wm - a1;
                                col0[row * 32 + 32] += a1;
                            }
                            __syncwarp();
                        }
                    } else {
                        const float dPs = fmaf(dxc, cxf + ah.x, dyc * (cyf + ah.y));
                        const float exs = cxf - h.x, eys = cyf - h.y;
                        const float dhs2 = fmaf(exs, exs, eys * eys);
                        // the next depth's inputs read ahead of this depth's window stores (as above)
                        float4 zk = S.zc[0];   // (alpha, alpha kappa, alpha dz2, alpha z^2)
                        float mz = mcol[0], wz = S.z2[0];
#pragma unroll 4
                        for (int iz = 0; iz < dt.tz; ++iz) {
                            float sqs = 0.f, sqr = 0.f;
                            const float rho_s = leg_delta_m<WB, FAST>(dPs, dhs2, zk, rs, sqs);
                            const float rho_r = leg_delta_m<WB, FAST>(dPr, dhr2, zk, rr, sqr);
                            const float th = leg_log<LPT>(rho_r, g, c0rel + leg_log<LPT>(rho_s, g, 0.f));
                            const float tc = fmaxf(th, 0.f);   // within EDGE_EPS below 0: the first row
                            const float tm = __fadd_rd(tc, MAGIC);                 // MAGIC + floor(tc)
                            const float f = __fsub_rn(tc, __fsub_rn(tm, MAGIC));
                            const bool v = fabsf(th - cmid) <= chc;
                            float W = (WB == 1) ? wz * (sqs + sqr) : 1.f;
                            if constexpr (AA) {   // anti-aliasing (as above)
                                const float zi = fmaf((float)iz, aa_dz, aa_z0);
                                const float vv = fmaf(g.aa_v0k, zi, g.aa_v0sq);
                                const float fs = aa_leg_lin(fmaf(zi, zi, dhs2), vv, g.aa_kq);
                                const float fr = aa_leg_lin(fmaf(zi, zi, dhr2), vv, g.aa_kq);
                                W *= aa_weight_r(g.aa_c, exs, eys, exr, eyr, fs, fr);
                            }
                            const float wm = v ? tp * W * mz : 0.f;
                            const int row = v ? __float_as_int(tm) - MAGIC_BITS : 0;
                            const float a1 = wm * f;
                            zk = S.zc[iz + 1];
                            mz = mcol[iz + 1];
                            wz = S.z2[iz + 1];
                            col0[row * 32] += wm - a1;
                            col0[row * 32 + 32] += a1;
                        }
                    }
                }
            }
        }
        __syncwarp();
        if (ok) {
            const int nr = min(rows, g.nt - lo);
            for (int r = 0; r < nr; ++r) prow[lo + r] += S.buf[warp][r][lane];
        }
        __syncthreads();
    }
}

// out[perm[k]][t] = sum over parts p of partial[p][k][t] (fixed order); rows of traces
// without an offset bin were zeroed before.
__global__ void k_dm_reduce(const int* __restrict__ bin_start, int n_bins, const int* __restrict__ perm,
                            const float* __restrict__ partial, int parts, int nt,
                            float* __restrict__ out)
{
    const int nvalid = bin_start[n_bins];
    const long long total = (long long)nvalid * nt;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long k = i / nt, t = i - k * nt;
        float s = 0.f;
        for (int p = 0; p < parts; ++p) s += partial[((long long)p * nvalid + k) * nt + t];
        out[(long long)perm[k] * nt + t] = s;
    }
}

size_t demigrate_smem_bytes() { return sizeof(DmSmem); }

template <int VEL, int WGT, bool FAST>
static cudaError_t dm_launch_t(const GeomParams& g, const DmTile& dt, const TraceSet& tr,
                               const float* image, float* partial, int* status, int max_chunks,
                               cudaStream_t s)
{
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(DmSmem));
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)max_chunks, (unsigned)g.n_bins, (unsigned)dt.parts);
        kern<<<grid, DM_THREADS, sizeof(DmSmem), s>>>(g, dt, tr, image, partial, status);
        return cudaGetLastError();
    };
    if constexpr (VEL == VK_LINEAR)
        return with_lg<FAST>(g.lg_terms, [&](auto L) { return go(k_demigrate<VEL, WGT, FAST, decltype(L)::value>); });
    else
        return go(k_demigrate<VEL, WGT, FAST, LP_SHORT>);
}

cudaError_t launch_demigrate(const GeomParams& g, const DmTile& dt, const TraceSet& tr,
                             const float* image, float* partial, int* status, int max_chunks,
                             int vel_kind, int fast, cudaStream_t s)
{
    if (g.aa_c > 0.f) {   // operator anti-aliasing: kernels of its own (the plan refuses other models)
        const int key = (vel_kind == VK_LINEAR ? 6 : 0) + g.weight * 2 + (fast ? 1 : 0);
        switch (key) {
            case 0: return dm_launch_t<VK_CONST, W_AA | 0, false>(g, dt, tr, image, partial, status, max_chunks, s);
            case 1: return dm_launch_t<VK_CONST, W_AA | 0, true>(g, dt, tr, image, partial, status, max_chunks, s);
            case 2: return dm_launch_t<VK_CONST, W_AA | 1, false>(g, dt, tr, image, partial, status, max_chunks, s);
            case 3: return dm_launch_t<VK_CONST, W_AA | 1, true>(g, dt, tr, image, partial, status, max_chunks, s);
            case 4: return dm_launch_t<VK_CONST, W_AA | 2, false>(g, dt, tr, image, partial, status, max_chunks, s);
            case 5: return dm_launch_t<VK_CONST, W_AA | 2, true>(g, dt, tr, image, partial, status, max_chunks, s);
            case 6: return dm_launch_t<VK_LINEAR, W_AA | 0, false>(g, dt, tr, image, partial, status, max_chunks, s);
            case 7: return dm_launch_t<VK_LINEAR, W_AA | 0, true>(g, dt, tr, image, partial, status, max_chunks, s);
            case 8: return dm_launch_t<VK_LINEAR, W_AA | 1, false>(g, dt, tr, image, partial, status, max_chunks, s);
            case 9: return dm_launch_t<VK_LINEAR, W_AA | 1, true>(g, dt, tr, image, partial, status, max_chunks, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (g.weight == KH_W_TRUE_AMP) {   // constant velocity only (the plan refuses the others)
        if (vel_kind != VK_CONST) return cudaErrorInvalidValue;
        return fast ? dm_launch_t<VK_CONST, 2, true>(g, dt, tr, image, partial, status, max_chunks, s)
                    : dm_launch_t<VK_CONST, 2, false>(g, dt, tr, image, partial, status, max_chunks, s);
    }
    const int key = vel_kind * 4 + g.weight * 2 + (fast ? 1 : 0);
    switch (key) {
        case 0: return dm_launch_t<VK_CONST, 0, false>(g, dt, tr, image, partial, status, max_chunks, s);
        case 1: return dm_launch_t<VK_CONST, 0, true>(g, dt, tr, image, partial, status, max_chunks, s);
        case 2: return dm_launch_t<VK_CONST, 1, false>(g, dt, tr, image, partial, status, max_chunks, s);
        case 3: return dm_launch_t<VK_CONST, 1, true>(g, dt, tr, image, partial, status, max_chunks, s);
        case 4: return dm_launch_t<VK_LINEAR, 0, false>(g, dt, tr, image, partial, status, max_chunks, s);
        case 5: return dm_launch_t<VK_LINEAR, 0, true>(g, dt, tr, image, partial, status, max_chunks, s);
        case 6: return dm_launch_t<VK_LINEAR, 1, false>(g, dt, tr, image, partial, status, max_chunks, s);
        case 7: return dm_launch_t<VK_LINEAR, 1, true>(g, dt, tr, image, partial, status, max_chunks, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_dm_reduce(const TraceSet& tr, int n_bins, const float* partial, int parts, int nt,
                             float* out, int ntr, cudaStream_t s)
{
    const long long total = (long long)ntr * nt;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    k_dm_reduce<<<std::max(blocks, 1), 256, 0, s>>>(tr.bin_start, n_bins, tr.perm, partial, parts, nt, out);
    return cudaGetLastError();
}

}  // namespace kh
