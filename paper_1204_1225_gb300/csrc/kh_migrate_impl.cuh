// Migration kernel (Eq. 1, Sec. 3): output-stationary gather over an image tile and one
// offset bin.
//
// CTA = 8 consumer warps + 1 producer warp.  Each consumer thread owns NZ = 16 consecutive
// z samples of one image column and keeps their FP32 accumulators in registers for the
// whole kernel; nothing is accumulated in global memory.  The producer warp walks the
// bin's traces (sorted by bin), culls those whose midpoint is outside the aperture of the
// tile footprint, bounds the two-way time over the tile box to a sample window
// [lo, hi], computes the trace's FP64 reference at the tile centre (linear v(z)), and
// stages the window into a 3-deep shared-memory ring with one cp.async.bulk per trace
// (16-byte aligned, no multicast) completing on the stage's mbarrier.  FP32 traces arrive as
// (sample, step) pairs, so one 8-byte shared load and one FMA give an interpolated sample.
// Consumers evaluate tau for their points (kh_tau.cuh; linear v(z): per-leg logarithms with the
// source leg cached per source position), read the staged samples, interpolate linearly,
// weight and accumulate; a warp whose window is not clipped and whose lanes all lie in the
// aperture and the grid skips the validity test.  All mbarrier waits are bounded; a wait that
// runs out sets the plan's status word and the CTA leaves only after its copies have landed.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstddef>
#include <type_traits>

#include "kh_tau.cuh"

namespace kh {

template <typename TT>
__device__ __forceinline__ float to_f32(TT v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

constexpr int MAX_ZG = 16;          // z-groups per CTA (cz)
constexpr int SLACK = 16;           // zeroed elements after the ring (reads one past a window)
constexpr int LEAD = 16;            // zeroed elements before the ring (a window clipped at t0 may be
                                    // indexed at -1 when tau is a rounding error below 0)

struct __align__(16) MigSmem {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    int cnt[STAGES];
    int last[STAGES];
    int row[4];                 // cell range of the tile (cx0, cx1, first row - 1, last row)
    int2 rng[MAX_CELL_ROWS];    // staging warp: sorted trace range of each cell row of the tile
    unsigned stat[2];           // staging warp: traces examined and staged for this tile
    // per staged trace
    float4 hdr[STAGES][BMAX];   // (sx, sy, rx, ry)
    float4 hda[STAGES][BMAX];   // linear: (c_x-2s_x, c_y-2s_y, c_x-2r_x, c_y-2r_y)
    float4 refs[STAGES][BMAX];  // linear: source-leg LegRef
    float4 refr[STAGES][BMAX];  // linear: receiver-leg LegRef
    float2 mid[STAGES][BMAX];   // FP32 midpoint (aperture test)
    int4 win[STAGES][BMAX];     // x: tau_ref - lo (float bits), y: smem index of sample lo minus
                                // MAGIC_BITS, z/w: c_mid/c_half (float bits) of the valid range
                                // 0 <= tau - lo <= hi - lo (EDGE_EPS wider on each side); sign
                                // bit of z: every column of the
                                // tile inside the aperture; sign bit of w: window not clipped
    float tb[STAGES][BMAX];     // lo dt + t0: T_s + T_r = (tau - lo) dt + tb (gradient mode)
    float4 zc[MAX_ZG * NZ];     // per-z constants: linear v, z_constants_m; constant v, (z^2, w_z);
                                // table, (w_z, z^2)
    float z2[MAX_ZG * NZ];      // linear: gamma(z) of the weight
    float zero[4];
};
static_assert(offsetof(MigSmem, zero) % 16 == 0, "the zero sample (pair) must be 16-byte aligned");

__host__ __device__ constexpr size_t mig_static_bytes() { return (sizeof(MigSmem) + 127) / 128 * 128; }

// Dynamic shared memory of one CTA when two CTAs share an SM's 228 KB (the runtime reserves
// 1 KB per CTA; 128 B of static shared variables).
constexpr size_t CTA_SMEM_BUDGET = 228 * 1024 / 2 - 1024 - 128;

// Nodes [tnh][tnz] (16-byte padded), then for KH_F16 one float4 (c0, c1, c2, 0) per h row: the
// row's reference polynomial in the normalised node depth (the nodes hold T minus it in FP16).
__host__ __device__ inline size_t table_node_bytes(const GeomParams& g)
{
    const size_t es = g.tdt == KH_F32 ? 4 : 2;
    return ((size_t)g.tnh * g.tnz * es + 15) / 16 * 16;
}

__host__ __device__ inline size_t table_bytes(const GeomParams& g)
{
    if (!g.table) return 0;
    return table_node_bytes(g) + (g.tdt == KH_F16 ? (size_t)g.tnh * sizeof(float4) : 0);
}

// Per consumer thread and depth, the cached source leg of the current source position (see
// mig_consumer): (C1 ln(1 + rho_s), sqrt(q_s)) for linear v(z), (dR_s, R_s) for time migration and
// the constant-velocity true-amplitude kernels, T_s for the tables (the radial table's shared copy
// leaves no room for more at two CTAs per SM).  The other constant-velocity kernels keep no cache:
// their leg is one square root, and surveys whose traces do not arrive shot by shot (the batched
// jobs') would recompute it per trace anyway.
__host__ __device__ inline size_t src_cache_bytes(const GeomParams& g)
{
    if (g.table || g.gtab) return (size_t)NZ * CONSUMERS * sizeof(float);
    // gradient: the thread's weighted image values, and for linear v(z) (C1 ln(1 + rho_s), (q/w)_s)
    // and sqrt(q_s)
    if (g.grad) return (size_t)NZ * CONSUMERS * (g.kabs > 0.0 ? sizeof(float2) + 2 * sizeof(float) : sizeof(float));
    return (g.kabs > 0.0 || g.pstm || g.weight == KH_W_TRUE_AMP) ? (size_t)NZ * CONSUMERS * sizeof(float2) : 0;
}

// Elements of one stage's sample area: a full trace always fits, so every trace is stageable.
// Plain samples: 16 KB per stage.  SamplePair rows hold half as many samples per byte; they take
// the largest stage at which two CTAs of the linear path (static part, ring, 32 KB source-leg
// cache) still fit.  With a traveltime table, the largest stage up to 16 KB at which two CTAs
// fit beside the table, but at least 8 KB (a large F32 table then runs one CTA per SM).  The
// gradient kernel's 64 KB of per-thread data leaves 8.75 KB per stage of slope rows at two CTAs
// per SM.
constexpr int PAIR_STAGE_BYTES = 19712;   // 2464 pairs, 1 KB of margin per SM
static_assert(((sizeof(MigSmem) + 127) / 128 * 128) +
                      ((LEAD + STAGES * (PAIR_STAGE_BYTES / 8) + SLACK) * 8 + 15) / 16 * 16 +
                      NZ * CONSUMERS * sizeof(float2) <= CTA_SMEM_BUDGET,
              "two CTAs of the pair-staged linear kernel must fit on one SM");
static_assert(PAIR_STAGE_BYTES / 8 >= (PAIR_MAX_NT + 5) / 2 * 2, "a whole pair row must fit one stage");
static_assert(((sizeof(MigSmem) + 127) / 128 * 128) + ((LEAD + STAGES * (8960 / 4) + SLACK) * 4 + 15) / 16 * 16 +
                      NZ * CONSUMERS * (sizeof(float2) + 2 * sizeof(float)) <= CTA_SMEM_BUDGET,
              "two CTAs of the linear gradient kernel must fit on one SM");
__host__ __device__ inline int mig_cap(const GeomParams& g)
{
    const int ealign = g.elem_align;
    const int need = (g.nt + 2 * ealign + ealign - 1) / ealign * ealign;
    long long bytes = g.grad ? 8960 : g.pairs ? PAIR_STAGE_BYTES : 16384;
    if (g.table) {
        const long long room = (long long)CTA_SMEM_BUDGET - (long long)mig_static_bytes() -
                               (long long)table_bytes(g) - (long long)src_cache_bytes(g) -
                               (long long)(LEAD + SLACK) * g.esize - 16;
        bytes = room / STAGES / 1024 * 1024;
        bytes = bytes > 16384 ? 16384 : (bytes < 8192 ? 8192 : bytes);
    }
    const int base = (int)(bytes / g.esize);
    return need > base ? need : base;
}

__host__ __device__ inline size_t mig_ring_bytes(const GeomParams& g)
{
    return (((size_t)LEAD + STAGES * mig_cap(g) + SLACK) * g.esize + 15) / 16 * 16;
}

inline size_t mig_smem_bytes(const GeomParams& g)
{
    return mig_static_bytes() + mig_ring_bytes(g) + table_bytes(g) + src_cache_bytes(g);
}

template <typename TB>
__device__ __forceinline__ float tab_f32(TB v);
template <>
__device__ __forceinline__ float tab_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float tab_f32<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float tab_f32<unsigned short>(unsigned short v) { return (float)v; }

// Radial table, step 1 (once per thread and trace leg): the table interpolated in h at the
// horizontal distance sqrt(dh2), at the K depth nodes jb .. jb + K - 1 that span the thread's
// 16 depths.
template <typename TB, int K, bool FAST>
__device__ __forceinline__ void tab_profile(const TB* tab, const GeomParams& g, float dh2, int jb, float* p)
{
    const float u = fminf(hsqrt<FAST>(dh2) * g.tinv, g.thmax);
    const int ih = (int)u;
    const float fh = u - (float)ih;
    const TB* r0 = tab + ih * g.tnz + jb;
    const TB* r1 = r0 + g.tnz;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float a = tab_f32<TB>(r0[k]), b = tab_f32<TB>(r1[k]);
        p[k] = fmaf(fh, b - a, a);
    }
    if constexpr (std::is_same<TB, __half>::value) {
        // FP16 residuals: add the rows' reference polynomials, interpolated in h like the nodes
        // (the interpolation is linear in the coefficients)
        const float4* cf = reinterpret_cast<const float4*>(reinterpret_cast<const char*>(tab) + table_node_bytes(g));
        const float4 q0 = cf[ih], q1 = cf[ih + 1];
        const float c0 = fmaf(fh, q1.x - q0.x, q0.x), c1 = fmaf(fh, q1.y - q0.y, q0.y);
        const float c2 = fmaf(fh, q1.z - q0.z, q0.z);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float u = (float)(jb + k) * g.tunz;
            p[k] += fmaf(fmaf(c2, u, c1), u, c0);
        }
    }
}

// Step 2 (per depth): depth nodes sit every M image samples from the thread's first depth,
// so depth i lies in node interval i / M at fraction (i % M) / M, both compile-time.
template <int M>
__device__ __forceinline__ float tab_depth(const float* p, int i)
{
    const int j = i / M, r = i % M;
    return r == 0 ? p[j] : fmaf((float)r * (1.f / M), p[j + 1] - p[j], p[j]);
}

// One leg's profile at K node rows from its location's table ([row][column], x fastest): the lerp
// in x between the column's two node columns (c0 points at node column gi of the first row; the
// next row follows gnx later).  The lanes of a warp (consecutive image columns) read a few
// consecutive nodes of one row per load.
template <int K>
__device__ __forceinline__ void grid_profile(const float* __restrict__ c0, int gnx, float fx, float* p)
{
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float a = __ldg(c0 + k * gnx), b = __ldg(c0 + k * gnx + 1);
        p[k] = fmaf(fx, b - a, a);
    }
}

// The migration kernel's sample read: th = tau - lo (window-relative sample position); valid
// iff |th - cmid| <= chalf, i.e. 0 <= th <= hi - lo up to EDGE_EPS; linear interpolation between
// samples floor(th) and floor(th) + 1 (adding 1.5 * 2^23 rounded down leaves floor(th) in the low
// mantissa bits), th below 0 read as 0; invalid points read the zeros at zero_off.
template <typename TT>
__device__ __forceinline__ float sample_at(const TT* data, float th, int base, float cmid, float chalf,
                                           int zero_off)
{
    const bool ok = fabsf(th - cmid) <= chalf;
    th = fmaxf(th, 0.f);
    const float tm = __fadd_rd(th, MAGIC);
    const float f = __fsub_rn(th, __fsub_rn(tm, MAGIC));
    const int off = ok ? __float_as_int(tm) + base : zero_off;
    if constexpr (std::is_same<TT, SamplePair>::value) {
        const float2 p = *reinterpret_cast<const float2*>(data + off);
        return fmaf(f, p.y, p.x);
    } else {
        const float d0 = to_f32<TT>(data[off]);
        const float d1 = to_f32<TT>(data[off + 1]);
        return fmaf(f, d1 - d0, d0);
    }
}

// sample_at without the validity test, for traces whose window is not clipped and whose every
// lane and depth lies in the tile box (so 0 <= th <= hi - lo).  Indexes the ring from its
// lead (base + LEAD); the unsigned clamp to the last readable pair keeps any index in bounds.
template <typename TT>
__device__ __forceinline__ float sample_unchecked(const TT* ring, float th, int base_lead, unsigned last)
{
    const float tm = __fadd_rd(th, MAGIC);
    const float f = __fsub_rn(th, __fsub_rn(tm, MAGIC));
    const unsigned off = min((unsigned)(__float_as_int(tm) + base_lead), last);
    if constexpr (std::is_same<TT, SamplePair>::value) {
        const float2 p = *reinterpret_cast<const float2*>(ring + off);
        return fmaf(f, p.y, p.x);
    } else {
        const float d0 = to_f32<TT>(ring[off]);
        const float d1 = to_f32<TT>(ring[off + 1]);
        return fmaf(f, d1 - d0, d0);
    }
}

// ------------------------------------------------------------------ producer warp
// The sorted traces one CTA examines: its bin's whole range, or with a (bin, cell) start table
// one range per row of the cells that meet the tile footprint widened by the aperture margin
// (cells of a row are consecutive in the sort order).  Every trace the staging cull would keep
// lies in those cells: its midpoint is within the cull radius, margin - 1 m, of the footprint.
// The row state (cx0, cx1, current row, last row) lives in shared memory, written by the
// staging warp only: it changes once per cell row, and keeping it out of registers leaves the
// kernel's register budget to the consumers.
// The tile's cell range, written by one thread before the tile's set-up barrier.
__device__ __forceinline__ void tile_cells(int* row, const TraceSet& tr, const TileBox& box)
{
    if (!tr.cell_start) return;
    const CellGrid& cg = tr.cg;
    auto cell = [&](double v, double g0, int n) {
        const double f = floor((v - g0) * cg.inv_cs);
        return (int)fmin(fmax(f, -1.0), (double)n);
    };
    const int cx0 = max(0, cell((double)box.xlo - cg.margin, cg.gx0, cg.ncx));
    const int cx1 = min(cg.ncx - 1, cell((double)box.xhi + cg.margin, cg.gx0, cg.ncx));
    const int cy0 = max(0, cell((double)box.ylo - cg.margin, cg.gy0, cg.ncy));
    const int cy1 = min(cg.ncy - 1, cell((double)box.yhi + cg.margin, cg.gy0, cg.ncy));
    row[0] = cx0;
    row[1] = cx1;
    row[2] = cy0 - 1;
    row[3] = (cx0 <= cx1) ? cy1 : cy0 - 1;
}

// The tile's sorted trace range of every cell row, written by the staging warp into shared
// memory (rng[0 .. nr - 1]); the walk keeps its row index and count in shared memory too
// (row[2], row[3]), so that it adds no register to the staging loop.
__device__ __forceinline__ void tile_rows(int* row, int2* rng, const TraceSet& tr, int bin)
{
    const int ncx = tr.cg.ncx;
    const int* cs = tr.cell_start + (long long)bin * ncx * tr.cg.ncy;
    const int cx0 = row[0], cx1 = row[1], cy0 = row[2] + 1, nr = row[3] - row[2];
    for (int i = threadIdx.x & 31; i < nr; i += 32) {
        const int cy = cy0 + i;
        rng[i] = make_int2(cs[cy * ncx + cx0], cs[cy * ncx + cx1 + 1]);
    }
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        row[2] = -1;
        row[3] = nr;
    }
    __syncwarp();
}

// Moves (cur, te) to the next non-empty cell row; leaves cur >= te when none is left.
__device__ __forceinline__ void next_row(int* row, const int2* rng, int& cur, int& te)
{
    int ri = row[2];
    const int nr = row[3];
    while (cur >= te && ri + 1 < nr) {
        ++ri;
        cur = rng[ri].x;
        te = rng[ri].y;
    }
    __syncwarp();
    if ((threadIdx.x & 31) == 0) row[2] = ri;
    __syncwarp();
}

// `n` is the number of stages this CTA's producer has filled before (mbarrier phases carry
// over from one work item to the next in the persistent kernel); returns the new count.
// The window-relative time the consumers evaluate is tau - lo (sample index floor(tau - lo)).
template <int VEL, typename TT, int WGT = 0>
__device__ __forceinline__ int mig_producer(MigSmem& S, TT* data, int cap, const GeomParams& g,
                                            const TraceSet& tr, const TT* __restrict__ traces, int bin,
                                            const TileBox& box, const WaitCfg& wc, int n, int tile_id = 0)
{
    const int lane = threadIdx.x & 31;
    const double inv_kdt = (VEL == VK_LINEAR) ? 1.0 / (g.kabs * g.dtd) : 0.0;
    PstmTile pt{};
    if constexpr (VEL == VK_PSTM) pt = pstm_tile(g, box);
    int cur = tr.bin_start[bin], te = tr.bin_start[bin + 1];
    if (tr.cell_start) {   // the first non-empty cell row of the tile
        tile_rows(S.row, S.rng, tr, bin);
        cur = te = 0;
        next_row(S.row, S.rng, cur, te);
    }
    if (lane == 0) S.stat[0] = S.stat[1] = 0u;
    const int n_begin = n;
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
            bool clipped = true;
            float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 m = make_float2(0.f, 0.f);
            if (k < te) {
                h = tr.hdr[k];
                m = tr.mid[k];
                ok = true;
                if (g.use_aperture) {
                    const float ax = fmaxf(fmaxf(box.xlo - m.x, m.x - box.xhi), 0.f);
                    const float ay = fmaxf(fmaxf(box.ylo - m.y, m.y - box.yhi), 0.f);
                    ok = ax * ax + ay * ay <= g.A2cull;
                }
                if (ok) {
                    if constexpr (VEL == VK_GRID) {
                        // the window from the tile's node bounds of both legs' tables; a negative
                        // location (a position with no table) skips the trace
                        const int ls = __float_as_int(h.y), lr = __float_as_int(h.w);
                        ok = ls >= 0 && lr >= 0;
                        if (ok) {
                            const float2 bs = __ldg(&g.gbnd[(long long)ls * g.gtiles + tile_id]);
                            const float2 br = __ldg(&g.gbnd[(long long)lr * g.gtiles + tile_id]);
                            ok = sample_window(__fadd_rn(bs.x, br.x), __fadd_rn(bs.y, br.y), g, lo, hi, &clipped);
                        }
                    } else {
                        ok = trace_window(h, box, VEL == VK_TABLE ? (g.k == 0.0 ? VK_CONST : VK_LINEAR) : VEL,
                                          g, lo, hi, &clipped, &pt);
                    }
                    lo_al = lo & ~(g.elem_align - 1);
                    len_al = (hi + 1 - lo_al + g.elem_align - 1) & ~(g.elem_align - 1);
                }
            }
            const unsigned okm = __ballot_sync(0xffffffffu, ok);
            int pre = ok ? len_al : 0;   // inclusive prefix of window lengths
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
            int bytes = fits ? len_al * g.esize : 0;
            int used_add = fits ? len_al : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
                used_add += __shfl_xor_sync(0xffffffffu, used_add, o);
            }
            if (fits) {
                const int slot = cnt + rank;
                const int dst = s * cap + used + excl;
                double tau_ref = (VEL == VK_TABLE) ? g.c0 + 0.5 : -g.t0d / g.dtd;
                if constexpr (VEL == VK_LINEAR) {
                    LegRef rs, rr;
                    float qis = 0.f, qir = 0.f;
                    const double ls = leg_reference(box.cx, box.cy, box.cz, h.x, h.y, g, rs, &qis);
                    const double lr = leg_reference(box.cx, box.cy, box.cz, h.z, h.w, g, rr, &qir);
                    tau_ref = __dadd_rn(tau_ref, __dmul_rn(__dadd_rn(ls, lr), inv_kdt));
                    // (R_c^2, (q_c + 2)/u_c, w_c, 1/u_c) per leg
                    S.refs[s][slot] = make_float4(rs.Rc2, qis, rs.wc, rs.iuc);
                    S.refr[s][slot] = make_float4(rr.Rc2, qir, rr.wc, rr.iuc);
                    S.hda[s][slot] = make_float4((float)(box.cx - 2.0 * h.x), (float)(box.cy - 2.0 * h.y),
                                                 (float)(box.cx - 2.0 * h.z), (float)(box.cy - 2.0 * h.w));
                } else if constexpr (VEL == VK_CONST && (WGT & 3) == 2) {
                    // the true-amplitude kernels take the legs relative to the tile centre: FP64 legs
                    // at the tile centre c, R_ac = |c - a|, and tau_c = (R_sc + R_rc) / (v0 dt) - t0/dt
                    {
                    const double esx = __dadd_rn(box.cx, -(double)h.x), esy = __dadd_rn(box.cy, -(double)h.y);
                    const double erx = __dadd_rn(box.cx, -(double)h.z), ery = __dadd_rn(box.cy, -(double)h.w);
                    const double zc2 = __dmul_rn(box.cz, box.cz);
                    const double rsc = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(esx, esx), __dmul_rn(esy, esy)), zc2));
                    const double rrc = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(erx, erx), __dmul_rn(ery, ery)), zc2));
                    tau_ref = __dadd_rn(tau_ref, __ddiv_rn(__dadd_rn(rsc, rrc), __dmul_rn(g.v0, g.dtd)));
                    S.refs[s][slot] = make_float4((float)rsc, (float)rrc, 0.f, 0.f);
                    S.hda[s][slot] = make_float4((float)(box.cx - 2.0 * h.x), (float)(box.cy - 2.0 * h.y),
                                                 (float)(box.cx - 2.0 * h.z), (float)(box.cy - 2.0 * h.w));
                    }
                } else if constexpr (VEL == VK_PSTM) {
                    // FP64 legs at the tile centre (x_c, t0_c): R_ac = sqrt(|c - a|^2 + ze_c^2) on the
                    // straight rays of the RMS medium, and tau_c = C1(t0_c) (R_sc + R_rc) - t0/dt
                    const double esx = __dadd_rn(box.cx, -(double)h.x), esy = __dadd_rn(box.cy, -(double)h.y);
                    const double erx = __dadd_rn(box.cx, -(double)h.z), ery = __dadd_rn(box.cy, -(double)h.w);
                    const double rsc = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(esx, esx), __dmul_rn(esy, esy)), pt.pze2));
                    const double rrc = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(erx, erx), __dmul_rn(ery, ery)), pt.pze2));
                    const double sc = __dadd_rn(rsc, rrc);
                    tau_ref = __dadd_rn(tau_ref, __dmul_rn(pt.pc1, sc));
                    S.refs[s][slot] = make_float4((float)rsc, (float)rrc, (float)sc, 0.f);
                    S.hda[s][slot] = make_float4((float)(box.cx - 2.0 * h.x), (float)(box.cy - 2.0 * h.y),
                                                 (float)(box.cx - 2.0 * h.z), (float)(box.cy - 2.0 * h.w));
                }
                S.hdr[s][slot] = h;
                S.mid[s][slot] = m;
                S.tb[s][slot] = (float)__dadd_rn(__dmul_rn((double)lo, g.dtd), g.t0d);
                // every column of the tile inside the aperture: the column test is monotone in
                // |column - midpoint| per axis, so the corner farthest on both axes decides it
                bool whole = false;
                if (g.use_aperture) {
                    const float ex = fmaxf(fabsf(__fsub_rn(box.xlo, m.x)), fabsf(__fsub_rn(box.xhi, m.x)));
                    const float ey = fmaxf(fabsf(__fsub_rn(box.ylo, m.y)), fabsf(__fsub_rn(box.yhi, m.y)));
                    whole = __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)) <= (g.use_taper ? g.ap_core2 : g.A2);
                }
                const float lim = (float)(hi - lo);
                // w: c_half, its sign bit set when the window was not clipped at 0 or nt - 1 (then
                // every point of the tile box has 0 <= tau - lo <= hi - lo by construction)
                S.win[s][slot] = make_int4(__float_as_int((float)(tau_ref - (double)lo)),
                                           dst + (lo - lo_al) - MAGIC_BITS,
                                           __float_as_int(0.5f * lim) | (whole ? (int)0x80000000 : 0),
                                           __float_as_int(0.5f * lim + EDGE_EPS) | (clipped ? 0 : (int)0x80000000));
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
            if (lane == 0) {
                S.stat[0] += (unsigned)consumed;
                S.stat[1] += (unsigned)nfit;
            }
            if (cur >= te && tr.cell_start) next_row(S.row, S.rng, cur, te);   // the tile's next cell row
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
    if (wc.stats && lane == 0) {
        atomicAdd(&wc.stats[0], (unsigned long long)S.stat[0]);
        atomicAdd(&wc.stats[1], (unsigned long long)S.stat[1]);
        atomicAdd(&wc.stats[2], 1ull);
    }
    if (failed) {
        if (lane == 0) atomicOr(wc.status, 1);
        // let every copy already issued land before the CTA can exit
        const int first = n - STAGES > n_begin ? n - STAGES : n_begin;
        for (int f = first; f < n; ++f)
            mbar_wait_bounded(&S.full[f % STAGES], (f / STAGES) & 1, 0, WAIT_NS, nullptr);
    }
    return n;
}

// Column (tx, ty) and z-group of consumer thread `tid` in the tile.  When the layer's footprint
// allows it, a warp covers an 8 x 4 block of columns instead of 32 x 1 or 16 x 2: a compact
// footprint leaves fewer lanes idle where the aperture boundary crosses the warp.
__device__ __forceinline__ void thread_column(const TileShape& ts, int tid, int& tx, int& ty, int& tzg)
{
    const int layer = ts.cx * ts.cy;
    tzg = tid / layer;
    const int r = tid - tzg * layer;
    if ((ts.cx & 7) == 0 && (ts.cy & 3) == 0) {
        const int wl = r >> 5, lane = r & 31, bx = ts.cx >> 3;
        tx = (wl % bx) * 8 + (lane & 7);
        ty = (wl / bx) * 4 + (lane >> 3);
    } else {
        tx = r % ts.cx;
        ty = r / ts.cx;
    }
}

// ------------------------------------------------------------------ consumer warps
// `n`: stages consumed before this tile (see mig_producer); returns the new count.
//
// Linear v(z): the source leg of a contribution depends only on the column and the source
// position, and traces of one bin arrive shot by shot (the bin sort is stable), so each thread
// keeps (C1 ln(1 + rho_s), sqrt(q_s)) of its 16 depths for the current source in `srcc` (its
// own slots, [i * CONSUMERS + tid]) and recomputes them only when the (warp-uniform) source
// changes.  tau - lo = c0rel + C1 ln(1 + rho_s) + C1 ln(1 + rho_r) with c0rel = tau_ref - lo,
// each leg's logarithm from the per-leg fit (LPT = its length).  The weight's gamma(z)
// multiplies each depth's sum once, before the store.
template <int VEL, int WGT, bool FAST, typename TT, int LPT, typename TB>
__device__ __forceinline__ int mig_consumer(MigSmem& S, const TT* data, const GeomParams& g,
                                            const TileShape& ts, int x0, int y0, int z0,
                                            const TileBox& box, int bin, float* __restrict__ image,
                                            const WaitCfg& wc, const TB* tab, float2* srcc, int cap, int n)
{
    constexpr int WB = WGT & 3;                 // the weight (KH_W_*)
    constexpr bool AA = (WGT & W_AA) != 0;      // operator anti-aliasing compiled in (constant v)
    const int tid = threadIdx.x, lane = tid & 31;
    int tx, ty, tzg;
    thread_column(ts, tid, tx, ty, tzg);
    const int ix = x0 + tx, iy = y0 + ty, izb = z0 + tzg * NZ;
    const bool col_ok = ix < g.nx && iy < g.ny;
    const float cxf = col_coord(g.ox, ix, g.dx);
    const float cyf = (g.dim == 3) ? col_coord(g.oy, iy, g.dy) : 0.f;
    const double xd = grid_coord(g.ox, ix, g.dx), yd = (g.dim == 3) ? grid_coord(g.oy, iy, g.dy) : 0.0;
    const float dxc = (float)(xd - box.cx), dyc = (float)(yd - box.cy);
    const float4* zc = &S.zc[tzg * NZ];
    const float* zg = &S.z2[tzg * NZ];   // linear: gamma(z) of the weight
    const int zero_off = (int)(((const char*)S.zero - (const char*)data) / (int)sizeof(TT));

    float acc[NZ];
#pragma unroll
    for (int i = 0; i < NZ; ++i) acc[i] = 0.f;
    float2* my_src = srcc + tid;
    unsigned psx = 0xffffffffu, psy = 0xffffffffu;   // source of the cached leg (NaN bits: none)
    const TT* ring = data - LEAD;
    const unsigned ring_last = (unsigned)(LEAD + STAGES * cap + SLACK - 2);   // the kernel's ring
    const bool zfull = izb + NZ <= g.nz;   // all 16 depths of this thread lie in the grid
    // anti-aliasing: the range [aa_lo, aa_hi] of z^2 over the thread's depths (constant velocity)
    // or of z (v0 + k z, with the thread's first depth aa_z0 and the depth step aa_dz)
    float aa_lo = 0.f, aa_hi = 0.f, aa_z0 = 0.f, aa_dz = 0.f;
    if constexpr (AA && VEL == VK_CONST) {
        const float za = zc[0].z, zb = zc[NZ - 1].z;
        aa_lo = (za <= 0.f && zb >= 0.f) ? 0.f : fminf(za * za, zb * zb);
        aa_hi = fmaxf(za * za, zb * zb);
    } else if constexpr (AA && VEL == VK_LINEAR) {
        aa_z0 = (float)grid_coord(g.oz, izb, g.dz);
        aa_dz = (float)g.dz;
        const float zl = (float)grid_coord(g.oz, izb + NZ - 1, g.dz);
        aa_lo = fminf(aa_z0, zl);
        aa_hi = fmaxf(aa_z0, zl);
    }
    // gridded model: the column's node column and fraction, and its first node row (threads
    // whose depths all lie below the image read the last rows)
    const float* gcol = nullptr;
    float gfx = 0.f;
    if constexpr (VEL == VK_GRID) {
        const int gi = grid_col(g, ix, &gfx);
        const int jb = min(g.gzoff + izb / LPT, g.gnz - (NZ / LPT + 1));
        gcol = g.gtab + (long long)jb * g.gnx + gi;
    }
    // gridded model: the receiver table nodes of the next trace of the stage, read one trace
    // ahead so that their L2 latency overlaps this trace's depth loop (pf_t: the trace they
    // belong to, -1: none); not with nodes at every depth (17 nodes per column would spill)
    constexpr bool GPF = (VEL == VK_GRID) && (NZ / LPT + 1) <= 9;
    constexpr int GK = GPF ? NZ / LPT + 1 : 1;
    float pfa[GK], pfb[GK];
    int pf_t = -1;

    bool failed = false;
    while (true) {
        const int s = n % STAGES;
        if (!warp_wait(&S.full[s], (n / STAGES) & 1, wc.polls, wc.ns, wc.status)) {
            failed = true;
            break;
        }
        const int cnt = S.cnt[s];
        const int last = S.last[s];
        for (int t = 0; t < cnt; ++t) {
            const int4 w = S.win[s][t];
            bool inside = col_ok;
            float tp = 1.f;   // aperture taper of this column (1 in the taper's core)
            if (g.use_aperture && w.z >= 0) {   // sign bit of w.z: every column is inside (its core)
                const float2 m = S.mid[s][t];
                inside = inside && in_aperture(cxf, cyf, m.x, m.y, g.A2);
                if (g.use_taper && inside) tp = aperture_taper(cxf, cyf, m.x, m.y, g);
            }
            if (!__any_sync(0xffffffffu, inside)) continue;
            const float c0rel = __int_as_float(w.x);
            const float cmid = __int_as_float(w.z & 0x7fffffff);
            const float chalf = inside ? __int_as_float(w.w & 0x7fffffff) : -1.f;
            const float4 h = S.hdr[s][t];
            // unclipped window, and every lane inside the aperture (its untapered core, with a
            // taper) with all 16 depths in the grid: every tau is inside the window, no validity
            // test and no taper are needed
            const bool unchecked = w.w < 0 && (!g.use_taper || w.z < 0) && __all_sync(0xffffffffu, inside && zfull);
            if constexpr (VEL == VK_TABLE) {
                // T_s + T_r in table units from the radial table; the source leg T_s is cached
                // per source position like the linear path's
                constexpr int M = LPT;            // depth nodes every M samples (1, 2 or 4)
                constexpr int K = NZ / M + 1;     // nodes spanning the thread's 16 depths
                float* my_ts = reinterpret_cast<float*>(srcc) + tid;
                const int jb = izb / M;
                const float dxs = cxf - h.x, dys = cyf - h.y;
                const float dhs2 = fmaf(dxs, dxs, dys * dys);
                if (__float_as_uint(h.x) != psx || __float_as_uint(h.y) != psy) {   // new source
                    float ps[K];
                    tab_profile<TB, K, FAST>(tab, g, dhs2, jb, ps);
#pragma unroll
                    for (int i = 0; i < NZ; ++i) my_ts[i * CONSUMERS] = tab_depth<M>(ps, i);
                    psx = __float_as_uint(h.x);
                    psy = __float_as_uint(h.y);
                }
                const float dxr = cxf - h.z, dyr = cyf - h.w;
                const float dhr2 = fmaf(dxr, dxr, dyr * dyr);
                float pr[K];
                tab_profile<TB, K, FAST>(tab, g, dhr2, jb, pr);
                auto zloop = [&](auto checked, auto tapered) {
#pragma unroll
                    for (int i = 0; i < NZ; ++i) {
                        const float th = fmaf(my_ts[i * CONSUMERS] + tab_depth<M>(pr, i), g.C1, c0rel);
                        float val;
                        if constexpr (decltype(checked)::value)
                            val = sample_at<TT>(data, th, w.y, cmid, chalf, zero_off);
                        else
                            val = sample_unchecked<TT>(ring, th, w.y + LEAD, ring_last);
                        if constexpr (decltype(tapered)::value) val *= tp;
                        // w_z multiplies the sum once, at the store
                        if constexpr (WB == 1) {
                            const float Rsum = hsqrt<FAST>(dhs2 + zc[i].y) + hsqrt<FAST>(dhr2 + zc[i].y);
                            acc[i] = fmaf(Rsum, val, acc[i]);
                        }
                        else acc[i] += val;
                    }
                };
                if (unchecked) zloop(std::false_type(), std::false_type());
                else if (g.use_taper) zloop(std::true_type(), std::true_type());
                else zloop(std::true_type(), std::false_type());
            } else if constexpr (VEL == VK_GRID) {
                // T_s + T_r from the two legs' first-arrival tables (global memory, L2-resident):
                // per leg the profile at the thread's K node rows, then linear in depth; the
                // source leg is cached per source location
                constexpr int M = LPT;            // depth nodes every M samples (1, 2 or 4)
                constexpr int K = NZ / M + 1;
                float* my_ts = reinterpret_cast<float*>(srcc) + tid;
                const int ls = __float_as_int(h.y), lr = __float_as_int(h.w);
                const float dxs = cxf - h.x, dxr = cxf - h.z;
                const float dhs2 = dxs * dxs, dhr2 = dxr * dxr;
                if ((unsigned)ls != psx) {   // new source location
                    float ps[K];
                    grid_profile<K>(gcol + (long long)ls * g.gstride, g.gnx, gfx, ps);
#pragma unroll
                    for (int i = 0; i < NZ; ++i) my_ts[i * CONSUMERS] = tab_depth<M>(ps, i);
                    psx = (unsigned)ls;
                }
                float pr[K];
                if (GPF && pf_t == t) {
#pragma unroll
                    for (int k = 0; k < K; ++k) pr[k] = fmaf(gfx, pfb[k] - pfa[k], pfa[k]);
                } else {
                    grid_profile<K>(gcol + (long long)lr * g.gstride, g.gnx, gfx, pr);
                }
                pf_t = -1;
                if (GPF && t + 1 < cnt) {   // the next trace's receiver nodes, in flight during this loop
                    const int ln = __float_as_int(S.hdr[s][t + 1].w);
                    if (ln >= 0) {
                        const float* c0 = gcol + (long long)ln * g.gstride;
#pragma unroll
                        for (int k = 0; k < K; ++k) {
                            pfa[k] = __ldg(c0 + k * g.gnx);
                            pfb[k] = __ldg(c0 + k * g.gnx + 1);
                        }
                        pf_t = t + 1;
                    }
                }
                auto zloop = [&](auto checked, auto tapered) {
#pragma unroll
                    for (int i = 0; i < NZ; ++i) {
                        const float th = fmaf(my_ts[i * CONSUMERS] + tab_depth<M>(pr, i), g.C1, c0rel);
                        float val;
                        if constexpr (decltype(checked)::value)
                            val = sample_at<TT>(data, th, w.y, cmid, chalf, zero_off);
                        else
                            val = sample_unchecked<TT>(ring, th, w.y + LEAD, ring_last);
                        if constexpr (decltype(tapered)::value) val *= tp;
                        // w_z multiplies the sum once, at the store
                        if constexpr (WB == 1) {
                            const float Rsum = hsqrt<FAST>(dhs2 + zc[i].y) + hsqrt<FAST>(dhr2 + zc[i].y);
                            acc[i] = fmaf(Rsum, val, acc[i]);
                        }
                        else acc[i] += val;
                    }
                };
                if (unchecked) zloop(std::false_type(), std::false_type());
                else if (g.use_taper) zloop(std::true_type(), std::true_type());
                else zloop(std::true_type(), std::false_type());
            } else if constexpr (VEL == VK_PSTM) {
                // time migration relative to the tile centre: per leg R_a - R_ac = (q_a - q_ac) /
                // (R_a + R_ac) with q_a - q_ac = dP_a + (ze^2 - ze_c^2), so that
                // tau - lo = c0rel + (C1(t0) - C1(t0_c)) S_c + C1(t0) (dR_s + dR_r) carries only
                // quantities of a few tens of samples; the source leg (dR_s, R_s) is cached per
                // source position like the linear path's
                const float4 a = S.hda[s][t];
                const float4 rf = S.refs[s][t];   // (R_sc, R_rc, S_c, -)
                if (__float_as_uint(h.x) != psx || __float_as_uint(h.y) != psy) {   // new source
                    const float dPs = fmaf(dxc, cxf + a.x, dyc * (cyf + a.y));
                    const float exs = cxf - h.x, eys = cyf - h.y;
                    const float dhs2 = fmaf(exs, exs, eys * eys);
#pragma unroll
                    for (int i = 0; i < NZ; ++i) {
                        const float4 c = zc[i];   // (ze^2, ze^2 - ze_c^2, C1(t0), C1(t0) - C1(t0_c))
                        const float R = hsqrt<FAST>(dhs2 + c.x);
                        my_src[i * CONSUMERS] = make_float2((dPs + c.y) * hrcp<FAST>(R + rf.x), R);
                    }
                    psx = __float_as_uint(h.x);
                    psy = __float_as_uint(h.y);
                }
                const float dPr = fmaf(dxc, cxf + a.z, dyc * (cyf + a.w));
                const float exr = cxf - h.z, eyr = cyf - h.w;
                const float dhr2 = fmaf(exr, exr, eyr * eyr);
                auto zloop = [&](auto checked, auto tapered) {
#pragma unroll
                    for (int i = 0; i < NZ; ++i) {
                        const float4 c = zc[i];
                        const float2 sv = my_src[i * CONSUMERS];   // (dR_s, R_s)
                        const float R = hsqrt<FAST>(dhr2 + c.x);
                        const float dR = (dPr + c.y) * hrcp<FAST>(R + rf.y);
                        const float th = fmaf(c.z, sv.x + dR, fmaf(c.w, rf.z, c0rel));
                        float val;
                        if constexpr (decltype(checked)::value)
                            val = sample_at<TT>(data, th, w.y, cmid, chalf, zero_off);
                        else
                            val = sample_unchecked<TT>(ring, th, w.y + LEAD, ring_last);
                        if constexpr (decltype(tapered)::value) val *= tp;
                        // W = w_z (R_s + R_r); w_z multiplies the sum once, at the store
                        if constexpr (WB == 1) acc[i] = fmaf(sv.y + R, val, acc[i]);
                        else acc[i] += val;
                    }
                };
                if (unchecked) zloop(std::false_type(), std::false_type());
                else if (g.use_taper) zloop(std::true_type(), std::true_type());
                else zloop(std::true_type(), std::false_type());
            } else if constexpr (VEL == VK_CONST && WB != 2) {
                const float dxs = cxf - h.x, dys = cyf - h.y;
                const float dxr = cxf - h.z, dyr = cyf - h.w;
                // anti-aliasing: skip a trace whose every weight here is 0; evaluate the weight
                // per contribution only where the warp's depth range holds weights below 1
                int aacls = 1;
                if constexpr (AA) {
                    aacls = aa_class(g.aa_c, dxs, dys, dxr, dyr, aa_lo, aa_hi, inside);
                    if (aacls == 0) continue;
                }
                const float dhs2 = fmaf(dxs, dxs, dys * dys);
                const float dhr2 = fmaf(dxr, dxr, dyr * dyr);
                auto zloop = [&](auto checked, auto tapered, auto alias) {
#pragma unroll
                    for (int i = 0; i < NZ; ++i) {
                        const float Rs = hsqrt<FAST>(dhs2 + zc[i].x), Rr = hsqrt<FAST>(dhr2 + zc[i].x);
                        const float Ssum = Rs + Rr;
                        const float th = fmaf(Ssum, g.C1, fmaf(Ssum, g.C1lo, c0rel));
                        float val;
                        if constexpr (decltype(checked)::value)
                            val = sample_at<TT>(data, th, w.y, cmid, chalf, zero_off);
                        else
                            val = sample_unchecked<TT>(ring, th, w.y + LEAD, ring_last);
                        if constexpr (decltype(tapered)::value) val *= tp;
                        if constexpr (decltype(alias)::value) val *= aa_weight<FAST>(g.aa_c, dxs, dys, dxr, dyr, Rs, Rr);
                        // w_z multiplies the sum once, at the store
                        if constexpr (WB == 1) acc[i] = fmaf(Ssum, val, acc[i]);
                        else acc[i] += val;
                    }
                };
                using T_ = std::true_type;
                using F_ = std::false_type;
                bool done = false;
                if constexpr (AA) {
                    if (aacls == 2) {
                        if (unchecked) zloop(F_(), F_(), T_());
                        else zloop(T_(), T_(), T_());
                        done = true;
                    }
                }
                if (done) {
                } else if (unchecked) zloop(F_(), F_(), F_());
                else if (g.use_taper) zloop(T_(), T_(), F_());
                else zloop(T_(), F_(), F_());
            } else if constexpr (VEL == VK_CONST) {
                // the true-amplitude weight: each leg relative to the tile centre: R_a - R_ac = (q_a - q_ac) / (R_a + R_ac) with
                // q_a - q_ac = dP_a + (z^2 - z_c^2), so tau - lo = c0rel + C1 (dR_s + dR_r) carries only
                // quantities of a few tens of samples (the full two-way time, hundreds of samples,
                // is in the FP64 reference); the source leg (dR_s, R_s) is cached per source position
                // anti-aliasing classes as in the direct branch
                int aacls = 1;
                if constexpr (AA) {
                    aacls = aa_class(g.aa_c, cxf - h.x, cyf - h.y, cxf - h.z, cyf - h.w, aa_lo, aa_hi, inside);
                    if (aacls == 0) continue;
                }
                const float4 a = S.hda[s][t];
                const float4 rf = S.refs[s][t];   // (R_sc, R_rc, -, -)
                if (__float_as_uint(h.x) != psx || __float_as_uint(h.y) != psy) {   // new source
                    const float dPs = fmaf(dxc, cxf + a.x, dyc * (cyf + a.y));
                    const float exs = cxf - h.x, eys = cyf - h.y;
                    const float dhs2 = fmaf(exs, exs, eys * eys);
#pragma unroll
                    for (int i = 0; i < NZ; ++i) {
                        const float4 c = zc[i];   // (z^2, z^2 - z_c^2, z, 1 off the surface row)
                        const float R = hsqrt<FAST>(dhs2 + c.x);
                        my_src[i * CONSUMERS] = make_float2((dPs + c.y) * hrcp<FAST>(fmaxf(R + rf.x, 1e-30f)), R);
                    }
                    psx = __float_as_uint(h.x);
                    psy = __float_as_uint(h.y);
                }
                const float dPr = fmaf(dxc, cxf + a.z, dyc * (cyf + a.w));
                const float exr = cxf - h.z, eyr = cyf - h.w;
                const float dhr2 = fmaf(exr, exr, eyr * eyr);
                auto zloop = [&](auto checked, auto tapered, auto alias) {
#pragma unroll
                    for (int i = 0; i < NZ; ++i) {
                        const float4 c = zc[i];
                        const float2 sv = my_src[i * CONSUMERS];   // (dR_s, R_s)
                        const float Rr = hsqrt<FAST>(dhr2 + c.x);
                        const float dR = (dPr + c.y) * hrcp<FAST>(fmaxf(Rr + rf.y, 1e-30f));
                        const float Rs = sv.y;
                        const float th = fmaf(g.C1, sv.x + dR, c0rel);
                        float val;
                        if constexpr (decltype(checked)::value)
                            val = sample_at<TT>(data, th, w.y, cmid, chalf, zero_off);
                        else
                            val = sample_unchecked<TT>(ring, th, w.y + LEAD, ring_last);
                        if constexpr (decltype(tapered)::value) val *= tp;
                        // the weight per contribution (0 on the surface row, where it is undefined);
                        // with anti-aliasing both weights share the legs' reciprocals
                        float W;
                        if constexpr (decltype(alias)::value) {
                            const float is = hrcp<FAST>(fmaxf(Rs, 1e-30f)), ir = hrcp<FAST>(fmaxf(Rr, 1e-30f));
                            W = c.w != 0.f ? ta_weight_r<FAST>(c.z, Rs, Rr, is, ir, g.dim == 3) *
                                                 aa_weight_r(g.aa_c, cxf - h.x, cyf - h.y, exr, eyr, is, ir)
                                           : 0.f;
                        } else {
                            W = c.w != 0.f ? ta_weight<FAST>(c.z, Rs, Rr, g.dim == 3) : 0.f;
                        }
                        acc[i] = fmaf(W, val, acc[i]);
                    }
                };
                using T_ = std::true_type;
                using F_ = std::false_type;
                bool done = false;
                if constexpr (AA) {
                    if (aacls == 2) {
                        if (unchecked) zloop(F_(), F_(), T_());
                        else zloop(T_(), T_(), T_());
                        done = true;
                    }
                }
                if (done) {
                } else if (unchecked) zloop(F_(), F_(), F_());
                else if (g.use_taper) zloop(T_(), T_(), F_());
                else zloop(T_(), F_(), F_());
            } else {
                // anti-aliasing classes as in the constant-velocity branches
                int aacls = 1;
                if constexpr (AA && VEL == VK_LINEAR) {
                    aacls = aa_class_lin(g, cxf - h.x, cyf - h.y, cxf - h.z, cyf - h.w, aa_lo, aa_hi, inside);
                    if (aacls == 0) continue;
                }
                const float4 a = S.hda[s][t];
                if (__float_as_uint(h.x) != psx || __float_as_uint(h.y) != psy) {   // new source
                    const float4 rs = S.refs[s][t];
                    const float dPs = fmaf(dxc, cxf + a.x, dyc * (cyf + a.y));
                    const float exs = cxf - h.x, eys = cyf - h.y;
                    const float dhs2 = fmaf(exs, exs, eys * eys);
#pragma unroll
                    for (int i = 0; i < NZ; ++i) {
                        float sqs = 0.f;
                        const float rho_s = leg_delta_m<WB, FAST>(dPs, dhs2, zc[i], rs, sqs);
                        my_src[i * CONSUMERS] = make_float2(leg_log<LPT>(rho_s, g, 0.f), sqs);
                    }
                    psx = __float_as_uint(h.x);
                    psy = __float_as_uint(h.y);
                }
                const float4 rr = S.refr[s][t];
                const float dPr = fmaf(dxc, cxf + a.z, dyc * (cyf + a.w));
                const float exr = cxf - h.z, eyr = cyf - h.w;
                const float dhr2 = fmaf(exr, exr, eyr * eyr);
                auto zloop = [&](auto checked, auto tapered, auto alias) {
#pragma unroll
                    for (int i = 0; i < NZ; ++i) {
                        float sqr = 0.f;
                        const float2 sv = my_src[i * CONSUMERS];   // (C1 ln(1 + rho_s), sqrt(q_s))
                        const float rho_r = leg_delta_m<WB, FAST>(dPr, dhr2, zc[i], rr, sqr);
                        const float th = leg_log<LPT>(rho_r, g, c0rel + sv.x);
                        float val;
                        if constexpr (decltype(checked)::value)
                            val = sample_at<TT>(data, th, w.y, cmid, chalf, zero_off);
                        else
                            val = sample_unchecked<TT>(ring, th, w.y + LEAD, ring_last);
                        if constexpr (decltype(tapered)::value) val *= tp;
                        if constexpr (decltype(alias)::value) {
                            // each leg's slowness factor at this depth (FP32 geometry: the weight
                            // is flat where rounding could move it)
                            const float zi = fmaf((float)i, aa_dz, aa_z0);
                            const float vv = fmaf(g.aa_v0k, zi, g.aa_v0sq);
                            const float exs = cxf - h.x, eys = cyf - h.y;
                            const float fs = aa_leg_lin(fmaf(zi, zi, fmaf(exs, exs, eys * eys)), vv, g.aa_kq);
                            const float fr = aa_leg_lin(fmaf(zi, zi, dhr2), vv, g.aa_kq);
                            val *= aa_weight_r(g.aa_c, exs, eys, exr, eyr, fs, fr);
                        }
                        // gamma(z) multiplies the sum once, at the store
                        if constexpr (WB == 1) acc[i] = fmaf(sv.y + sqr, val, acc[i]);
                        else acc[i] += val;
                    }
                };
                using T_ = std::true_type;
                using F_ = std::false_type;
                bool done = false;
                if constexpr (AA && VEL == VK_LINEAR) {
                    if (aacls == 2) {
                        if (unchecked) zloop(F_(), F_(), T_());
                        else zloop(T_(), T_(), T_());
                        done = true;
                    }
                }
                if (done) {
                } else if (unchecked) zloop(F_(), F_(), F_());
                else if (g.use_taper) zloop(T_(), T_(), F_());
                else zloop(T_(), F_(), F_());
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[s]);
        ++n;
        if (last) break;
    }
    if (failed) {
        if (lane == 0) atomicOr(wc.status, 1);
        return n;
    }
    if (!col_ok) return n;
    if constexpr (WB == 1) {
#pragma unroll
        for (int i = 0; i < NZ; ++i)
            acc[i] *= (VEL == VK_TABLE || VEL == VK_GRID) ? zc[i].x : zg[i];
    }
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
    return n;
}

// ------------------------------------------------------------------ gradient consumer
// dB/d(v0, k) of B(m, D) = <m, migrate(D)>: per contribution W m (D[i+1] - D[i]) dT/dth,
// with dT/dth summed over both legs (the 1/dt of dtau/dth is applied in the final sum):
//   constant v:  dT/dv0 = -(R_s + R_r)/v0^2;
//   linear v(z): with q/w = sqrt(q/(q+2)) per leg and vz = v0 + k z,
//                dT/dv0 = -(q/w)_sum (1/v0 + 1/vz)/|k|,
//                dT/dk  = -sgn(k) (T_s + T_r)/|k| + (q/w)_sum (2/k - z/vz)/|k|.
// The traces arrive as slope rows D[i+1] - D[i] (one read per contribution).  Linear v(z): the
// source leg (its logarithm term, q/w and sqrt(q)) is cached per source position as in the
// migration, and tau - lo adds the per-leg logarithms.  Each thread sums its 16 z in FP32 per
// (column, trace) and carries FP64 totals; per-warp FP64 partials go to `partial` for a
// fixed-order final sum.
template <int VEL, int WGT, bool FAST, typename TT, int LPT>
__device__ void vg_consumer(MigSmem& S, const TT* data, const GeomParams& g, const TileShape& ts,
                            int x0, int y0, int z0, const TileBox& box, int bin,
                            const float* __restrict__ image, double* __restrict__ partial,
                            const WaitCfg& wc, float2* srcc)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int tx, ty, tzg;
    thread_column(ts, tid, tx, ty, tzg);
    const int ix = x0 + tx, iy = y0 + ty, izb = z0 + tzg * NZ;
    const bool col_ok = ix < g.nx && iy < g.ny;
    const float cxf = col_coord(g.ox, ix, g.dx);
    const float cyf = (g.dim == 3) ? col_coord(g.oy, iy, g.dy) : 0.f;
    const double xd = grid_coord(g.ox, ix, g.dx), yd = (g.dim == 3) ? grid_coord(g.oy, iy, g.dy) : 0.0;
    const float dxc = (float)(xd - box.cx), dyc = (float)(yd - box.cy);
    const float4* zc = &S.zc[tzg * NZ];
    const float* zg = &S.z2[tzg * NZ];   // linear: gamma(z)
    const int zero_off = (int)(((const char*)S.zero - (const char*)data) / (int)sizeof(TT));
    const float dtf = (float)g.dtd;
    const float inv_v0 = (float)(1.0 / g.v0), inv_v0sq = (float)(1.0 / (g.v0 * g.v0));
    const float inv_ka = (VEL == VK_LINEAR) ? (float)(1.0 / g.kabs) : 0.f;
    const float sgnk = g.k < 0.0 ? -1.f : 1.f;
    const float two_over_k = (VEL == VK_LINEAR) ? (float)(2.0 / g.k) : 0.f;
    const float inv_a = (VEL == VK_LINEAR) ? (float)(1.0 / g.a) : 0.f;
    const float zb = (float)(g.oz + izb * g.dz), dzf = (float)g.dz;

    // per thread and depth in shared memory: the image value times gamma(z) (the weight's depth
    // factor), and for linear v(z) the source-leg cache (C1 ln(1 + rho_s), (q/w)_s) and sqrt(q_s)
    float* my_mv = reinterpret_cast<float*>(srcc) + tid;
    float2* my_lq = srcc + NZ * CONSUMERS / 2 + tid;
    float* my_sq = reinterpret_cast<float*>(srcc) + 3 * NZ * CONSUMERS + tid;
#pragma unroll
    for (int i = 0; i < NZ; ++i) {
        const float m = (col_ok && izb + i < g.nz)
                            ? image[(((long long)bin * g.ny + iy) * g.nx + ix) * (long long)g.nz + izb + i]
                            : 0.f;
        my_mv[i * CONSUMERS] = (VEL == VK_LINEAR && WGT == 1) ? zg[i] * m : m;
    }
    double G0 = 0.0, G1 = 0.0;
    unsigned psx = 0xffffffffu, psy = 0xffffffffu;

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
            const int4 w = S.win[s][t];
            bool inside = col_ok;
            float tp = 1.f;   // aperture taper of this column
            if (g.use_aperture && w.z >= 0) {   // sign bit of w.z: every column is inside (its core)
                const float2 m = S.mid[s][t];
                inside = inside && in_aperture(cxf, cyf, m.x, m.y, g.A2);
                if (g.use_taper && inside) tp = aperture_taper(cxf, cyf, m.x, m.y, g);
            }
            if (!__any_sync(0xffffffffu, inside)) continue;
            const float c0rel = __int_as_float(w.x);
            const float cmid = __int_as_float(w.z & 0x7fffffff);
            const float chalf = inside ? __int_as_float(w.w & 0x7fffffff) : -1.f;
            const float tbase = S.tb[s][t];
            const float4 h = S.hdr[s][t];
            float g0 = 0.f, g1 = 0.f;
            if constexpr (VEL == VK_CONST) {
                const float dxs = cxf - h.x, dys = cyf - h.y;
                const float dxr = cxf - h.z, dyr = cyf - h.w;
                const float dhs2 = fmaf(dxs, dxs, dys * dys);
                const float dhr2 = fmaf(dxr, dxr, dyr * dyr);
#pragma unroll
                for (int i = 0; i < NZ; ++i) {
                    const float4 c = zc[i];
                    const float Rs = hsqrt<FAST>(dhs2 + c.x);
                    const float Rr = hsqrt<FAST>(dhr2 + c.x);
                    const float Ssum = Rs + Rr;
                    const float th = fmaf(Ssum, g.C1, fmaf(Ssum, g.C1lo, c0rel));
                    const float tm = __fadd_rd(fmaxf(th, 0.f), MAGIC);   // MAGIC + floor(th), th >= 0
                    const bool ok = fabsf(th - cmid) <= chalf;
                    const int off = ok ? __float_as_int(tm) + w.y : zero_off;
                    const float slope = to_f32<TT>(data[off]);   // slope rows: d[i + 1] - d[i]
                    const float W = (WGT == 1) ? zg[i] * Ssum : 1.f;
                    g0 = fmaf(W * my_mv[i * CONSUMERS] * slope, -Ssum * inv_v0sq, g0);
                }
            } else {
                const float4 rr = S.refr[s][t], a = S.hda[s][t];
                if (__float_as_uint(h.x) != psx || __float_as_uint(h.y) != psy) {   // new source
                    const float4 rs = S.refs[s][t];
                    const float dPs = fmaf(dxc, cxf + a.x, dyc * (cyf + a.y));
                    const float exs = cxf - h.x, eys = cyf - h.y;
                    const float dhs2 = fmaf(exs, exs, eys * eys);
#pragma unroll
                    for (int i = 0; i < NZ; ++i) {
                        float sqs, qws;
                        const float rho_s = leg_delta_grad_m<FAST>(dPs, dhs2, zc[i], rs, sqs, qws);
                        my_lq[i * CONSUMERS] = make_float2(leg_log<LPT>(rho_s, g, 0.f), qws);
                        my_sq[i * CONSUMERS] = sqs;
                    }
                    psx = __float_as_uint(h.x);
                    psy = __float_as_uint(h.y);
                }
                const float dPr = fmaf(dxc, cxf + a.z, dyc * (cyf + a.w));
                const float exr = cxf - h.z, eyr = cyf - h.w;
                const float dhr2 = fmaf(exr, exr, eyr * eyr);
#pragma unroll 4
                for (int i = 0; i < NZ; ++i) {
                    const float4 zk = zc[i];   // (alpha, alpha kappa, alpha dz2, alpha z^2)
                    float sqr, qwr;
                    const float rho_r = leg_delta_grad_m<FAST>(dPr, dhr2, zk, rr, sqr, qwr);
                    const float2 lq = my_lq[i * CONSUMERS];   // (C1 ln(1 + rho_s), (q/w)_s)
                    const float th = leg_log<LPT>(rho_r, g, c0rel + lq.x);
                    const float tm = __fadd_rd(fmaxf(th, 0.f), MAGIC);   // MAGIC + floor(th), th >= 0
                    const bool ok = fabsf(th - cmid) <= chalf;
                    const int off = ok ? __float_as_int(tm) + w.y : zero_off;
                    const float slope = to_f32<TT>(data[off]);   // slope rows: d[i + 1] - d[i]
                    // gamma(z) is folded into the stored image value
                    const float W = (WGT == 1) ? my_sq[i * CONSUMERS] + sqr : 1.f;
                    const float wms = W * my_mv[i * CONSUMERS] * slope;
                    const float inv_vz = zk.x * inv_a;
                    const float z = fmaf((float)i, dzf, zb);
                    const float qw = lq.y + qwr;
                    const float Tsum = fmaf(th, dtf, tbase);
                    const float dTv = -qw * (inv_v0 + inv_vz) * inv_ka;
                    const float dTk = (fmaf(qw, fmaf(-z, inv_vz, two_over_k), -sgnk * Tsum)) * inv_ka;
                    g0 = fmaf(wms, dTv, g0);
                    g1 = fmaf(wms, dTk, g1);
                }
            }
            G0 += (double)(g0 * tp);
            G1 += (double)(g1 * tp);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[s]);
        ++n;
        if (last) break;
    }
    if (failed) {
        if (lane == 0) atomicOr(wc.status, 1);
        G0 = 0.0;
        G1 = 0.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        G0 += __shfl_xor_sync(0xffffffffu, G0, o);
        G1 += __shfl_xor_sync(0xffffffffu, G1, o);
    }
    if (lane == 0) {
        const long long slot = ((long long)blockIdx.y * gridDim.x + blockIdx.x) * CONSUMER_WARPS + warp;
        partial[2 * slot] = G0;
        partial[2 * slot + 1] = G1;
    }
}

// Per-z constants of a tile's depth range [z0, z0 + cz NZ), written by all threads (the same
// layout in both modes).
template <int VEL, int MODE>
__device__ __forceinline__ void tile_z_setup(MigSmem& S, const GeomParams& g, const TileShape& ts, int z0,
                                             const TileBox& box)
{
    for (int i = threadIdx.x; i < ts.cz * NZ; i += blockDim.x) {
        const double z = grid_coord(g.oz, z0 + i, g.dz);
        if constexpr (VEL == VK_LINEAR) {
            float gamma;
            S.zc[i] = z_constants_m(z, box.cz, g, gamma);
            S.z2[i] = gamma;
        } else if constexpr (VEL == VK_TABLE || VEL == VK_GRID) {
            const float wz = (g.weight == 1 && fabs(z) >= 1e-6 * fabs(g.dz)) ? (float)(z * g.wscale) : 0.f;
            S.zc[i] = make_float4(wz, (float)(z * z), 0.f, 0.f);
        } else if constexpr (VEL == VK_PSTM) {
            // time migration: z is the two-way vertical time t0; the leg is the straight ray of
            // the RMS velocity, R = sqrt(h^2 + ze^2) with ze = v_rms t0 / 2, and
            // tau = (R_s + R_r) C1(t0) - t0/dt with C1(t0) = 1 / (v_rms dt); stored relative to the
            // tile centre: (ze^2, ze^2 - ze_c^2, C1(t0), C1(t0) - C1(t0_c)), and w_z = ze / (2 r0^2)
            const PstmTile pt = pstm_tile(g, box);
            const double vr = sqrt(vrms2_of(g.v0, g.pk, z));
            const double ze = 0.5 * vr * z;
            const double c1 = 1.0 / (vr * g.dtd);
            S.zc[i] = make_float4((float)(ze * ze), (float)(ze * ze - pt.pze2), (float)c1, (float)(c1 - pt.pc1));
            S.z2[i] = (g.weight == 1 && fabs(z) >= 1e-6 * fabs(g.dz)) ? (float)(ze * g.wscale) : 0.f;
        } else {
            // constant velocity: (z^2, z^2 - z_c^2, z, 1 off the surface row: where the true-amplitude
            // weight is defined), and w_z of the obliquity weight
            const double dq = __dadd_rn(__dmul_rn(z, z), -__dmul_rn(box.cz, box.cz));
            S.zc[i] = make_float4((float)(z * z), (float)dq, (float)z, fabs(z) >= 1e-6 * fabs(g.dz) ? 1.f : 0.f);
            S.z2[i] = (g.weight == 1 && fabs(z) >= 1e-6 * fabs(g.dz)) ? (float)(z * g.wscale) : 0.f;
        }
    }
}

// Shared body of the migration kernel (MODE 0: image out) and of the gradient kernel
// (MODE 1: image in, per-warp partials out).
template <int VEL, int WGT, bool FAST, typename TT, int LPT, int MODE, typename TB = float>
__device__ __forceinline__ void kernel_body(const GeomParams& g, const TileShape& ts, const TraceSet& tr,
                                            const TT* __restrict__ traces, float* __restrict__ image,
                                            int cap, const WaitCfg& wc, double* __restrict__ partial)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MigSmem& S = *reinterpret_cast<MigSmem*>(smem_raw);
    TT* ring = reinterpret_cast<TT*>(smem_raw + mig_static_bytes());
    TT* data = ring + LEAD;
    __shared__ int s_abort;
    const int bin = blockIdx.y;
    int t = blockIdx.x;
    const int tzi = t % ts.tiles_z;
    t /= ts.tiles_z;
    const int txi = t % ts.tiles_x, tyi = t / ts.tiles_x;
    const int x0 = txi * ts.cx, y0 = tyi * ts.cy, z0 = tzi * ts.cz * NZ;

    const TileBox box = tile_box(g, x0, y0, z0, ts.cx, ts.cy, ts.cz * NZ);

    if (threadIdx.x == 0) {
        // a wait in another CTA of this plan already ran out: results are invalid anyway (the
        // other status bits report skipped inputs, not a stalled launch)
        s_abort = *reinterpret_cast<const volatile int*>(wc.status) & 1;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], CONSUMER_WARPS);
        }
        S.zero[0] = S.zero[1] = S.zero[2] = S.zero[3] = 0.f;
        tile_cells(S.row, tr, box);
        fence_barrier_init();
    }
    // per-z constants of the tile and a zero-filled ring (edge reads stay finite)
    tile_z_setup<VEL, MODE>(S, g, ts, z0, box);
    {
        const int total = LEAD + STAGES * cap + SLACK;
        for (int i = threadIdx.x; i < total; i += blockDim.x) ring[i] = TT(0.f);
    }
    TB* tab = reinterpret_cast<TB*>(smem_raw + mig_static_bytes() + mig_ring_bytes(g));
    float2* srcc = reinterpret_cast<float2*>(smem_raw + mig_static_bytes() + mig_ring_bytes(g) + table_bytes(g));
    if constexpr (VEL == VK_TABLE) {
        const uint4* src = reinterpret_cast<const uint4*>(g.table);
        uint4* dst = reinterpret_cast<uint4*>(tab);
        const int n16 = (int)(table_bytes(g) / 16);
        for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    if (s_abort) return;
    if (threadIdx.x >= CONSUMERS) {
        mig_producer<VEL, TT, WGT>(S, data, cap, g, tr, traces, bin, box, wc, 0, (int)blockIdx.x);
    } else if constexpr (MODE == 0) {
        mig_consumer<VEL, WGT, FAST, TT, LPT, TB>(S, data, g, ts, x0, y0, z0, box, bin, image, wc, tab, srcc, cap,
                                                  0);
    } else {
        vg_consumer<VEL, WGT, FAST, TT, LPT>(S, data, g, ts, x0, y0, z0, box, bin, image, partial, wc, srcc);
    }
}

template <int VEL, int WGT, bool FAST, typename TT, int LPT, typename TB = float>
__global__ void __launch_bounds__(THREADS, 2)
    k_migrate(GeomParams g, TileShape ts, TraceSet tr, const TT* __restrict__ traces,
              float* __restrict__ image, int cap, WaitCfg wc)
{
    kernel_body<VEL, WGT, FAST, TT, LPT, 0, TB>(g, ts, tr, traces, image, cap, wc, nullptr);
}

template <int VEL, int WGT, bool FAST, typename TT, int LPT>
__global__ void __launch_bounds__(THREADS, 2)
    k_vgrad(GeomParams g, TileShape ts, TraceSet tr, const TT* __restrict__ traces,
            const float* __restrict__ image, int cap, WaitCfg wc, double* __restrict__ partial)
{
    kernel_body<VEL, WGT, FAST, TT, LPT, 1>(g, ts, tr, traces, const_cast<float*>(image), cap, wc, partial);
}

// ------------------------------------------------------------------ launch (per trace type)
template <int VEL, int WGT, bool FAST, typename TT>
static cudaError_t launch_migrate_t(const GeomParams& g, const TileShape& t, const TraceSet& tr,
                                   const void* traces, float* image, const WaitCfg& w, cudaStream_t s)
{
    const size_t smem = mig_smem_bytes(g);
    const dim3 grid((unsigned)(t.tiles_x * t.tiles_y * t.tiles_z), (unsigned)g.n_bins);
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, THREADS, smem, s>>>(g, t, tr, static_cast<const TT*>(traces), image, mig_cap(g), w);
        return cudaGetLastError();
    };
    if constexpr (VEL == VK_LINEAR) {
        return with_lg<FAST>(g.lg_terms,
                             [&](auto L) { return go(k_migrate<VEL, WGT, FAST, TT, decltype(L)::value>); });
    } else if constexpr (VEL == VK_GRID) {
        // the LPT slot carries the tables' depth-node stride M
        switch (g.tm) {
            case 1: return go(k_migrate<VEL, WGT, FAST, TT, 1>);
            case 2: return go(k_migrate<VEL, WGT, FAST, TT, 2>);
            case 4: return go(k_migrate<VEL, WGT, FAST, TT, 4>);
            default: return cudaErrorInvalidValue;
        }
    } else if constexpr (VEL == VK_TABLE) {
        // the LPT slot carries the table's depth-node stride M
        auto tb = [&](auto M) -> cudaError_t {
            constexpr int m = decltype(M)::value;
            if (g.tdt == KH_F16) return go(k_migrate<VEL, WGT, FAST, TT, m, __half>);
            if (g.tdt == KH_U16) return go(k_migrate<VEL, WGT, FAST, TT, m, unsigned short>);
            return go(k_migrate<VEL, WGT, FAST, TT, m, float>);
        };
        switch (g.tm) {
            case 1: return tb(std::integral_constant<int, 1>());
            case 2: return tb(std::integral_constant<int, 2>());
            case 4: return tb(std::integral_constant<int, 4>());
            default: return cudaErrorInvalidValue;
        }
    } else {
        return go(k_migrate<VEL, WGT, FAST, TT, LP_SHORT>);
    }
}

// Operator anti-aliasing (g.aa_c > 0): the kernels compiled with the W_AA bit, instantiated in
// translation units of their own (kh_migrate_aa_<type>.cu) so that they build beside the others;
// constant velocity for every trace type, v0 + k z for FP32 traces (the plan refuses the others).
template <typename TT>
cudaError_t launch_migrate_aa_t(const GeomParams& g, const TileShape& t, const TraceSet& tr, const void* traces,
                                float* image, int vel, int fast, const WaitCfg& w, cudaStream_t s)
{
    if (vel == VK_LINEAR) {   // v0 + k z: FP32 traces only (the plan refuses the others)
        if constexpr (std::is_same<TT, float>::value || std::is_same<TT, SamplePair>::value) {
            switch (g.weight * 2 + (fast ? 1 : 0)) {
                case 0: return launch_migrate_t<VK_LINEAR, W_AA | 0, false, TT>(g, t, tr, traces, image, w, s);
                case 1: return launch_migrate_t<VK_LINEAR, W_AA | 0, true, TT>(g, t, tr, traces, image, w, s);
                case 2: return launch_migrate_t<VK_LINEAR, W_AA | 1, false, TT>(g, t, tr, traces, image, w, s);
                case 3: return launch_migrate_t<VK_LINEAR, W_AA | 1, true, TT>(g, t, tr, traces, image, w, s);
                default: return cudaErrorInvalidValue;
            }
        } else {
            return cudaErrorInvalidValue;
        }
    }
    if (vel != VK_CONST) return cudaErrorInvalidValue;
    switch (g.weight * 2 + (fast ? 1 : 0)) {
        case 0: return launch_migrate_t<VK_CONST, W_AA | 0, false, TT>(g, t, tr, traces, image, w, s);
        case 1: return launch_migrate_t<VK_CONST, W_AA | 0, true, TT>(g, t, tr, traces, image, w, s);
        case 2: return launch_migrate_t<VK_CONST, W_AA | 1, false, TT>(g, t, tr, traces, image, w, s);
        case 3: return launch_migrate_t<VK_CONST, W_AA | 1, true, TT>(g, t, tr, traces, image, w, s);
        case 4: return launch_migrate_t<VK_CONST, W_AA | 2, false, TT>(g, t, tr, traces, image, w, s);
        case 5: return launch_migrate_t<VK_CONST, W_AA | 2, true, TT>(g, t, tr, traces, image, w, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename TT>
cudaError_t launch_migrate_dtype(const GeomParams& g, const TileShape& t, const TraceSet& tr, const void* traces,
                                 float* image, int vel, int fast, const WaitCfg& w, cudaStream_t s)
{
    if (g.weight == KH_W_TRUE_AMP) {   // constant velocity only (the plan refuses the others)
        if (vel != VK_CONST) return cudaErrorInvalidValue;
        return fast ? launch_migrate_t<VK_CONST, 2, true, TT>(g, t, tr, traces, image, w, s)
                    : launch_migrate_t<VK_CONST, 2, false, TT>(g, t, tr, traces, image, w, s);
    }
    const int key = vel * 4 + g.weight * 2 + (fast ? 1 : 0);
    switch (key) {
        case 0: return launch_migrate_t<VK_CONST, 0, false, TT>(g, t, tr, traces, image, w, s);
        case 1: return launch_migrate_t<VK_CONST, 0, true, TT>(g, t, tr, traces, image, w, s);
        case 2: return launch_migrate_t<VK_CONST, 1, false, TT>(g, t, tr, traces, image, w, s);
        case 3: return launch_migrate_t<VK_CONST, 1, true, TT>(g, t, tr, traces, image, w, s);
        case 4: return launch_migrate_t<VK_LINEAR, 0, false, TT>(g, t, tr, traces, image, w, s);
        case 5: return launch_migrate_t<VK_LINEAR, 0, true, TT>(g, t, tr, traces, image, w, s);
        case 6: return launch_migrate_t<VK_LINEAR, 1, false, TT>(g, t, tr, traces, image, w, s);
        case 7: return launch_migrate_t<VK_LINEAR, 1, true, TT>(g, t, tr, traces, image, w, s);
        case 8:
        case 9: return launch_migrate_t<VK_TABLE, 0, true, TT>(g, t, tr, traces, image, w, s);
        case 10:
        case 11: return launch_migrate_t<VK_TABLE, 1, true, TT>(g, t, tr, traces, image, w, s);
        case 12: return launch_migrate_t<VK_PSTM, 0, false, TT>(g, t, tr, traces, image, w, s);
        case 13: return launch_migrate_t<VK_PSTM, 0, true, TT>(g, t, tr, traces, image, w, s);
        case 14: return launch_migrate_t<VK_PSTM, 1, false, TT>(g, t, tr, traces, image, w, s);
        case 15: return launch_migrate_t<VK_PSTM, 1, true, TT>(g, t, tr, traces, image, w, s);
        case 16:
        case 17: return launch_migrate_t<VK_GRID, 0, true, TT>(g, t, tr, traces, image, w, s);
        case 18:
        case 19: return launch_migrate_t<VK_GRID, 1, true, TT>(g, t, tr, traces, image, w, s);
        default: return cudaErrorInvalidValue;
    }
}

// Gradient kernel (FP32 traces, analytic traveltimes only).
template <int VEL, int WGT, bool FAST>
static cudaError_t launch_vgrad_t(const GeomParams& g, const TileShape& t, const TraceSet& tr,
                                 const float* traces, const float* image, const WaitCfg& w, double* partial,
                                 cudaStream_t s)
{
    const size_t smem = mig_smem_bytes(g);
    const dim3 grid((unsigned)(t.tiles_x * t.tiles_y * t.tiles_z), (unsigned)g.n_bins);
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, THREADS, smem, s>>>(g, t, tr, traces, image, mig_cap(g), w, partial);
        return cudaGetLastError();
    };
    if constexpr (VEL == VK_LINEAR)
        return with_lg<FAST>(g.lg_terms,
                             [&](auto L) { return go(k_vgrad<VEL, WGT, FAST, float, decltype(L)::value>); });
    else
        return go(k_vgrad<VEL, WGT, FAST, float, LP_SHORT>);
}

// ------------------------------------------------------------------ batched persistent launch
// One CTA per (SM, resident slot) loops over a work list of (job, tile, bin) items, longest
// first, taking the next item from one global counter (a scheduler index, never image data).
// Each item is the tile computation of k_migrate with the job's own geometry, tile shape,
// headers, traces and image; the mbarrier ring and its phases persist across items.  All jobs
// of one launch share the ln(1 + rho) fit length LPT (the host launches the jobs of each fit
// length separately).  A wait that ran out anywhere in the launch (status word) stops
// every CTA at its next item.
template <int VEL, int WGT, bool FAST, typename TT, int LPT>
__global__ void __launch_bounds__(THREADS, 2)
    k_migrate_batched(const BatchJob* __restrict__ jobs, const int4* __restrict__ items, int n_items,
                      int* __restrict__ next, GeomParams g_ring, WaitCfg wc)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MigSmem& S = *reinterpret_cast<MigSmem*>(smem_raw);
    TT* ring = reinterpret_cast<TT*>(smem_raw + mig_static_bytes());
    TT* data = ring + LEAD;
    float2* srcc = reinterpret_cast<float2*>(smem_raw + mig_static_bytes() + mig_ring_bytes(g_ring));
    __shared__ int s_item;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], CONSUMER_WARPS);
        }
        S.zero[0] = S.zero[1] = S.zero[2] = S.zero[3] = 0.f;
        fence_barrier_init();
    }
    const int cap = mig_cap(g_ring);
    for (int i = threadIdx.x; i < LEAD + STAGES * cap + SLACK; i += blockDim.x) ring[i] = TT(0.f);
    int n = 0;   // stages filled (producer warp) or consumed (consumer warps) so far
    while (true) {
        __syncthreads();   // the previous item's per-z constants and s_item are no longer read
        if (threadIdx.x == 0) {
            const int bad = *reinterpret_cast<const volatile int*>(wc.status);
            s_item = bad ? n_items : atomicAdd(next, 1);
        }
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int4 w = items[it];
        const GeomParams g = jobs[w.x].g;
        const TileShape ts = jobs[w.x].ts;
        const TraceSet tr = jobs[w.x].tr;
        int t = w.y;
        const int tzi = t % ts.tiles_z;
        t /= ts.tiles_z;
        const int txi = t % ts.tiles_x, tyi = t / ts.tiles_x;
        const int x0 = txi * ts.cx, y0 = tyi * ts.cy, z0 = tzi * ts.cz * NZ;
        const int bin = w.z;
        const TileBox box = tile_box(g, x0, y0, z0, ts.cx, ts.cy, ts.cz * NZ);
        tile_z_setup<VEL, 0>(S, g, ts, z0, box);
        if (threadIdx.x == 0) tile_cells(S.row, tr, box);
        __syncthreads();
        if (threadIdx.x >= CONSUMERS) {
            n = mig_producer<VEL, TT>(S, data, cap, g, tr, static_cast<const TT*>(jobs[w.x].traces),
                                      bin, box, wc, n);
        } else {
            n = mig_consumer<VEL, WGT, FAST, TT, LPT, float>(S, data, g, ts, x0, y0, z0, box, bin,
                                                             jobs[w.x].image, wc, nullptr, srcc, cap, n);
        }
    }
}

template <int VEL, int WGT, bool FAST, typename TT>
static cudaError_t launch_batched_t(const GeomParams& gm, const BatchJob* jobs, const int4* items,
                                   int n_items, int* next, int lg_terms, const WaitCfg& w, int ctas,
                                   int* ctas_out, cudaStream_t s)
{
    const size_t smem = mig_smem_bytes(gm);
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e;
        if (ctas <= 0) {   // set-up only: shared-memory attribute and the occupancy-sized grid
            int dev = 0, nsm = 0, occ = 0;
            if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                cudaSuccess)
                return e;
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, THREADS, smem)) != cudaSuccess)
                return e;
            int c = nsm * (occ > 0 ? occ : 1);
            if (c > n_items) c = n_items;
            if (ctas_out) *ctas_out = c;
            return cudaSuccess;
        }
        kern<<<ctas, THREADS, smem, s>>>(jobs, items, n_items, next, gm, w);
        return cudaGetLastError();
    };
    if constexpr (VEL == VK_LINEAR)
        return with_lg<FAST>(lg_terms,
                             [&](auto L) { return go(k_migrate_batched<VEL, WGT, FAST, TT, decltype(L)::value>); });
    else
        return go(k_migrate_batched<VEL, WGT, FAST, TT, LP_SHORT>);
}

template <typename TT>
cudaError_t launch_batched_dtype(const GeomParams& gm, const BatchJob* jobs, const int4* items, int n_items,
                                 int* next, int vel, int weight, int fast, int lg_terms, const WaitCfg& w,
                                 int ctas, int* ctas_out, cudaStream_t s)
{
    const int key = vel * 4 + weight * 2 + (fast ? 1 : 0);
    switch (key) {
        case 0: return launch_batched_t<VK_CONST, 0, false, TT>(gm, jobs, items, n_items, next, lg_terms, w, ctas, ctas_out, s);
        case 1: return launch_batched_t<VK_CONST, 0, true, TT>(gm, jobs, items, n_items, next, lg_terms, w, ctas, ctas_out, s);
        case 2: return launch_batched_t<VK_CONST, 1, false, TT>(gm, jobs, items, n_items, next, lg_terms, w, ctas, ctas_out, s);
        case 3: return launch_batched_t<VK_CONST, 1, true, TT>(gm, jobs, items, n_items, next, lg_terms, w, ctas, ctas_out, s);
        case 4: return launch_batched_t<VK_LINEAR, 0, false, TT>(gm, jobs, items, n_items, next, lg_terms, w, ctas, ctas_out, s);
        case 5: return launch_batched_t<VK_LINEAR, 0, true, TT>(gm, jobs, items, n_items, next, lg_terms, w, ctas, ctas_out, s);
        case 6: return launch_batched_t<VK_LINEAR, 1, false, TT>(gm, jobs, items, n_items, next, lg_terms, w, ctas, ctas_out, s);
        case 7: return launch_batched_t<VK_LINEAR, 1, true, TT>(gm, jobs, items, n_items, next, lg_terms, w, ctas, ctas_out, s);
        default: return cudaErrorInvalidValue;
    }
}


}  // namespace kh
