// Device helpers: shared-memory mbarriers, bulk async copies (non-multicast), bounded
// waits and the fast-math primitives of the hot loop.  sm_100+ PTX, written for sm_103a.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kh_internal.h"

namespace kh {

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Makes barrier initialisation visible to the async (bulk-copy) proxy.
__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking probe of the phase (used when a poll budget is set, so one poll is one probe).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of `bar` with the given parity to complete.  Gives up, returning
// false, after `polls` polls (if > 0), after `ns` nanoseconds of wall clock, or as soon as
// another CTA has raised the status word (if `status` is not NULL).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long polls,
                                                  long long ns, const int* status)
{
    if (polls > 0) {
        for (long long i = 0; i < polls; ++i)
            if (mbar_test_wait(bar, parity)) return true;
        return false;
    }
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 0) {
            if ((long long)(global_ns() - t0) > ns) return false;
            if (status && *reinterpret_cast<const volatile int*>(status) != 0) return false;
        }
    }
}

// Every lane of the warp waits (so each lane acquires the phase) and the warp agrees on the
// outcome, so a wait that runs out for one lane ends the loop for all lanes together.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, long long polls,
                                          long long ns, const int* status)
{
    const bool ok = mbar_wait_bounded(bar, parity, polls, ns, status);
    return __all_sync(0xffffffffu, ok);
}

// One contiguous global -> shared copy by the bulk-copy engine; completion is counted in
// bytes on `bar`.  dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---- hot-loop math: hardware approximations (FAST) or IEEE-rounded / accurate library calls
template <bool FAST>
__device__ __forceinline__ float hsqrt(float x)
{
    if constexpr (FAST) {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    } else {
        return __fsqrt_rn(x);
    }
}

template <bool FAST>
__device__ __forceinline__ float hrsqrt(float x)
{
    if constexpr (FAST) {
        float r;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    } else {
        return __frcp_rn(__fsqrt_rn(x));
    }
}

template <bool FAST>
__device__ __forceinline__ float hrcp(float x)
{
    if constexpr (FAST) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    } else {
        return __frcp_rn(x);
    }
}

template <bool FAST>
__device__ __forceinline__ float hlog2(float x)
{
    if constexpr (FAST) {
        float r;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    } else {
        return log2f(x);
    }
}

// Grid coordinate o + i h in FP64 without contraction (the same value in every kernel).
__device__ __forceinline__ double grid_coord(double o, int i, double h)
{
    return __dadd_rn(o, __dmul_rn((double)i, h));
}

// True-amplitude weight (KH_W_TRUE_AMP, constant velocity): the weight of the asymptotic Kirchhoff
// inversion for the reflection coefficient with its global constants dropped,
//     W = (R_s R_r)^((dim - 1) / 2) |det[g, D u_x (, D u_y)]| / |g|^2,
// g = e_s + e_r, e_a = (x - a) / R_a, D u = sum_a (u - e_a (e_a . u)) / R_a.  Evaluated in closed form:
// with c = e_s . e_r, D acts on the normal of span{e_s, e_r} as 1/R_s + 1/R_r and its adjugate maps
// g to (1/R_s + 1/R_r)(1 + c)(e_s / R_s + e_r / R_r) (3D), while |g|^2 = 2 (1 + c), so
//     3D: W = z (R_s + R_r) (1/R_s^2 + 1/R_r^2) / 2,    2D: W = z sqrt(R_s R_r) (1/R_s^2 + 1/R_r^2) / 2,
// free of the cancellation of the determinant's entries (e.g. 1 - e_x^2 near horizontal rays).
template <bool FAST>
__device__ __forceinline__ float ta_weight_r(float z, float Rs, float Rr, float is, float ir, bool three_d)
{
    const float s2 = fmaf(is, is, ir * ir);   // is = 1 / R_s, ir = 1 / R_r
    return 0.5f * z * (three_d ? Rs + Rr : hsqrt<FAST>(Rs * Rr)) * s2;
}

template <bool FAST>
__device__ __forceinline__ float ta_weight(float z, float Rs, float Rr, bool three_d)
{
    return ta_weight_r<FAST>(z, Rs, Rr, hrcp<FAST>(Rs), hrcp<FAST>(Rr), three_d);
}

// Operator anti-aliasing weight (constant velocity, aa_c = trace spacing / (v0 dt) > 0): the moveout
// between adjacent traces L = aa_c max(|p_x|, |p_y|) samples, p = (x - s)_h / R_s + (x - r)_h / R_r;
// 1 up to one sample, 0 from two, cos^2(pi (L - 1) / 2) between.  (dxa, dya): column minus point a.
// is, ir: 1 / R_s, 1 / R_r (1 / max(R, 1e-30)).
__device__ __forceinline__ float aa_weight_r(float aa_c, float dxs, float dys, float dxr, float dyr, float is, float ir)
{
    const float L = aa_c * fmaxf(fabsf(fmaf(dxs, is, dxr * ir)), fabsf(fmaf(dys, is, dyr * ir)));
    if (L <= 1.f) return 1.f;
    if (L >= 2.f) return 0.f;
    const float c = __cosf(1.57079632679f * (L - 1.f));
    return c * c;
}

template <bool FAST>
__device__ __forceinline__ float aa_weight(float aa_c, float dxs, float dys, float dxr, float dyr, float Rs, float Rr)
{
    return aa_weight_r(aa_c, dxs, dys, dxr, dyr, hrcp<FAST>(fmaxf(Rs, 1e-30f)), hrcp<FAST>(fmaxf(Rr, 1e-30f)));
}

// Warp-uniform class of the anti-aliasing weight over one trace's contributions to the active
// lanes' columns over a range of depths: 0 every weight is 0 (L >= 2), 1 every weight is 1
// (L <= 1), 2 mixed.  A component a f_s + b f_r of p (a, b: the column's horizontal offsets from
// source and receiver along one axis, f_a the leg's factor at the depth) has terms of fixed sign
// whose size falls with depth when f_a does: the component is at most its terms' sizes at the
// shallowest depth (fs0, fr0) summed, and at least, over the whole range, their sizes at the
// deepest depth (fs1, fr1) summed where a and b share a sign, else the larger of (deepest size of
// one term) - (shallowest size of the other).  Classes decided on these bounds differ from the
// per-contribution weight only where FP32 rounding puts L at 1 or 2, where the weight's slope is 0.
__device__ __forceinline__ int aa_class_f(float aa_c, float dxs, float dys, float dxr, float dyr, float fs0,
                                          float fs1, float fr0, float fr1, bool active)
{
    auto comp = [&](float a, float b, float& ub, float& lb) {
        const float a0 = fabsf(a) * fs0, a1 = fabsf(a) * fs1, b0 = fabsf(b) * fr0, b1 = fabsf(b) * fr1;
        ub = a0 + b0;
        lb = (a * b >= 0.f) ? a1 + b1 : fmaxf(fmaxf(a1 - b0, b1 - a0), 0.f);
    };
    float ubx, lbx, uby, lby;
    comp(dxs, dxr, ubx, lbx);
    comp(dys, dyr, uby, lby);
    if (__all_sync(0xffffffffu, !active || aa_c * fmaxf(lbx, lby) >= 2.f)) return 0;
    if (__all_sync(0xffffffffu, !active || aa_c * fmaxf(ubx, uby) <= 1.f)) return 1;
    return 2;
}

// Constant velocity: f_a = 1 / R_a (1 / v0 is in aa_c), falling with z^2 over [z2lo, z2hi].
__device__ __forceinline__ int aa_class(float aa_c, float dxs, float dys, float dxr, float dyr, float z2lo,
                                        float z2hi, bool active)
{
    const float hs2 = fmaf(dxs, dxs, dys * dys), hr2 = fmaf(dxr, dxr, dyr * dyr);
    return aa_class_f(aa_c, dxs, dys, dxr, dyr, rsqrtf(fmaxf(hs2 + z2lo, 1e-30f)), rsqrtf(fmaxf(hs2 + z2hi, 1e-30f)),
                      rsqrtf(fmaxf(hr2 + z2lo, 1e-30f)), rsqrtf(fmaxf(hr2 + z2hi, 1e-30f)), active);
}

// v0 + k z: a leg's factor, the size of its time's horizontal gradient per metre of horizontal
// offset, 1 / (R g sqrt(1 + s^2)) = 1 / sqrt(R^2 (v0 (v0 + k z) + k^2 R^2 / 4)) with R^2 = h^2 + z^2
// (vv = v0 (v0 + k z), kq = k^2 / 4).
__device__ __forceinline__ float aa_leg_lin(float R2, float vv, float kq)
{
    return rsqrtf(fmaxf(R2 * fmaf(kq, R2, vv), 1e-30f));
}

// v0 + k z over the depths [ztop, zbot]: for k >= 0 and ztop >= 0 both R^2 and v0 + k z grow with
// depth, so each factor falls; otherwise no bound (every weight evaluated).
__device__ __forceinline__ int aa_class_lin(const GeomParams& g, float dxs, float dys, float dxr, float dyr,
                                            float ztop, float zbot, bool active)
{
    float fs0 = 3e38f, fs1 = 0.f, fr0 = 3e38f, fr1 = 0.f;
    if (g.aa_v0k >= 0.f && ztop >= 0.f) {
        const float hs2 = fmaf(dxs, dxs, dys * dys), hr2 = fmaf(dxr, dxr, dyr * dyr);
        const float vv0 = fmaf(g.aa_v0k, ztop, g.aa_v0sq), vv1 = fmaf(g.aa_v0k, zbot, g.aa_v0sq);
        fs0 = aa_leg_lin(fmaf(ztop, ztop, hs2), vv0, g.aa_kq);
        fs1 = aa_leg_lin(fmaf(zbot, zbot, hs2), vv1, g.aa_kq);
        fr0 = aa_leg_lin(fmaf(ztop, ztop, hr2), vv0, g.aa_kq);
        fr1 = aa_leg_lin(fmaf(zbot, zbot, hr2), vv1, g.aa_kq);
    }
    return aa_class_f(g.aa_c, dxs, dys, dxr, dyr, fs0, fs1, fr0, fr1, active);
}

// Gridded model (KH_VEL_GRID): node column gi of image column ix in the tables' node grid and the
// column's fraction between node columns gi and gi + 1 (FP64, clamped so that gi + 1 is a node);
// the migration's reads and the tile bounds both take it from here.
__device__ __forceinline__ int grid_col(const GeomParams& g, int ix, float* frac)
{
    const double u = __ddiv_rn(__dadd_rn(grid_coord(g.ox, ix, g.dx), -g.gox), g.gh);
    int gi = (int)floor(u);
    gi = gi < 0 ? 0 : (gi > g.gnx - 2 ? g.gnx - 2 : gi);
    if (frac) *frac = (float)(u - (double)gi);
    return gi;
}

// Column coordinate o + i h in FP64 without contraction, rounded to FP32 (the same value the
// aperture decision uses everywhere).
__device__ __forceinline__ float col_coord(double o, int i, double h)
{
    return (float)__dadd_rn(o, __dmul_rn((double)i, h));
}

// The aperture decision in FP32 with a fixed order and no contraction.
__device__ __forceinline__ bool in_aperture(float cx, float cy, float mx, float my, float A2)
{
    const float ex = __fsub_rn(cx, mx), ey = __fsub_rn(cy, my);
    return __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)) <= A2;
}

// Aperture taper of a column inside the aperture: 1 within the core radius, then a raised cosine
// of the horizontal distance d to the trace midpoint, (1 + cos(pi (d - core) / band)) / 2, down
// to 0 at the aperture.
__device__ __forceinline__ float aperture_taper(float cx, float cy, float mx, float my, const GeomParams& g)
{
    const float ex = __fsub_rn(cx, mx), ey = __fsub_rn(cy, my);
    const float d2 = __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey));
    if (d2 <= g.ap_core2) return 1.f;
    const float x = fminf(__fmul_rn(__fsub_rn(sqrtf(d2), g.ap_core), g.ap_invband), 1.f);
    return 0.5f + 0.5f * cospif(x);
}

// Offset bin in FP64 (uniform bins; X == n_bins * w goes to the last bin; beyond: -1).
__device__ __forceinline__ int offset_bin(float sx, float sy, float rx, float ry, int n_bins,
                                          double w)
{
    const double ex = __dadd_rn((double)sx, -(double)rx);
    const double ey = __dadd_rn((double)sy, -(double)ry);
    const double X = __dsqrt_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)));
    const double b = floor(__ddiv_rn(X, w));
    if (b < (double)n_bins) return (int)b;
    if (X == __dmul_rn((double)n_bins, w)) return n_bins - 1;
    return -1;
}

// One-way traveltime in FP32 for window bounds (not the hot loop): constant or linear v(z).
// Every operation is rounded explicitly (no contraction), so that every kernel that bounds a
// window gets the same bounds, and with them the same window-relative times.
__device__ __forceinline__ float tt_bound(float h, float z, int vel, float v0, float k)
{
    const float R = __fsqrt_rn(__fadd_rn(__fmul_rn(h, h), __fmul_rn(z, z)));
    if (vel == VK_CONST || k == 0.f) return __fdiv_rn(R, v0);
    const float vz = __fadd_rn(v0, __fmul_rn(k, z));
    const float g = __fsqrt_rn(__fmul_rn(v0, vz));
    const float s = __fdiv_rn(__fmul_rn(fabsf(k), R), __fmul_rn(2.f, g));
    if (s < 1e-3f) return __fmul_rn(__fdiv_rn(R, g), __fsub_rn(1.f, __fmul_rn(__fmul_rn(s, s), 1.f / 6.f)));
    return __fdiv_rn(__fmul_rn(2.f, asinhf(s)), fabsf(k));
}

}  // namespace kh
