// The two-way time tau = (T_s + T_r - t0)/dt of one (image point, trace) pair, as the
// migration, demigration and gradient kernels evaluate it.
//
// Constant velocity: tau from R_s + R_r directly (two square roots).
//
// Linear v(z) = v0 + k z: T = arccosh(1 + q)/|k|, q = k^2 R^2 / (2 v0 (v0 + k z)), so
// e^{|k| T} = u = 1 + q + w with w = sqrt(q (q + 2)).  Evaluated directly in FP32 this
// loses ~1e-7 of T (about 3e-5 samples at T ~ 1 s), too much for 1e-5 image parity.
// Instead every (tile, trace) pair gets an FP64 reference at the tile centre c (computed
// once by the staging warp, or per lane in the adjoint), and each point evaluates only the
// change relative to it in cancellation-free form:
//     q - q_c = alpha(z) (dP + kappa(z) R_c^2 + (z^2 - z_c^2)),   dP = |x_h - s_h|^2 - |c_h - s_h|^2
//             = alpha(z) ((x_h - c_h).(x_h + c_h - 2 s_h) + ...),  kappa(z) = -k (z - z_c)/(v0 + k z_c)
//     w - w_c = (q - q_c)(q + q_c + 2)/(w + w_c)
//     u/u_c - 1 = (q - q_c)(1 + (q + q_c + 2)/(w + w_c)) / u_c
//     tau - tau_c = (ln(u_s/u_sc) + ln(u_r/u_rc)) / (|k| dt),
// with the per-z products alpha, alpha kappa, alpha (z^2 - z_c^2), alpha z^2 formed in FP64,
// and each leg's ln(1 + rho) from a polynomial fitted on the host for the tile's per-leg
// |rho| bound (leg_log), so that the source leg's term can be cached or shared.
#pragma once

#include <type_traits>

#include "kh_device.cuh"

namespace kh {

// Per-leg fit lengths of the kernels (migration, adjoint, gradient): every length of LG_TERMS
// with the fast
// math variants; the IEEE variants take LG_MONO (monomial) or LP_LONG (shifted), the
// coefficients beyond the fitted length being zero.
template <bool FAST, typename F>
cudaError_t with_lg(int terms, F&& f)
{
    if constexpr (FAST) {
        switch (terms) {
            case 4: return f(std::integral_constant<int, 4>());
            case 5: return f(std::integral_constant<int, 5>());
            case 6: return f(std::integral_constant<int, 6>());
            case 8: return f(std::integral_constant<int, 8>());
            case 12: return f(std::integral_constant<int, 12>());
            case 20: return f(std::integral_constant<int, 20>());
            default: return cudaErrorInvalidValue;
        }
    } else {
        if (terms <= LG_MONO) return f(std::integral_constant<int, LG_MONO>());
        if (terms <= LP_LONG) return f(std::integral_constant<int, LP_LONG>());
        return cudaErrorInvalidValue;
    }
}

// Per-(tile, trace) data of one leg, FP32 copies of FP64 values.
struct LegRef {
    float Rc2;   // |c - x_a|^2
    float qc;    // q at the tile centre
    float wc;    // sqrt(q_c (q_c + 2))
    float iuc;   // 1 / u_c
};

// FP64 reference of one leg: returns ln u_c and fills the FP32 copies (and, if qc2i is given,
// (q_c + 2)/u_c, the form the kernels' leg evaluation takes).
__device__ __forceinline__ double leg_reference(double cx, double cy, double cz, double hx, double hy,
                                                const GeomParams& g, LegRef& r, float* qc2i = nullptr)
{
    // explicit roundings (no contraction), so that every kernel computes the same reference
    const double ex = __dadd_rn(cx, -hx), ey = __dadd_rn(cy, -hy);
    const double Rc2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(cz, cz));
    const double qc = __ddiv_rn(__dmul_rn(g.a, Rc2), __dadd_rn(g.v0, __dmul_rn(g.k, cz)));
    const double wc = __dsqrt_rn(__dmul_rn(qc, __dadd_rn(qc, 2.0)));
    const double uc = __dadd_rn(__dadd_rn(1.0, qc), wc);
    r.Rc2 = (float)Rc2;
    r.qc = (float)qc;
    r.wc = (float)wc;
    r.iuc = (float)__drcp_rn(uc);
    if (qc2i) *qc2i = (float)__ddiv_rn(__dadd_rn(qc, 2.0), uc);
    return log1p(__dadd_rn(qc, wc));
}

// Per-z constants of the linear path, premultiplied by alpha(z):
// (alpha, alpha kappa, alpha (z^2 - z_c^2), alpha z^2), and gamma(z) for the weight.
__device__ __forceinline__ float4 z_constants_m(double z, double zc, const GeomParams& g, float& gamma)
{
    // explicit roundings (no contraction), so that every kernel computes the same constants
    const double vz = __dadd_rn(g.v0, __dmul_rn(g.k, z));
    const double alpha = __ddiv_rn(g.a, vz);
    const double kappa = __ddiv_rn(__dmul_rn(-g.k, __dadd_rn(z, -zc)), __dadd_rn(g.v0, __dmul_rn(g.k, zc)));
    gamma = (g.weight == 1 && fabs(z) >= 1e-6 * fabs(g.dz))
                ? (float)__dmul_rn(__dmul_rn(z, g.wscale), __dsqrt_rn(__ddiv_rn(vz, g.a)))
                : 0.f;
    return make_float4((float)alpha, (float)__dmul_rn(alpha, kappa),
                       (float)__dmul_rn(__dmul_rn(alpha, __dadd_rn(z, -zc)), __dadd_rn(z, zc)),
                       (float)__dmul_rn(__dmul_rn(alpha, z), z));
}

// base + C1 ln(1 + rho) for one leg from the per-leg fit (lgc = C1-scaled coefficients):
// Horner in rho itself for NT <= LG_MONO, in t = rho lg_s + lg_o for the longer fits, then
// rho (C1 + rho C1 Q) + base.  The rounding of C1 + rho C1 Q (half an ulp of C1, times |rho|) is
// that of ln(1 + rho) itself scaled by C1; the FP32 rounding error C1lo of C1 is of the same
// size and is left out.
template <int NT>
__device__ __forceinline__ float leg_log(float rho, const GeomParams& g, float base)
{
    const float x = (NT <= LG_MONO) ? rho : fmaf(rho, g.lg_s, g.lg_o);
    float p = g.lgc[NT - 1];
#pragma unroll
    for (int i = NT - 2; i >= 1; --i) p = fmaf(p, x, g.lgc[i]);
    return fmaf(rho, fmaf(rho, p, g.C1), base);
}

// One leg of the linear path: returns rho_leg = u/u_c - 1 and sqrt(q) (for the weight), from
// the per-z constants zk = (alpha, alpha kappa, alpha (z^2 - z_c^2), alpha z^2) and the
// per-trace reference rm = (R_c^2, (q_c + 2)/u_c, w_c, 1/u_c).  q itself is evaluated directly,
// so that it keeps its relative precision as R -> 0, where w = sqrt(q (q + 2)) has an
// infinite slope; q - q_c comes from the cancellation-free form and only scales the result:
//     q - q_c = alpha dP + alpha kappa R_c^2 + alpha (z^2 - z_c^2),   q = alpha dh^2 + alpha z^2,
//     u/u_c - 1 = (q - q_c) (q/u_c + (q_c + 2)/u_c) / (w + w_c) + (q - q_c)/u_c.
template <int WGT, bool FAST>
__device__ __forceinline__ float leg_delta_m(float dP, float dh2, const float4& zk, const float4& rm, float& sq)
{
    const float dq = fmaf(zk.x, dP, fmaf(zk.y, rm.x, zk.z));
    const float q = fmaf(zk.x, dh2, zk.w);
    float w;
    if constexpr (WGT == 1) {
        sq = hsqrt<FAST>(q);
        w = sq * hsqrt<FAST>(q + 2.f);
    } else {
        sq = 0.f;
        w = hsqrt<FAST>(q * (q + 2.f));
    }
    const float gi = fmaf(fmaf(q, rm.w, rm.y), hrcp<FAST>(w + rm.z), rm.w);
    return dq * gi;
}

// Smallest and largest one-way time from a surface point at horizontal distance [hmin, hmax]
// from the tile footprint to any depth in [zlo, zhi].  T grows with h at fixed z; at fixed h,
// q(z) = (h^2 + z^2)/(v0 (v0 + k z)) has its only interior stationary point (a minimum) at
// z* = k h^2 / (v0 + sqrt(v0^2 + k^2 h^2)).
__device__ __forceinline__ void leg_bounds(float hmin, float hmax, float zlo, float zhi, int vel,
                                           float v0, float k, float& tmin, float& tmax)
{
    const float kk = (vel == VK_CONST) ? 0.f : k;
    const float kh2 = __fmul_rn(__fmul_rn(kk, hmin), hmin);
    float zs = __fdiv_rn(kh2, __fadd_rn(v0, __fsqrt_rn(__fadd_rn(__fmul_rn(v0, v0), __fmul_rn(kk, kh2)))));
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
    dmin = __fsqrt_rn(__fadd_rn(__fmul_rn(ax, ax), __fmul_rn(ay, ay)));
    const float bx = fmaxf(fabsf(px - xlo), fabsf(px - xhi));
    const float by = fmaxf(fabsf(py - ylo), fabsf(py - yhi));
    dmax = __fsqrt_rn(__fadd_rn(__fmul_rn(bx, bx), __fmul_rn(by, by)));
}

struct TileBox {
    float xlo, xhi, ylo, yhi, zlo, zhi;   // FP32 box of the valid samples (window bounds)
    double cx, cy, cz;                    // FP64 centre (linear-path reference point)
};

// Time-migration constants of a tile: 1 / largest and 1 / smallest v_rms over its times (v_rms is
// monotone in t0, so its extremes are at the ends), and at the centre time t0_c the equivalent
// depth squared ze_c^2 and C1(t0_c) = 1 / (v_rms(t0_c) dt).  Only the time-migration kernels
// compute them, so no other kernel carries them in registers.
struct PstmTile {
    float ivlo, ivhi;
    double pze2, pc1;
};

// leg_delta_m plus q/w = sqrt(q / (q + 2)) for the velocity derivatives; sq = sqrt(q) always.
// With fast math, one approximate 1/sqrt(q + 2) serves both w = sqrt(q) (q + 2)/sqrt(q + 2)
// and q/w = sqrt(q)/sqrt(q + 2).
template <bool FAST>
__device__ __forceinline__ float leg_delta_grad_m(float dP, float dh2, const float4& zk, const float4& rm,
                                                  float& sq, float& qw)
{
    const float dq = fmaf(zk.x, dP, fmaf(zk.y, rm.x, zk.z));
    const float q = fmaf(zk.x, dh2, zk.w);
    sq = hsqrt<FAST>(q);
    const float q2 = q + 2.f;
    const float ri = hrsqrt<FAST>(q2);
    const float w = sq * (q2 * ri);
    qw = sq * ri;
    const float gi = fmaf(fmaf(q, rm.w, rm.y), hrcp<FAST>(w + rm.z), rm.w);
    return dq * gi;
}

// Sample window [lo, hi] of a trace whose two-way time lies in [tsum_lo, tsum_hi] over the tile
// (seconds; FP32), widened by 2 samples plus a relative 2e-4 and g.tslack and clipped to
// [0, nt - 1]; *clipped reports a clip.  False when the window misses the trace.
__device__ __forceinline__ bool sample_window(float tsum_lo, float tsum_hi, const GeomParams& g, int& lo, int& hi,
                                              bool* clipped)
{
    const float inv_dt = __fdiv_rn(1.f, g.dt);
    const float tlo = __fmul_rn(__fsub_rn(tsum_lo, g.t0), inv_dt);
    const float thi = __fmul_rn(__fsub_rn(tsum_hi, g.t0), inv_dt);
    const float slo = __fadd_rn(__fadd_rn(2.f, __fmul_rn(2e-4f, fabsf(tlo))), g.tslack);
    const float shi = __fadd_rn(__fadd_rn(2.f, __fmul_rn(2e-4f, fabsf(thi))), g.tslack);
    const float flo = floorf(tlo - slo), fhi = ceilf(thi + shi) + 1.f;
    if (!(fhi >= 1.f && flo <= (float)(g.nt - 2))) return false;   // also NaN
    lo = flo < 0.f ? 0 : (int)flo;
    hi = fhi > (float)(g.nt - 1) ? g.nt - 1 : (int)fhi;
    if (clipped) *clipped = flo < 0.f || fhi > (float)(g.nt - 1);
    return hi > lo;
}

// Sample window [lo, hi] of one trace over a tile box, from the time bounds of both legs with
// a slack of 2 + 2e-4 |tau| samples for FP32 rounding; false if no valid sample can reach the box.
__device__ __forceinline__ bool trace_window(const float4& h, const TileBox& box, int vel,
                                             const GeomParams& g, int& lo, int& hi, bool* clipped = nullptr,
                                             const PstmTile* pt = nullptr)
{
    const float v0 = (float)g.v0, kf = (float)g.k;
    float hs0, hs1, hr0, hr1, ts0, ts1, tr0, tr1;
    rect_dist(h.x, h.y, box.xlo, box.xhi, box.ylo, box.yhi, hs0, hs1);
    rect_dist(h.z, h.w, box.xlo, box.xhi, box.ylo, box.yhi, hr0, hr1);
    if (vel == VK_PSTM) {
        // time migration, T = sqrt((t0/2)^2 + h^2 / v_rms(t0)^2) over t0 in [zlo, zhi] (t0 >= 0):
        // each term is bounded on its own, v_rms being monotone in t0
        const float ulo = __fmul_rn(0.5f, box.zlo), uhi = __fmul_rn(0.5f, box.zhi);
        const float qlo = __fmul_rn(ulo, ulo), qhi = __fmul_rn(uhi, uhi);
        auto leg = [](float q, float hh, float iv) {
            const float e = __fmul_rn(hh, iv);
            return __fsqrt_rn(__fadd_rn(q, __fmul_rn(e, e)));
        };
        ts0 = leg(qlo, hs0, pt->ivlo);
        ts1 = leg(qhi, hs1, pt->ivhi);
        tr0 = leg(qlo, hr0, pt->ivlo);
        tr1 = leg(qhi, hr1, pt->ivhi);
    } else {
        leg_bounds(hs0, hs1, box.zlo, box.zhi, vel, v0, kf, ts0, ts1);
        leg_bounds(hr0, hr1, box.zlo, box.zhi, vel, v0, kf, tr0, tr1);
    }
    return sample_window(__fadd_rn(ts0, tr0), __fadd_rn(ts1, tr1), g, lo, hi, clipped);
}

// Tile box (FP32, for the window bounds) and FP64 centre (reference point) of the tile
// starting at (x0, y0, z0) with ext_x x ext_y columns and ext_z depth samples.
__device__ __forceinline__ TileBox tile_box(const GeomParams& g, int x0, int y0, int z0, int ext_x,
                                            int ext_y, int ext_z)
{
    const int xe = min(x0 + ext_x, g.nx) - 1, ye = min(y0 + ext_y, g.ny) - 1;
    const int ze = min(z0 + ext_z, g.nz) - 1;
    TileBox box;
    const float xa = col_coord(g.ox, x0, g.dx), xb = col_coord(g.ox, xe, g.dx);
    const float ya = g.dim == 3 ? col_coord(g.oy, y0, g.dy) : 0.f;
    const float yb = g.dim == 3 ? col_coord(g.oy, ye, g.dy) : 0.f;
    const float za = (float)(g.oz + z0 * g.dz), zb = (float)(g.oz + ze * g.dz);
    box.xlo = fminf(xa, xb);
    box.xhi = fmaxf(xa, xb);
    box.ylo = fminf(ya, yb);
    box.yhi = fmaxf(ya, yb);
    box.zlo = fminf(za, zb);
    box.zhi = fmaxf(za, zb);
    box.cx = __dadd_rn(g.ox, __dmul_rn(0.5 * (x0 + xe), g.dx));
    box.cy = g.dim == 3 ? __dadd_rn(g.oy, __dmul_rn(0.5 * (y0 + ye), g.dy)) : 0.0;
    box.cz = __dadd_rn(g.oz, __dmul_rn(0.5 * (z0 + ze), g.dz));
    return box;
}

__device__ __forceinline__ PstmTile pstm_tile(const GeomParams& g, const TileBox& box)
{
    PstmTile t;
    const double vc = sqrt(vrms2_of(g.v0, g.pk, box.cz));
    const double zec = 0.5 * vc * box.cz;
    t.pze2 = zec * zec;
    t.pc1 = 1.0 / (vc * g.dtd);
    const double va = sqrt(vrms2_of(g.v0, g.pk, box.zlo)), vb = sqrt(vrms2_of(g.v0, g.pk, box.zhi));
    t.ivlo = (float)(1.0 / fmax(va, vb)) * (1.f - 1e-6f);
    t.ivhi = (float)(1.0 / fmin(va, vb)) * (1.f + 1e-6f);
    return t;
}

}  // namespace kh
