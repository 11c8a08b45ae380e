// The two-way time tau = (T_s + T_r - t0)/dt of one (image point, trace) pair, as the
// migration, demigration and gradient kernels evaluate it.
//
// Constant velocity: tau from R_s + R_r directly (two square roots).
//
// Linear v(z) = v0 + k z: T = arccosh(1 + q)/|k|, q = k^2 R^2 / (2 v0 (v0 + k z)), so
// e^{|k| T} = u = 1 + q + w with w = sqrt(q (q + 2)).  Evaluated directly in FP32 this
// loses ~1e-7 of T (about 3e-5 samples at T ~ 1 s), too much for 1e-5 image parity.
// Instead every (tile, trace) pair gets an FP64 reference at the tile centre c (computed
// once by the staging warp), and each point evaluates only the change relative to it in
// cancellation-free form:
//     q - q_c = alpha(z) (dP + kappa(z) R_c^2 + (z^2 - z_c^2)),   dP = |x_h - s_h|^2 - |c_h - s_h|^2
//             = alpha(z) ((x_h - c_h).(x_h + c_h - 2 s_h) + ...),  kappa(z) = -k (z - z_c)/(v0 + k z_c)
//     w - w_c = (q - q_c)(q + q_c + 2)/(w + w_c)
//     u/u_c - 1 = (q - q_c)(1 + (q + q_c + 2)/(w + w_c)) / u_c
//     tau - tau_c = ln((u_s/u_sc)(u_r/u_rc)) / (|k| dt),
// with ln(1 + rho) from a polynomial fitted on the host for the tile's |rho| bound.
#pragma once

#include "kh_device.cuh"

namespace kh {

// Per-(tile, trace) data of one leg, FP32 copies of FP64 values.
struct LegRef {
    float Rc2;   // |c - x_a|^2
    float qc;    // q at the tile centre
    float wc;    // sqrt(q_c (q_c + 2))
    float iuc;   // 1 / u_c
};

// FP64 reference of one leg: returns ln u_c and fills the FP32 copies.
__device__ __forceinline__ double leg_reference(double cx, double cy, double cz, double hx, double hy,
                                                const GeomParams& g, LegRef& r)
{
    const double ex = cx - hx, ey = cy - hy;
    const double Rc2 = ex * ex + ey * ey + cz * cz;
    const double qc = g.a * Rc2 / (g.v0 + g.k * cz);
    const double wc = sqrt(qc * (qc + 2.0));
    r.Rc2 = (float)Rc2;
    r.qc = (float)qc;
    r.wc = (float)wc;
    r.iuc = (float)(1.0 / (1.0 + qc + wc));
    return log1p(qc + wc);
}

// Per-z constants of the linear path for depth z and tile-centre depth zc.
struct ZConst {
    float alpha, kappa, dz2, gamma;
};

__device__ __forceinline__ ZConst z_constants(double z, double zc, const GeomParams& g)
{
    ZConst c;
    const double vz = g.v0 + g.k * z;
    c.alpha = (float)(g.a / vz);
    c.kappa = (float)(-g.k * (z - zc) / (g.v0 + g.k * zc));
    c.dz2 = (float)((z - zc) * (z + zc));
    // W = z (R_s + R_r) / (2 r0^2) with R = sqrt(q) sqrt(vz / a)
    c.gamma = (g.weight == 1 && fabs(z) >= 1e-6 * fabs(g.dz)) ? (float)(z * g.wscale * sqrt(vz / g.a)) : 0.f;
    return c;
}

// ln(1 + rho) = rho (1 + rho Q), Q a polynomial in t = (rho - m)/h fitted on the tile's rho
// interval [m - h, m + h] (coefficients g.lp[1..NT-1]).
template <int NT>
__device__ __forceinline__ float log1p_poly(float rho, const GeomParams& g)
{
    const float t = fmaf(rho, g.lp_s, g.lp_o);
    float p = g.lp[NT - 1];
#pragma unroll
    for (int i = NT - 2; i >= 1; --i) p = fmaf(p, t, g.lp[i]);
    return fmaf(rho, rho * p, rho);
}

// One leg of the linear path: returns rho_leg = u/u_c - 1 and sqrt(q) (for the weight).
template <int WGT, bool FAST>
__device__ __forceinline__ float leg_delta(float dP, const ZConst& zc, const LegRef& r, float qc2,
                                           float& sq)
{
    const float E = fmaf(zc.kappa, r.Rc2, zc.dz2);
    const float dq = zc.alpha * (dP + E);
    const float q = fmaxf(r.qc + dq, 0.f);   // q >= 0; rounding can leave -1 ulp at R = 0
    float w;
    if constexpr (WGT == 1) {
        sq = hsqrt<FAST>(q);
        w = sq * hsqrt<FAST>(q + 2.f);
    } else {
        sq = 0.f;
        w = hsqrt<FAST>(q * (q + 2.f));
    }
    const float gq = fmaf(q + qc2, hrcp<FAST>(w + r.wc), 1.f);
    return (dq * r.iuc) * gq;
}

}  // namespace kh
