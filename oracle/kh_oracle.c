/*
 * FP64 CPU oracle for Kirchhoff prestack migration (Eq. 1 of "Distributed computing
 * of Seismic Imaging Algorithms", Sec. 3).  TEST INFRASTRUCTURE ONLY: it is called
 * by the tests, by smoke() and by the bench's CPU-baseline leg, never by the product
 * path.  It shares no code, header or constant with the CUDA library.
 *
 * It evaluates the definitions by brute force over every (image point, trace) pair,
 * in double precision, with no blocking or reordering:
 *
 *   I(x, X) = sum_traces W(x, x_s, x_r) * delta(X - |x_s - x_r|) * D(x_s, x_r, T(x,x_s) + T(x,x_r))
 *                                                                          (Sec. 3, Eq. 1)
 *
 * The delta selects one offset bin per trace; D is read at t = T_s + T_r by linear
 * interpolation; the traces near enough to an image point to carry its reflections (Sec. 3,
 * after Eq. 2) are those within a hard aperture on the horizontal distance from the image
 * column to the trace midpoint.  The paper names T and W (the propagation times and amplitude
 * in the model, Sec. 3) but gives no formula for either; the readings taken are:
 *   T, constant v:      R / v0,  R = |x - x_a| (sources/receivers at z = 0, Sec. 2)
 *   T, v(z) = v0 + k z:  T = (2/k) asinh(s),  s = k R / (2 sqrt(v0 (v0 + k z))),
 *                        the closed form of the circular-ray traveltime, written as
 *                        T = (R/g) h(s) with g = sqrt(v0 vz), h(s) = asinh(s)/s (series near 0)
 *   W = 1, or W = 1/2 (cos th_s + cos th_r) R_s R_r / R0^2 with cos th = z / R
 *                        (chord obliquity times spreading), W := 0 where |z| < 1e-6 |dz|.
 * Decisions that turn floating point into a discrete choice are taken in the same
 * precision as the GPU library: the offset bin in FP64, the aperture test in FP32
 * with a fixed operation order (no contraction; compile with -ffp-contract=off).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int dim;                 /* 2 or 3 */
    int nx, ny, nz;
    double ox, oy, oz, dx, dy, dz;
    int n_bins;
    double bin_width;
    int vel;                 /* 0 constant, 1 linear in z, 2 table of the linear model, 3 time
                                migration (double square root, RMS velocity of the linear model),
                                4 tables of a gridded model v(x, z) from the eikonal solver */
    double v0, k;
    int weight;              /* 0 W=1, 1 obliquity x spreading, 2 true amplitude (constant v) */
    double r0;
    double aperture;         /* <= 0: full aperture */
    int nt;
    double t0, dt;
    double table_spacing;    /* vel 2: node spacing of the radial traveltime table */
    double taper;            /* fraction of the aperture over which the weight tapers to 0 */
    /* vel 4: one first-arrival traveltime table per surface location, on the node grid
     * (gox + i gh, j gh), i < gnx, j < gnz (2D only) */
    const double* gtab;      /* [gnloc][gnx][gnz], z fastest */
    const float* gloc;       /* [gnloc] x of each table's surface point, increasing */
    int gnloc, gnx, gnz;
    double gox, gh;
    double aa_spacing;       /* vel 0, 1: trace spacing (m) of the operator anti-aliasing; <= 0: off */
} ko_desc;

/* Deliberate-mistake switch used only by the tests that show the pins catch errors.
 * 0 = the oracle as written. */
static int ko_mutation = 0;
void ko_set_mutation(int m) { ko_mutation = m; }

void ko_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int ko_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- traveltime and its derivatives (Sec. 3: T, the propagation time in the model) ---- */

/* asinh(s)/s and its derivative; Taylor series of asinh for small |s|. */
static void asinh_over_s(double s, double* h, double* hp)
{
    if (fabs(s) < 1e-2) {
        double s2 = s * s;
        *h = 1.0 - s2 / 6.0 + 3.0 * s2 * s2 / 40.0 - 5.0 * s2 * s2 * s2 / 112.0
             + 35.0 * s2 * s2 * s2 * s2 / 1152.0;
        *hp = s * (-1.0 / 3.0 + 3.0 * s2 / 10.0 - 15.0 * s2 * s2 / 56.0
                   + 35.0 * s2 * s2 * s2 / 144.0);
    } else {
        *h = asinh(s) / s;
        *hp = (1.0 / sqrt(1.0 + s * s) - *h) / s;
    }
}

/* Prestack time migration (vel 3): the image's vertical axis is the two-way vertical time t0 (its
 * "z" coordinates are seconds), and each leg takes the double-square-root time of a straight ray
 * through a medium of the RMS velocity of v(z) = v0 + k z down to the one-way vertical time t0/2:
 *     T_a = sqrt((t0/2)^2 + h_a^2 / v_rms(t0)^2),   h_a the horizontal distance,
 *     v_rms(t0)^2 = (2/t0) integral_0^{t0/2} v(tau)^2 dtau = v0^2 (e^{k t0} - 1) / (k t0),
 * since dz/dtau = v gives v(tau) = v0 e^{k tau} at one-way vertical time tau. */
static double vrms2(const ko_desc* d, double t0)
{
    const double x = d->k * t0;
    if (ko_mutation == 11) {   /* the interval velocity at t0/2 instead of the RMS velocity */
        const double v = d->v0 * exp(0.5 * x);
        return v * v;
    }
    if (fabs(x) < 1e-6) return d->v0 * d->v0 * (1.0 + x / 2.0 + x * x / 6.0);
    return d->v0 * d->v0 * expm1(x) / x;
}

static double dsr_leg(const ko_desc* d, double h, double t0)
{
    const double half = (ko_mutation == 12) ? t0 : 0.5 * t0;
    return sqrt(half * half + h * h / vrms2(d, t0));
}

/* One-way time from a surface point (z = 0) to a point at distance R and depth z (vel 3: R is
 * the horizontal distance and z the two-way vertical time). */
static void traveltime(const ko_desc* d, double R, double z, double* T, double* dTdv0, double* dTdk)
{
    if (d->vel == 3) {
        *T = dsr_leg(d, R, z);
        if (dTdv0) *dTdv0 = 0.0;
        if (dTdk) *dTdk = 0.0;
        return;
    }
    if (d->vel == 0) {
        *T = R / d->v0;
        if (dTdv0) *dTdv0 = -R / (d->v0 * d->v0);
        if (dTdk) *dTdk = 0.0;
        return;
    }
    double v0 = d->v0, k = d->k;
    double vz = v0 + k * z;
    double g = sqrt(v0 * vz);
    double s = k * R / (2.0 * g);
    double h, hp;
    asinh_over_s(s, &h, &hp);
    *T = R / g * h;
    if (dTdv0 || dTdk) {
        /* g^2 = v0 vz: dg/dv0 = (vz + v0)/(2g), dg/dk = v0 z/(2g);
         * s = k R/(2g): ds/dth = (R/2) (dk/dth g - k dg/dth) / g^2 */
        double dg_dv0 = (vz + v0) / (2.0 * g);
        double dg_dk = v0 * z / (2.0 * g);
        double ds_dv0 = 0.5 * R * (-k * dg_dv0) / (g * g);
        double ds_dk = 0.5 * R * (g - k * dg_dk) / (g * g);
        double a = -R / (g * g) * h, b = R / g * hp;
        if (ko_mutation == 5) b = -b;
        if (dTdv0) *dTdv0 = a * dg_dv0 + b * ds_dv0;
        if (dTdk) *dTdk = a * dg_dk + b * ds_dk;
    }
}

/* Table traveltime (vel 2): the model v(z) = v0 + k z depends on depth only, so the time
 * from a surface point to (h, z) (h = horizontal distance) is one function T(h, z).  It is
 * tabulated with the closed form at nodes h_i = i D (D = table_spacing) and, in depth, on
 * image depths: z_j = z_min + j D_z with z_min the shallowest image depth and D_z = m |dz|,
 * m the largest power of two not above min(4, D / |dz|) (at least 1), so the depth spacing
 * never exceeds D; it is read by bilinear interpolation in (h, z). */
static double table_dz(const ko_desc* d)
{
    const double r = d->table_spacing / fabs(d->dz);
    double m = 1.0;
    while (m < 4.0 && 2.0 * m <= r) m *= 2.0;
    return m * fabs(d->dz);
}

static double table_node(const ko_desc* d, double h, double z)
{
    ko_desc m = *d;
    m.vel = (d->k == 0.0) ? 0 : 1;
    double T;
    traveltime(&m, sqrt(h * h + z * z), z, &T, NULL, NULL);
    return T;
}

static double table_traveltime(const ko_desc* d, double h, double z)
{
    const double D = d->table_spacing, Dz = table_dz(d);
    const double za = (d->dz >= 0) ? d->oz : d->oz + (d->nz - 1) * d->dz;
    const double uh = h / D, uz = (z - za) / Dz;
    const double ih = floor(uh), jz = floor(uz);
    const double fh = uh - ih, fz = uz - jz;
    const double h0 = ih * D, h1 = (ih + 1.0) * D, z0 = za + jz * Dz, z1 = za + (jz + 1.0) * Dz;
    const double a = (1.0 - fz) * table_node(d, h0, z0) + fz * table_node(d, h0, z1);
    const double b = (1.0 - fz) * table_node(d, h1, z0) + fz * table_node(d, h1, z1);
    return (1.0 - fh) * a + fh * b;
}

int ko_traveltime(const ko_desc* d, long n, const double* R, const double* z, double* T,
                  double* dTdv0, double* dTdk)
{
    for (long i = 0; i < n; ++i)
        traveltime(d, R[i], z[i], &T[i], dTdv0 ? &dTdv0[i] : NULL, dTdk ? &dTdk[i] : NULL);
    return 0;
}

/* ---- first-arrival traveltimes in a laterally varying model v(x, z) (vel 4) ----
 *
 * Sec. 3 takes T from the high-frequency limit of ray theory, one path per source and image
 * point: the first-arrival time, the viscosity solution of the eikonal equation |grad T| = s
 * (slowness s = 1/v) with T = 0 at the surface point x_s.  It is computed on a node grid
 * (ox + i h, j h), i < nx, j < nz (row 0 is the surface), as follows.
 *
 * Factorisation (additive, Luo & Qian, J. Sci. Comput. 52, 2012): T = T0 + tau with
 * T0 = s0 |x - x_s|, the exact time of the constant slowness s0 = s(x_s), removes the point-source
 * singularity that costs a plain first-order scheme its accuracy; tau solves
 * |grad T0 + grad tau| = s.
 * Discretisation: the Godunov upwind scheme on tau.  Along x, the one-sided slopes
 * grad_x T0 + (tau - tau_left)/h and grad_x T0 + (tau_right - tau)/h enter as
 * max(tau - c_x, 0)^2 / h^2 with c_x = min(tau_left - h g_x, tau_right + h g_x), g = grad T0 at the
 * node (likewise c_z along z), so the node equation
 *     max(tau - c_x, 0)^2 + max(tau - c_z, 0)^2 = (h s)^2
 * is the plain upwind equation with shifted neighbour values, solved in closed form:
 *     tau = min(c_x, c_z) + h s                                   if |c_x - c_z| >= h s,
 *     tau = (c_x + c_z + sqrt(2 (h s)^2 - (c_x - c_z)^2)) / 2     otherwise.
 * Solution: fast sweeping (Zhao, Math. Comp. 74, 2005): Gauss-Seidel passes over the grid in the
 * orderings (i up, j up), (i down, j up), (i down, j down), (i up, j down), each node taking the
 * smaller of its value and the update; rounds of four passes repeat until the largest decrease of
 * a round is at most `tol` (seconds; 0: until nothing changes).
 * Source treatment (a reading): the nodes with |x_i - x_s| <= 2 h in the first three rows keep
 * the straight-ray time |x - x_s| (s0 + s(x)) / 2 (trapezoid rule for the slowness along the
 * segment; s0 linear along the surface row) and are not updated.
 * Every operation is one IEEE double operation in the order written (s = 1 / v). */
static double godunov(double a, double b, double fh)
{
    const double d = a - b;
    if (fabs(d) >= fh) return fmin(a, b) + fh;
    const double disc = 2.0 * (fh * fh) - d * d;
    if (ko_mutation == 16) return 0.5 * ((a + b) - sqrt(disc));   /* wrong root */
    return 0.5 * ((a + b) + sqrt(disc));
}

/* T[nx][nz] (z fastest) from the surface point (xs, 0); v [nx][nz] in m/s.  Returns the number of
 * rounds, or -1 if max_rounds did not suffice. */
int ko_eikonal(int nx, int nz, double ox, double h, const float* v, double xs, int max_rounds, double tol,
               double* T)
{
    if (nx < 2 || nz < 2 || !(h > 0.0)) return -1;
    const long n = (long)nx * nz;
    double* s = (double*)malloc(sizeof(double) * (size_t)n);
    double* tau = (double*)malloc(sizeof(double) * (size_t)n);
    unsigned char* fixed = (unsigned char*)calloc((size_t)n, 1);
    if (!s || !tau || !fixed) { free(s); free(tau); free(fixed); return -1; }
    for (long q = 0; q < n; ++q) s[q] = 1.0 / (double)v[q];
    const double u = (xs - ox) / h;
    long i0 = (long)floor(u);
    if (i0 < 0) i0 = 0;
    if (i0 > nx - 2) i0 = nx - 2;
    const double f = u - (double)i0;
    const double s0 = s[i0 * nz] + f * (s[(i0 + 1) * nz] - s[i0 * nz]);
    for (long i = 0; i < nx; ++i) {
        const double dx = (ox + (double)i * h) - xs;
        const int near = fabs(dx) <= 2.0 * h;
        for (long j = 0; j < nz; ++j) {
            const long q = i * nz + j;
            tau[q] = INFINITY;
            if (near && j <= 2) {
                const double zj = (double)j * h;
                const double dist = sqrt(dx * dx + zj * zj);
                /* T = s0 dist + tau = dist (s0 + s) / 2 */
                tau[q] = (ko_mutation == 17) ? dist * (s[q] - s0) : dist * (0.5 * (s[q] - s0));
                fixed[q] = 1;
            }
        }
    }
    const double hs0 = h * s0;
    int rounds = -1;
    for (int r = 0; r < max_rounds; ++r) {
        double most = 0.0;
        for (int pass = 0; pass < 4; ++pass) {
            const int iup = (pass == 0 || pass == 3), jup = (pass < 2);
            for (long ii = 0; ii < nx; ++ii) {
                const long i = iup ? ii : nx - 1 - ii;
                const double dx = (ox + (double)i * h) - xs;
                for (long jj = 0; jj < nz; ++jj) {
                    const long j = jup ? jj : nz - 1 - jj;
                    const long q = i * nz + j;
                    if (fixed[q]) continue;
                    const double zj = (double)j * h;
                    const double g = hs0 / sqrt(dx * dx + zj * zj);   /* h |grad T0| / |x - x_s| */
                    double gx = g * dx, gz = g * zj;                   /* h grad T0 */
                    if (ko_mutation == 19) { gx = -gx; gz = -gz; }   /* shifts of the wrong sign */
                    const double cl = (i > 0) ? tau[q - nz] - gx : INFINITY;
                    const double cr = (i < nx - 1) ? tau[q + nz] + gx : INFINITY;
                    const double cu = (j > 0) ? tau[q - 1] - gz : INFINITY;
                    const double cd = (j < nz - 1) ? tau[q + 1] + gz : INFINITY;
                    const double a = fmin(cl, cr), b = fmin(cu, cd);
                    if (a == INFINITY && b == INFINITY) continue;
                    const double t = godunov(a, b, h * s[q]);
                    if (t < tau[q]) {
                        const double dec = tau[q] - t;
                        if (dec > most) most = dec;
                        tau[q] = t;
                    }
                }
            }
        }
        if (most <= tol || ko_mutation == 18) {   /* 18: stop after one round */
            rounds = r + 1;
            break;
        }
    }
    for (long i = 0; i < nx; ++i) {
        const double dx = (ox + (double)i * h) - xs;
        for (long j = 0; j < nz; ++j) {
            const double zj = (double)j * h;
            T[i * nz + j] = s0 * sqrt(dx * dx + zj * zj) + tau[i * nz + j];
        }
    }
    free(s);
    free(tau);
    free(fixed);
    return rounds;
}

/* Tables for nloc surface points (OpenMP over the points); rounds[l] as ko_eikonal returns it. */
int ko_grid_tables(int nx, int nz, double ox, double h, const float* v, int nloc, const float* loc,
                   int max_rounds, double tol, double* T, int* rounds)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
    for (int l = 0; l < nloc; ++l) {
        rounds[l] = ko_eikonal(nx, nz, ox, h, v, (double)loc[l], max_rounds, tol, T + (long)l * nx * nz);
        bad += rounds[l] < 0;
    }
    return bad;
}

/* Index of the table whose surface point is exactly x (the trace's source or receiver), or -1. */
static int grid_location(const ko_desc* d, float x)
{
    int lo = 0, hi = d->gnloc - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) / 2;
        if (d->gloc[mid] == x) return mid;
        if (d->gloc[mid] < x) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Table l read at (x, z) by bilinear interpolation between the four surrounding nodes (node
 * indices clamped to the grid, so the last node column or row is reached with fraction 1). */
static double grid_traveltime(const ko_desc* d, int l, double x, double z)
{
    double u = (x - d->gox) / d->gh, w = z / d->gh;
    if (ko_mutation == 14) { const double t = u; u = w; w = t; }   /* axes swapped */
    double iu = floor(u), jw = floor(w);
    if (iu > d->gnx - 2) iu = d->gnx - 2;
    if (iu < 0) iu = 0;
    if (jw > d->gnz - 2) jw = d->gnz - 2;
    if (jw < 0) jw = 0;
    const double fu = u - iu, fw = w - jw;
    const double* t = d->gtab + ((long)l * d->gnx + (long)iu) * d->gnz + (long)jw;
    const double a = (1.0 - fw) * t[0] + fw * t[1];
    const double b = (1.0 - fw) * t[d->gnz] + fw * t[d->gnz + 1];
    return (1.0 - fu) * a + fu * b;
}

int ko_grid_traveltime(const ko_desc* d, int l, long n, const double* x, const double* z, double* T)
{
    for (long i = 0; i < n; ++i) T[i] = grid_traveltime(d, l, x[i], z[i]);
    return 0;
}

/* True-amplitude weight (weight 2, constant velocity; a reading of Sec. 3's weight W, which carries
 * the propagation amplitude): the weight of the asymptotic Kirchhoff inversion
 * for the reflection coefficient (Beylkin 1985; Bleistein 1987), |h| / (a_s a_r |grad tau|^2), with
 * a_a the Green's-function amplitude of each leg and h the Beylkin determinant of
 * tau(x; xi) = (|x - s| + |x - r|) / v over the trace's midpoint xi at fixed offset (s = xi - o,
 * r = xi + o):
 *     3D: h = det[grad tau, d(grad tau)/d xi_1, d(grad tau)/d xi_2],   a = 1 / (4 pi R);
 *     2D: h = det[grad tau, d(grad tau)/d xi] (the (x, z) plane),       a ~ 1 / sqrt(R).
 * With e_a = (x - a) / R_a, grad tau = (e_s + e_r) / v and d e_a / d xi_k = (u_k - e_a (e_a . u_k)) / R_a
 * (u_k the surface direction xi_k moves; the sign of the columns does not change |h|).  The factors
 * of v and the constants of a_a and of the inversion formula are global and are dropped:
 *     W = (R_s R_r)^((dim - 1) / 2) |det[g, D u_1 (, D u_2)]| / |g|^2,
 *     g = e_s + e_r,  D u = sum_a (u - e_a (e_a . u)) / R_a.
 * It applies to time-differentiated data (the inversion's i omega; 3D).  At zero offset it is
 * 2 cos(theta) (3D) and cos(theta) (2D); at the specular point of a horizontal reflector in 3D it is
 * 2 cos(theta), which makes the image peak independent of the offset.  W := 0 where |z| < 1e-6 |dz|,
 * as for weight 1. */
static double ta_weight(const ko_desc* d, double x, double y, double z, double sx, double sy, double rx,
                        double ry)
{
    if (fabs(z) < 1e-6 * fabs(d->dz)) return 0.0;
    const double es[3] = {x - sx, y - sy, z}, er[3] = {x - rx, y - ry, z};
    const double Rs = sqrt(es[0] * es[0] + es[1] * es[1] + es[2] * es[2]);
    const double Rr = sqrt(er[0] * er[0] + er[1] * er[1] + er[2] * er[2]);
    double g[3], c1[3], c2[3];
    for (int i = 0; i < 3; ++i) g[i] = es[i] / Rs + er[i] / Rr;
    /* D u for u = x (c1) and u = y (c2) */
    for (int k = 0; k < 2; ++k) {
        double* c = k == 0 ? c1 : c2;
        const double psu = es[k] / Rs, pru = er[k] / Rr;   /* e_a . u_k */
        for (int i = 0; i < 3; ++i) {
            const double ui = (i == k) ? 1.0 : 0.0;
            c[i] = (ui - es[i] / Rs * psu) / Rs + (ui - er[i] / Rr * pru) / Rr;
        }
    }
    if (ko_mutation == 20) { c1[0] = -c1[0]; }   /* a sign error in one entry */
    double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    if (ko_mutation == 22) g2 = 4.0;   /* the |grad tau|^2 of the reflectivity inversion dropped */
    if (d->dim == 2) {
        /* the (x, z) plane: det[[g_x, c1_x], [g_z, c1_z]] */
        const double h = g[0] * c1[2] - g[2] * c1[0];
        return sqrt(Rs * Rr) * fabs(h) / g2;
    }
    const double h = g[0] * (c1[1] * c2[2] - c1[2] * c2[1]) - c1[0] * (g[1] * c2[2] - g[2] * c2[1]) +
                     c2[0] * (g[1] * c1[2] - g[2] * c1[1]);
    if (ko_mutation == 21) return Rs * Rr * fabs(h) / (Rs + Rr) / g2;   /* a spreading factor off */
    return Rs * Rr * fabs(h) / g2;
}

int ko_ta_weight(const ko_desc* d, long n, const double* p, double* W)
{
    /* p: [n][7] = (x, y, z, sx, sy, rx, ry) */
    for (long i = 0; i < n; ++i)
        W[i] = ta_weight(d, p[7 * i], p[7 * i + 1], p[7 * i + 2], p[7 * i + 3], p[7 * i + 4], p[7 * i + 5], p[7 * i + 6]);
    return 0;
}

/* Operator anti-aliasing (vel 0 or 1, aa_spacing > 0; a reading of the weight W of Eq. 1, which
 * carries the propagation amplitude, that also keeps the sum from aliasing): the operator's time
 * dip across the traces, the midpoint gradient of the two-way time in samples per metre,
 *     p = -(grad_h T_s + grad_h T_r) / dt,
 * times the trace spacing is the moveout L (samples) between adjacent traces,
 *     L = aa_spacing max(|p_x|, |p_y|).
 * A contribution whose moveout exceeds one sample would alias the highest frequencies the sampling
 * carries, so the weight keeps L <= 1 whole, removes L >= 2, and falls between as
 * cos^2(pi (L - 1) / 2) (dip limitation of the operator).
 * The horizontal gradient of one leg's time at the image point, h = (x - a)_h, R = |x - a|:
 *     constant v:   grad_h T = h / (v0 R);
 *     v0 + k z:     T = (2/k) asinh(s), s = k R / (2 g), g = sqrt(v0 (v0 + k z)), and g depends
 *                   on depth only, so grad_h T = (2/k) (k / (2 g)) (h / R) / sqrt(1 + s^2)
 *                   = h / (R g sqrt(1 + s^2)), which tends to h / (v0 R) as k -> 0
 * (0 where R = 0). */
static void aa_leg(const ko_desc* d, double hx, double hy, double z, double* gx, double* gy)
{
    const double R = sqrt(hx * hx + hy * hy + z * z);
    double f = 0.0;
    if (R > 0.0) {
        if (d->vel == 0) {
            f = 1.0 / (d->v0 * R);
        } else {
            const double g = sqrt(d->v0 * (d->v0 + d->k * z));
            const double sv = d->k * R / (2.0 * g);
            f = 1.0 / (R * g * sqrt(1.0 + sv * sv));
        }
    }
    *gx = hx * f;
    *gy = hy * f;
}

static double aa_weight(const ko_desc* d, double x, double y, double z, double sx, double sy, double rx,
                        double ry)
{
    if (d->aa_spacing <= 0.0) return 1.0;
    double gsx, gsy, grx, gry;
    aa_leg(d, x - sx, y - sy, z, &gsx, &gsy);
    aa_leg(d, x - rx, y - ry, z, &grx, &gry);
    double px = (gsx + grx) / d->dt;
    const double py = (gsy + gry) / d->dt;
    if (ko_mutation == 23) px = gsx / d->dt;   /* the receiver leg's dip dropped */
    const double L = d->aa_spacing * fmax(fabs(px), fabs(py));
    if (L <= 1.0) return 1.0;
    if (L >= 2.0) return 0.0;
    const double c = cos(0.5 * 3.14159265358979323846 * (L - 1.0));
    return c * c;
}

int ko_aa_weight(const ko_desc* d, long n, const double* p, double* W)
{
    /* p: [n][7] = (x, y, z, sx, sy, rx, ry) */
    for (long i = 0; i < n; ++i)
        W[i] = aa_weight(d, p[7 * i], p[7 * i + 1], p[7 * i + 2], p[7 * i + 3], p[7 * i + 4], p[7 * i + 5], p[7 * i + 6]);
    return 0;
}

/* Amplitude weight W(x, x_s, x_r) (Sec. 3, Eq. 1). */
static double weight(const ko_desc* d, double z, double Rs, double Rr)
{
    if (d->weight == 0 || ko_mutation == 1) return 1.0;
    if (fabs(z) < 1e-6 * fabs(d->dz)) return 0.0;
    double cs = z / Rs, cr = z / Rr;
    return 0.5 * (cs + cr) * Rs * Rr / (d->r0 * d->r0);
}

/* ---- offset bin (the delta(X - |x_s - x_r|) of Eq. 1), decided in FP64 ---- */
static int offset_bin(const ko_desc* d, float sx, float sy, float rx, float ry)
{
    double ex = (double)sx - (double)rx;
    double ey = (d->dim == 3) ? (double)sy - (double)ry : 0.0;
    double X = sqrt(ex * ex + ey * ey);
    double q = X / d->bin_width;
    double b = floor(q);
    if (ko_mutation == 4) b = floor(q + 0.5);
    if (b < (double)d->n_bins) return (int)b;
    if (X == (double)d->n_bins * d->bin_width) return d->n_bins - 1;
    return -1;
}

int ko_table_traveltime(const ko_desc* d, long n, const double* h, const double* z, double* T)
{
    for (long i = 0; i < n; ++i) T[i] = table_traveltime(d, h[i], z[i]);
    return 0;
}

int ko_bins(const ko_desc* d, long ntr, const float* sx, const float* sy, const float* rx,
            const float* ry, int* bin)
{
    for (long j = 0; j < ntr; ++j)
        bin[j] = offset_bin(d, sx[j], d->dim == 3 ? sy[j] : 0.f, rx[j], d->dim == 3 ? ry[j] : 0.f);
    return 0;
}

/* ---- aperture (the traces near enough to an image point, Sec. 3), decided in FP32 with a fixed order ---- */
static float col_coord(double o, int i, double h) { return (float)(o + (double)i * h); }

static int inside_aperture(const ko_desc* d, float cx, float cy, float sx, float sy, float rx,
                           float ry)
{
    if (d->aperture <= 0.0) return 1;
    float mx = (sx + rx) * 0.5f;
    float my = (sy + ry) * 0.5f;
    if (ko_mutation == 7) { mx = sx; my = sy; }
    if (ko_mutation == 9) { mx = sx + rx; my = sy + ry; }
    float ex = cx - mx;
    float ey = cy - my;
    float ex2 = ex * ex;
    float ey2 = ey * ey;
    float d2 = ex2 + ey2;
    float a2 = (float)(d->aperture * d->aperture);
    if (ko_mutation == 8) return d2 < a2;
    return d2 <= a2;
}

/* Aperture taper: the weight falls from 1 to 0 over the outer fraction f of the aperture as a
 * raised cosine of the horizontal distance d from the column to the trace midpoint:
 *   1 for d <= (1 - f) A,  (1 + cos(pi (d - (1 - f) A) / (f A))) / 2 for (1 - f) A < d <= A.
 * d is taken in FP64 from the FP32 column and midpoint coordinates of the aperture test. */
static double aperture_taper(const ko_desc* d, float cx, float cy, float sx, float sy, float rx, float ry)
{
    if (d->aperture <= 0.0 || d->taper <= 0.0) return 1.0;
    const double mx = (double)((sx + rx) * 0.5f), my = (double)((sy + ry) * 0.5f);
    const double ex = (double)cx - mx, ey = (double)cy - my;
    const double dist = sqrt(ex * ex + ey * ey);
    const double core = (1.0 - d->taper) * d->aperture;
    if (dist <= core) return 1.0;
    double x = (dist - core) / (d->taper * d->aperture);
    if (ko_mutation == 13) x = 1.0 - x;   /* taper reversed */
    return 0.5 * (1.0 + cos(3.14159265358979323846 * x));
}

/* ---- the contribution of one trace to one image point ---- */
typedef struct {
    int valid;      /* 0 <= tau <= nt-1 */
    int i;          /* left sample */
    double f;       /* fraction */
    double W;
    double dtau_dv0, dtau_dk;
} contrib;

static contrib contribution(const ko_desc* d, double x, double y, double z, double sx, double sy,
                            double rx, double ry, int want_grad)
{
    contrib c;
    memset(&c, 0, sizeof c);
    if (ko_mutation == 10 && d->aperture > 0.0) {
        double mx = 0.5 * (sx + rx) - x, my = 0.5 * (sy + ry) - y;
        if (mx * mx + my * my + z * z > d->aperture * d->aperture) return c;
    }
    double Rs = sqrt((x - sx) * (x - sx) + (y - sy) * (y - sy) + z * z);
    double Rr = sqrt((x - rx) * (x - rx) + (y - ry) * (y - ry) + z * z);
    if (ko_mutation == 3) Rr = Rs;
    double Ts, Tr, dsv = 0, dsk = 0, drv = 0, drk = 0;
    double zw = z;   /* the depth of the weight (vel 3: the equivalent depth v_rms t0 / 2) */
    if (d->vel == 3) {
        const double vr = sqrt(vrms2(d, z));
        Ts = dsr_leg(d, sqrt((x - sx) * (x - sx) + (y - sy) * (y - sy)), z);
        Tr = dsr_leg(d, sqrt((x - rx) * (x - rx) + (y - ry) * (y - ry)), z);
        /* straight rays through the RMS medium: R_a = v_rms T_a, depth v_rms t0 / 2 */
        Rs = vr * Ts;
        Rr = vr * Tr;
        zw = vr * 0.5 * z;
        if (fabs(z) < 1e-6 * fabs(d->dz)) zw = 0.0;
    } else if (d->vel == 2) {
        Ts = table_traveltime(d, sqrt((x - sx) * (x - sx) + (y - sy) * (y - sy)), z);
        Tr = table_traveltime(d, sqrt((x - rx) * (x - rx) + (y - ry) * (y - ry)), z);
        if (ko_mutation == 3) Tr = Ts;
    } else if (d->vel == 4) {
        /* each leg from its surface point's table; a point with no table contributes nothing */
        const int ls = grid_location(d, (float)sx), lr = grid_location(d, (float)rx);
        if (ls < 0 || lr < 0) return c;
        Ts = grid_traveltime(d, ls, x, z);
        Tr = grid_traveltime(d, ko_mutation == 15 ? ls : lr, x, z);
    } else {
        traveltime(d, Rs, z, &Ts, want_grad ? &dsv : NULL, want_grad ? &dsk : NULL);
        traveltime(d, Rr, z, &Tr, want_grad ? &drv : NULL, want_grad ? &drk : NULL);
    }
    double tau = (Ts + Tr - d->t0) / d->dt;
    if (ko_mutation == 2) tau = (Ts + Tr + d->t0) / d->dt;
    if (!(tau >= 0.0 && tau <= (double)(d->nt - 1))) return c;
    int i = (int)floor(tau);
    if (i > d->nt - 2) i = d->nt - 2;
    c.valid = 1;
    c.i = i;
    c.f = tau - (double)i;
    if (ko_mutation == 6) c.f = 1.0 - c.f;
    c.W = (d->vel == 3) ? (d->weight == 0 || ko_mutation == 1 ? 1.0
                                                              : (zw == 0.0 ? 0.0
                                                                           : 0.5 * (zw / Rs + zw / Rr) * Rs * Rr /
                                                                                 (d->r0 * d->r0)))
          : (d->weight == 2) ? ta_weight(d, x, y, z, sx, sy, rx, ry)
                             : weight(d, z, Rs, Rr);
    if ((d->vel == 0 || d->vel == 1) && d->aa_spacing > 0.0) c.W *= aa_weight(d, x, y, z, sx, sy, rx, ry);
    if (want_grad) {
        c.dtau_dv0 = (dsv + drv) / d->dt;
        c.dtau_dk = (dsk + drk) / d->dt;
    }
    return c;
}

static inline float hdr(const float* a, long j) { return a ? a[j] : 0.f; }

/* Migration, Eq. 1: image[b][iy][ix][iz] = sum over traces j of bin b in aperture of
 * W * ((1-f) D_j[i] + f D_j[i+1]).  traces: ntr x nt, image: n_bins x ny x nx x nz. */
int ko_migrate(const ko_desc* d, long ntr, const float* sx, const float* sy, const float* rx,
               const float* ry, const double* traces, double* image)
{
    const long ncol = (long)d->nx * d->ny, nz = d->nz, nt = d->nt;
    int* bin = (int*)malloc(sizeof(int) * (ntr > 0 ? ntr : 1));
    if (!bin) return 1;
    ko_bins(d, ntr, sx, sy, rx, ry, bin);
    memset(image, 0, sizeof(double) * (size_t)d->n_bins * ncol * nz);
#pragma omp parallel for schedule(dynamic, 4)
    for (long c = 0; c < ncol; ++c) {
        int iy = (int)(c / d->nx), ix = (int)(c % d->nx);
        double x = d->ox + ix * d->dx, y = (d->dim == 3) ? d->oy + iy * d->dy : 0.0;
        float cx = col_coord(d->ox, ix, d->dx), cy = (d->dim == 3) ? col_coord(d->oy, iy, d->dy) : 0.f;
        for (long j = 0; j < ntr; ++j) {
            if (bin[j] < 0) continue;
            float fsx = sx[j], fsy = hdr(sy, j), frx = rx[j], fry = hdr(ry, j);
            if (d->dim == 2) { fsy = 0.f; fry = 0.f; }
            if (!inside_aperture(d, cx, cy, fsx, fsy, frx, fry)) continue;
            const double tp = aperture_taper(d, cx, cy, fsx, fsy, frx, fry);
            const double* D = traces + j * nt;
            double* out = image + ((long)bin[j] * ncol + c) * nz;
            for (long iz = 0; iz < nz; ++iz) {
                double z = d->oz + iz * d->dz;
                contrib q = contribution(d, x, y, z, fsx, fsy, frx, fry, 0);
                if (!q.valid) continue;
                double val = (1.0 - q.f) * D[q.i] + q.f * D[q.i + 1];
                out[iz] += tp * q.W * val;
            }
        }
    }
    free(bin);
    return 0;
}

/* Migration at a list of image samples (flat indices into the n_bins x ny x nx x nz image). */
int ko_migrate_points(const ko_desc* d, long ntr, const float* sx, const float* sy, const float* rx,
                      const float* ry, const double* traces, long npts, const long* pidx,
                      double* out, long long* ncontrib)
{
    const long ncol = (long)d->nx * d->ny, nz = d->nz, nt = d->nt;
    int* bin = (int*)malloc(sizeof(int) * (ntr > 0 ? ntr : 1));
    if (!bin) return 1;
    ko_bins(d, ntr, sx, sy, rx, ry, bin);
    long long total = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
    for (long p = 0; p < npts; ++p) {
        long q = pidx[p];
        int iz = (int)(q % nz);
        long c = (q / nz) % ncol;
        int b = (int)(q / (nz * ncol));
        int iy = (int)(c / d->nx), ix = (int)(c % d->nx);
        double x = d->ox + ix * d->dx, y = (d->dim == 3) ? d->oy + iy * d->dy : 0.0;
        double z = d->oz + iz * d->dz;
        float cx = col_coord(d->ox, ix, d->dx), cy = (d->dim == 3) ? col_coord(d->oy, iy, d->dy) : 0.f;
        double acc = 0.0;
        for (long j = 0; j < ntr; ++j) {
            if (bin[j] != b) continue;
            float fsx = sx[j], fsy = hdr(sy, j), frx = rx[j], fry = hdr(ry, j);
            if (d->dim == 2) { fsy = 0.f; fry = 0.f; }
            if (!inside_aperture(d, cx, cy, fsx, fsy, frx, fry)) continue;
            ++total;
            contrib w = contribution(d, x, y, z, fsx, fsy, frx, fry, 0);
            if (!w.valid) continue;
            const double* D = traces + j * nt;
            acc += aperture_taper(d, cx, cy, fsx, fsy, frx, fry) * w.W * ((1.0 - w.f) * D[w.i] + w.f * D[w.i + 1]);
        }
        out[p] = acc;
    }
    if (ncontrib) *ncontrib = total;
    free(bin);
    return 0;
}

/* Demigration: the exact transpose of ko_migrate (Sec. 3's sum read from the data side: each
 * image point adds into the trace sample whose time is its source-plus-receiver traveltime).  traces_out[j][i] += W (1-f) m, traces_out[j][i+1] += W f m. */
int ko_demigrate(const ko_desc* d, long ntr, const float* sx, const float* sy, const float* rx,
                 const float* ry, const double* image, double* traces_out)
{
    const long ncol = (long)d->nx * d->ny, nz = d->nz, nt = d->nt;
    int* bin = (int*)malloc(sizeof(int) * (ntr > 0 ? ntr : 1));
    if (!bin) return 1;
    ko_bins(d, ntr, sx, sy, rx, ry, bin);
#pragma omp parallel for schedule(dynamic, 1)
    for (long j = 0; j < ntr; ++j) {
        double* D = traces_out + j * nt;
        memset(D, 0, sizeof(double) * nt);
        if (bin[j] < 0) continue;
        float fsx = sx[j], fsy = hdr(sy, j), frx = rx[j], fry = hdr(ry, j);
        if (d->dim == 2) { fsy = 0.f; fry = 0.f; }
        for (long c = 0; c < ncol; ++c) {
            int iy = (int)(c / d->nx), ix = (int)(c % d->nx);
            float cx = col_coord(d->ox, ix, d->dx), cy = (d->dim == 3) ? col_coord(d->oy, iy, d->dy) : 0.f;
            if (!inside_aperture(d, cx, cy, fsx, fsy, frx, fry)) continue;
            const double tp = aperture_taper(d, cx, cy, fsx, fsy, frx, fry);
            double x = d->ox + ix * d->dx, y = (d->dim == 3) ? d->oy + iy * d->dy : 0.0;
            const double* m = image + ((long)bin[j] * ncol + c) * nz;
            for (long iz = 0; iz < nz; ++iz) {
                double z = d->oz + iz * d->dz;
                contrib q = contribution(d, x, y, z, fsx, fsy, frx, fry, 0);
                if (!q.valid) continue;
                D[q.i] += tp * q.W * (1.0 - q.f) * m[iz];
                D[q.i + 1] += tp * q.W * q.f * m[iz];
            }
        }
    }
    free(bin);
    return 0;
}

/* Gradient of the bilinear form B(m, D) = sum_j sum_x W m[b_j, x] lerp(D_j, tau_j(x))
 * with respect to (v0, k): dB/dth = sum W m (D_j[i+1] - D_j[i]) dtau/dth.  This is
 * the velocity-model derivative that both the migration and the demigration operator
 * need in their backward pass; out[0] = dB/dv0, out[1] = dB/dk. */
int ko_vgrad(const ko_desc* d, long ntr, const float* sx, const float* sy, const float* rx,
             const float* ry, const double* image, const double* traces, double* out,
             double* abs_out)
{
    const long ncol = (long)d->nx * d->ny, nz = d->nz, nt = d->nt;
    int* bin = (int*)malloc(sizeof(int) * (ntr > 0 ? ntr : 1));
    double* part = (double*)calloc((size_t)(ncol > 0 ? ncol : 1) * 4, sizeof(double));
    if (!bin || !part) { free(bin); free(part); return 1; }
    ko_bins(d, ntr, sx, sy, rx, ry, bin);
#pragma omp parallel for schedule(dynamic, 4)
    for (long c = 0; c < ncol; ++c) {
        int iy = (int)(c / d->nx), ix = (int)(c % d->nx);
        double x = d->ox + ix * d->dx, y = (d->dim == 3) ? d->oy + iy * d->dy : 0.0;
        float cx = col_coord(d->ox, ix, d->dx), cy = (d->dim == 3) ? col_coord(d->oy, iy, d->dy) : 0.f;
        double gv = 0.0, gk = 0.0, av = 0.0, ak = 0.0;
        for (long j = 0; j < ntr; ++j) {
            if (bin[j] < 0) continue;
            float fsx = sx[j], fsy = hdr(sy, j), frx = rx[j], fry = hdr(ry, j);
            if (d->dim == 2) { fsy = 0.f; fry = 0.f; }
            if (!inside_aperture(d, cx, cy, fsx, fsy, frx, fry)) continue;
            const double tp = aperture_taper(d, cx, cy, fsx, fsy, frx, fry);
            const double* D = traces + j * nt;
            const double* m = image + ((long)bin[j] * ncol + c) * nz;
            for (long iz = 0; iz < nz; ++iz) {
                double z = d->oz + iz * d->dz;
                contrib q = contribution(d, x, y, z, fsx, fsy, frx, fry, 1);
                if (!q.valid) continue;
                q.W *= tp;
                double slope = D[q.i + 1] - D[q.i];
                gv += q.W * m[iz] * slope * q.dtau_dv0;
                gk += q.W * m[iz] * slope * q.dtau_dk;
                av += fabs(q.W * m[iz] * slope * q.dtau_dv0);
                ak += fabs(q.W * m[iz] * slope * q.dtau_dk);
            }
        }
        part[4 * c] = gv;
        part[4 * c + 1] = gk;
        part[4 * c + 2] = av;
        part[4 * c + 3] = ak;
    }
    out[0] = 0.0;
    out[1] = 0.0;
    double a0 = 0.0, a1 = 0.0;
    for (long c = 0; c < ncol; ++c) {
        out[0] += part[4 * c];
        out[1] += part[4 * c + 1];
        a0 += part[4 * c + 2];
        a1 += part[4 * c + 3];
    }
    if (abs_out) {
        abs_out[0] = a0;
        abs_out[1] = a1;
    }
    free(bin);
    free(part);
    return 0;
}

/* Two-way times source -> point -> receiver for every (point, trace) pair, for the
 * synthesis of test data: out[p * ntr + j] = T(x_p, s_j) + T(x_p, r_j). */
int ko_arrivals(const ko_desc* d, long npts, const double* px, const double* py, const double* pz,
                long ntr, const float* sx, const float* sy, const float* rx, const float* ry,
                double* out)
{
#pragma omp parallel for schedule(static)
    for (long p = 0; p < npts; ++p) {
        double x = px[p], y = (d->dim == 3) ? py[p] : 0.0, z = pz[p];
        for (long j = 0; j < ntr; ++j) {
            double ssy = (d->dim == 3) ? (double)sy[j] : 0.0, rry = (d->dim == 3) ? (double)ry[j] : 0.0;
            double Rs = sqrt((x - sx[j]) * (x - sx[j]) + (y - ssy) * (y - ssy) + z * z);
            double Rr = sqrt((x - rx[j]) * (x - rx[j]) + (y - rry) * (y - rry) + z * z);
            double Ts, Tr;
            if (d->vel == 3) {
                Ts = dsr_leg(d, sqrt((x - sx[j]) * (x - sx[j]) + (y - ssy) * (y - ssy)), z);
                Tr = dsr_leg(d, sqrt((x - rx[j]) * (x - rx[j]) + (y - rry) * (y - rry)), z);
            } else if (d->vel == 2) {
                Ts = table_traveltime(d, sqrt((x - sx[j]) * (x - sx[j]) + (y - ssy) * (y - ssy)), z);
                Tr = table_traveltime(d, sqrt((x - rx[j]) * (x - rx[j]) + (y - rry) * (y - rry)), z);
            } else if (d->vel == 4) {
                const int ls = grid_location(d, sx[j]), lr = grid_location(d, rx[j]);
                Ts = ls < 0 ? NAN : grid_traveltime(d, ls, x, z);
                Tr = lr < 0 ? NAN : grid_traveltime(d, lr, x, z);
            } else {
                traveltime(d, Rs, z, &Ts, NULL, NULL);
                traveltime(d, Rr, z, &Tr, NULL, NULL);
            }
            out[p * ntr + j] = Ts + Tr;
        }
    }
    return 0;
}

/* Work count of Eq. 2: number of (image point, in-aperture trace) pairs with a valid bin. */
long long ko_count(const ko_desc* d, long ntr, const float* sx, const float* sy, const float* rx,
                   const float* ry)
{
    const long ncol = (long)d->nx * d->ny;
    int* bin = (int*)malloc(sizeof(int) * (ntr > 0 ? ntr : 1));
    if (!bin) return -1;
    ko_bins(d, ntr, sx, sy, rx, ry, bin);
    long long total = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
    for (long j = 0; j < ntr; ++j) {
        if (bin[j] < 0) continue;
        float fsx = sx[j], fsy = hdr(sy, j), frx = rx[j], fry = hdr(ry, j);
        if (d->dim == 2) { fsy = 0.f; fry = 0.f; }
        long n = 0;
        for (long c = 0; c < ncol; ++c) {
            int iy = (int)(c / d->nx), ix = (int)(c % d->nx);
            float cx = col_coord(d->ox, ix, d->dx), cy = (d->dim == 3) ? col_coord(d->oy, iy, d->dy) : 0.f;
            n += inside_aperture(d, cx, cy, fsx, fsy, frx, fry);
        }
        total += (long long)n * d->nz;
    }
    free(bin);
    return total;
}
