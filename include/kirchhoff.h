/*
 * kirchhoff.h -- C ABI of a GB300 (sm_103a) library for Kirchhoff prestack migration.
 *
 * The operation is Eq. (1), Sec. 3 of "Distributed computing of Seismic Imaging
 * Algorithms":
 *
 *     I(x, X) = integral dx_s dx_r W(x, x_s, x_r) delta(X - |x_s - x_r|) D(x_s, x_r, T(x,x_s) + T(x,x_r))
 *
 * evaluated as a sum over recorded traces (Sec. 3: every sample of a trace adds into each image
 * point whose source-plus-receiver traveltime equals the sample's time), one offset image per
 * offset bin, at the cost f_K N_xyz N_tr of Eq. (2) where N_tr counts the traces near enough to
 * the image point to carry its reflections (Sec. 3 after Eq. 2; here a horizontal aperture).
 *
 * Conventions shared by every entry point
 *  - Every array argument is a DEVICE pointer owned by the caller unless stated.  Trace
 *    headers are FP32 metres: source (sx, sy), receiver (rx, ry), all at the surface
 *    z = 0 (Sec. 2).  For dim == 2, sy and ry may be NULL and are treated as 0.
 *  - Traces are row-major [ntr][nt] (time fastest) of the plan's trace dtype.
 *  - Images are FP32 row-major [n_bins][ny][nx][nz] (z fastest); ny == 1 for dim == 2.
 *  - Calls are asynchronous on `cuda_stream` (a cudaStream_t, NULL = legacy default
 *    stream).  Outputs are overwritten, never accumulated.  A plan may be used by one
 *    thread at a time.
 *  - Every failure returns a status code and sets a thread-local message readable with
 *    kirchhoff_last_error(); nothing aborts or traps.  Errors raised inside a kernel
 *    (a bounded wait that ran out, a trace position with no KH_VEL_GRID table) are reported by
 *    kirchhoff_sync(), which waits for the plan's work on the stream.
 *  - The plan owns its device workspace (trace sort order, headers, padded traces,
 *    traveltime tables); it grows on demand and is freed by kirchhoff_destroy().
 */
#ifndef KIRCHHOFF_H
#define KIRCHHOFF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define KH_API __attribute__((visibility("default")))
#else
#define KH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KH_OK = 0,
    KH_ERR_INVALID_ARG = 1,  /* NULL pointer, bad size, misaligned pointer, bad enum */
    KH_ERR_UNSUPPORTED = 2,  /* valid but not implemented (e.g. v(z) <= 0 inside the grid) */
    KH_ERR_OOM = 3,          /* device allocation for the plan workspace failed */
    KH_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    KH_ERR_TIMEOUT = 5,      /* a bounded in-kernel wait ran out; results are invalid */
    KH_ERR_INTERNAL = 6
} kh_status;

typedef enum { KH_F32 = 0, KH_F16 = 1, KH_BF16 = 2, KH_U16 = 3 } kh_dtype;

/* Traveltime T(x, x_a) from a surface point x_a to an image point x (Sec. 3: "times for
 * propagation in the model"; the paper gives no formula):
 *  KH_VEL_CONST:    T = R / v0, R = |x - x_a|.
 *  KH_VEL_LINEAR_Z: v(z) = v0 + k z, the circular-ray closed form
 *                   T = (2/k) asinh(k R / (2 sqrt(v0 (v0 + k z)))), evaluated as
 *                   T = arccosh(1 + q) / k, q = k^2 R^2 / (2 v0 (v0 + k z)).
 *  KH_VEL_TABLE:    the same v(z) = v0 + k z model read from a traveltime table.  Because
 *                   the model depends on depth only, the table of every surface location
 *                   is one radial table T(h, z) (h = horizontal distance), tabulated with
 *                   the closed form at nodes h_i = i D, z_j = z_a + j D (D = table_spacing,
 *                   z_a = D floor(shallowest image depth / D)) over the largest h of the
 *                   call's traces, stored as table_dtype, staged into shared memory and
 *                   read by bilinear interpolation in FP32.  table_dtype: KH_F32 (seconds),
 *                   KH_F16 (per h row, T minus the row's least-squares quadratic in the
 *                   normalised node depth, stored as FP16 beside the row's three FP32
 *                   coefficients) or KH_U16 (16-bit fixed point T = T_min + scale u,
 *                   scale = (T_max - T_min)/65535).  A migrate call
 *                   with a table plan reads the headers' extent back to the host (it
 *                   synchronises the stream).
 *  KH_VEL_PSTM:     prestack time migration (the PKTM of Sec. 4): the image's vertical axis
 *                   (oz, dz, nz) is the two-way vertical time t0 in seconds (t0 >= 0), and each
 *                   leg is the double-square-root time of a straight ray through a medium of
 *                   the RMS velocity of v(z) = v0 + k z down to the one-way vertical time t0/2,
 *                   T = sqrt((t0/2)^2 + h^2 / v_rms(t0)^2), h the horizontal distance,
 *                   v_rms(t0)^2 = v0^2 (e^{k t0} - 1) / (k t0).  Migration and the utilities
 *                   only (demigration and the velocity gradient refuse it).  The weight's
 *                   geometry is that of the straight rays: R = v_rms T, z = v_rms t0 / 2.
 *  KH_VEL_GRID:     a laterally varying model v(x, z) (dim 2), given on a node grid to
 *                   kirchhoff_grid_tables, which computes the first-arrival time table of every
 *                   surface location (see there); each leg reads its location's table by
 *                   bilinear interpolation.  v0 and k are not used.  Migration only (demigration,
 *                   the velocity gradient, the traveltime utility and the batched launch refuse
 *                   it).  The weight's geometry is that of straight rays (R = |x - x_a|). */
typedef enum { KH_VEL_CONST = 0, KH_VEL_LINEAR_Z = 1, KH_VEL_TABLE = 2, KH_VEL_PSTM = 3, KH_VEL_GRID = 4 } kh_vel;

/* Weight W(x, x_s, x_r) of Eq. (1) (it carries the propagation amplitude; no formula in the paper):
 *  KH_W_ONE:          W = 1.
 *  KH_W_OBLIQ_SPREAD: W = 1/2 (cos th_s + cos th_r) R_s R_r / r0^2 with cos th = z / R
 *                     (chord obliquity times spreading) = z (R_s + R_r) / (2 r0^2);
 *                     W = 0 where |z| < 1e-6 |dz|.
 *  KH_W_TRUE_AMP:     true amplitude, constant velocity only (KH_VEL_CONST): the weight of the
 *                     asymptotic Kirchhoff inversion for the reflection coefficient (Beylkin 1985,
 *                     Bleistein 1987), |h| / (a_s a_r |grad tau|^2) with h the Beylkin determinant of
 *                     the two-way time over the trace's midpoint at fixed offset and a_a the legs'
 *                     Green's-function amplitudes, with its global constants dropped:
 *                       W = (R_s R_r)^((dim - 1) / 2) |det[g, D u_x (, D u_y)]| / |g|^2,
 *                       g = e_s + e_r, e_a = (x - x_a) / R_a, D u = sum_a (u - e_a (e_a . u)) / R_a
 *                     (2D: the (x, z) plane), which reduces to z (R_s + R_r)(1/R_s^2 + 1/R_r^2) / 2 (3D)
 *                     and z sqrt(R_s R_r)(1/R_s^2 + 1/R_r^2) / 2 (2D), the form the kernels evaluate:
 *                     2 cos th (3D) or cos th (2D) at zero offset.
 *                     Applied to time-differentiated 3D data, a horizontal reflector's image has the
 *                     same peak at every offset and depth.  W = 0 where |z| < 1e-6 |dz|.  Migration
 *                     and demigration (the velocity gradient and the batched launch refuse it). */
typedef enum { KH_W_ONE = 0, KH_W_OBLIQ_SPREAD = 1, KH_W_TRUE_AMP = 2 } kh_weight;

typedef struct {
    int dim;                 /* 2 or 3 */
    int nx, ny, nz;          /* image samples; ny = 1 for dim = 2 */
    double ox, oy, oz;       /* image origin, metres (z positive down from the surface) */
    double dx, dy, dz;       /* image spacing, metres, > 0 */
    int n_bins;              /* offset bins: X in [b w, (b+1) w) goes to bin b; X = n_bins w goes to
                                the last bin; larger offsets are not imaged (Eq. 1's delta) */
    double bin_width;        /* w > 0, metres */
    kh_vel vel;
    double v0, k;            /* v(z) = v0 + k z; k ignored for KH_VEL_CONST */
    double table_spacing;    /* KH_VEL_TABLE: node spacing of the traveltime tables, metres */
    kh_dtype table_dtype;    /* KH_VEL_TABLE: KH_F32, KH_F16 (residual of a per-row quadratic) or
                                KH_U16 (offset + scale) */
    kh_weight weight;
    double r0;               /* spreading normaliser, metres (KH_W_OBLIQ_SPREAD) */
    double aperture;         /* horizontal image-column to trace-midpoint distance limit, metres;
                                <= 0 means every trace reaches every column ("traces close
                                enough", Sec. 3 after Eq. 2) */
    int nt;                  /* samples per trace, >= 2 */
    double t0, dt;           /* time of sample 0 and sample interval, seconds */
    kh_dtype trace_dtype;    /* storage type of the traces passed to migrate */
    double taper;            /* aperture taper: the weight falls from 1 to 0 over the outer fraction
                                `taper` of the aperture as a raised cosine of the column-to-midpoint
                                distance d, (1 + cos(pi (d - (1 - taper) A) / (taper A))) / 2 beyond
                                (1 - taper) A; in [0, 1), 0 = a hard mask; ignored without an
                                aperture.  Every operator (migrate, demigrate, velocity gradient)
                                applies it, so they stay each other's transpose and derivative. */
    double aa_spacing;       /* operator anti-aliasing, KH_VEL_CONST and KH_VEL_LINEAR_Z: the trace
                                (midpoint) spacing in metres, 0 = off.  With p the midpoint gradient
                                of the two-way time in samples per metre, p = (g_s + g_r) / dt, g_a
                                the horizontal gradient of leg a's time at the image point
                                ((x - x_a)_h / (v0 R_a) at constant velocity; (x - x_a)_h /
                                (R_a sqrt(v0 v(z) + k^2 R_a^2 / 4)) for v0 + k z), the moveout
                                between adjacent traces is L = aa_spacing max(|p_x|, |p_y|)
                                samples; the weight keeps L <= 1, removes L >= 2 and falls as
                                cos^2(pi (L - 1) / 2) between (dip limitation of the operator: the
                                aliased part of the sum is dropped).  Migrate and demigrate, and
                                the allocation-free entry point; the velocity gradient and the
                                batched launch refuse it (KH_ERR_UNSUPPORTED), and so does
                                KH_VEL_LINEAR_Z (k != 0) with 16-bit traces.  Negative or not
                                finite: KH_ERR_INVALID_ARG; > 0 with another velocity kind:
                                KH_ERR_UNSUPPORTED. */
} kh_desc;

typedef struct kh_plan_s* kh_plan;

/* Validates `d` and creates a plan.  On success *out owns host and device state.
 * Returns KH_ERR_INVALID_ARG for a NULL pointer or out-of-range field and
 * KH_ERR_UNSUPPORTED when v(z) <= 0 somewhere in [min(0, oz), oz + (nz-1) dz]. */
KH_API kh_status kirchhoff_create(const kh_desc* d, kh_plan* out);

/* Frees the plan and its device workspace (synchronises the device first).  NULL is a no-op. */
KH_API kh_status kirchhoff_destroy(kh_plan p);

/* Migration, Eq. (1): image[b][iy][ix][iz] = sum over traces j with offset bin b whose
 * midpoint lies within the aperture of column (ix, iy) of
 *     W * ((1 - f) D_j[i] + f D_j[i+1]),  tau = (T_s + T_r - t0)/dt, i = floor(tau), f = tau - i,
 * for 0 <= tau <= nt-1 (at tau = nt-1: i = nt-2, f = 1); other tau contribute nothing.
 * sx, sy, rx, ry: [ntr] FP32; traces: [ntr][nt] of the plan's trace_dtype, 16-byte
 * aligned; image: [n_bins][ny][nx][nz] FP32, overwritten.  ntr == 0 gives a zero image.
 * Accumulation is FP32; the result is bitwise reproducible run to run. */
KH_API kh_status kirchhoff_migrate(kh_plan p, int ntr, const float* sx, const float* sy, const float* rx,
                            const float* ry, const void* traces, float* image, void* cuda_stream);

/* Demigration: the transpose of kirchhoff_migrate for the same plan and headers (the
 * same sum read from the data side, Sec. 3).  image: [n_bins][ny][nx][nz] FP32;
 * traces_out: [ntr][nt] FP32, overwritten:
 *     traces_out[j][i] += W (1-f) image[b_j][x],  traces_out[j][i+1] += W f image[b_j][x]. */
KH_API kh_status kirchhoff_demigrate(kh_plan p, int ntr, const float* sx, const float* sy,
                              const float* rx, const float* ry, const float* image,
                              float* traces_out, void* cuda_stream);

/* Derivative of the bilinear form B(m, D) = <m, migrate(D)> with respect to the
 * velocity parameters (v0, k) of KH_VEL_LINEAR_Z (or v0 alone for KH_VEL_CONST):
 *     dB/dth = sum W m[b_j][x] (D_j[i+1] - D_j[i]) dtau/dth,  dtau/dth = (dT_s/dth + dT_r/dth)/dt.
 * It is the velocity-update gradient of the inverse flow (Sec. 4, Inverse PKTM) and serves
 * the backward pass of both migrate and demigrate.  image: FP32 [n_bins][ny][nx][nz];
 * traces: FP32 [ntr][nt]; out_dv0_dk: DEVICE double[2], overwritten.  Per-CTA FP64
 * partials are reduced in a fixed order (bitwise reproducible).  KH_ERR_UNSUPPORTED for
 * KH_VEL_TABLE. */
KH_API kh_status kirchhoff_velocity_grad(kh_plan p, int ntr, const float* sx, const float* sy,
                                  const float* rx, const float* ry, const float* image,
                                  const float* traces, double* out_dv0_dk, void* cuda_stream);

/* Traveltime evaluation (the T of Eq. 1 under the plan's velocity model) for n
 * elementwise (point, surface location) pairs: T[i] = T((px,py,pz)[i], (lx,ly)[i]) (for
 * KH_VEL_PSTM, pz is the two-way vertical time t0).  All arrays device FP32 [n]; ly/py may be
 * NULL for dim 2. */
KH_API kh_status kirchhoff_traveltime(kh_plan p, int n, const float* px, const float* py,
                               const float* pz, const float* lx, const float* ly, float* T,
                               void* cuda_stream);

/* Host-only report (no device work, no plan) of the ln(1 + rho) fits the linear-v(z) kernels
 * use for an image tile of cx x cy columns x (cz * 16) depths of descriptor `d`; the T of
 * Eq. (1) is the linear-gradient closed form, evaluated per leg as
 * T - T_c = ln(1 + rho) / |k| with rho = U/U_c - 1 relative to the tile centre c.
 *   two_leg_terms: length of the two-leg fit that accepts the tile;
 *   leg_terms:     length of the per-leg fit the kernels evaluate (4, 5, 6, 8, 12 or 20);
 *   leg_bound:     b, with rho in [expm1(-b), expm1(b)] for every leg over the tile;
 *   coef:          20 floats, the per-leg coefficients scaled by C1 = 1/(|k| dt):
 *                  C1 ln(1 + rho) = rho (coef[0] + rho sum_{j>=1} coef[j] x^(j-1)),
 *                  x = rho * scale + offset (scale 1, offset 0 up to 8 terms), zero beyond
 *                  leg_terms;
 *   c1:            C1 in FP64.
 * Any output pointer may be NULL.  Errors: KH_ERR_INVALID_ARG (bad descriptor or tile, or a
 * descriptor that is not linear v(z) with k != 0), KH_ERR_UNSUPPORTED (no fit length meets the
 * budget of 5e-6 samples for the tile). */
KH_API kh_status kirchhoff_fit_report(const kh_desc* d, int cx, int cy, int cz, int* two_leg_terms,
                                      int* leg_terms, double* leg_bound, float* coef, float* scale,
                                      float* offset, double* c1);

/* ---------------------------------------------------------------- velocity analysis
 * Sec. 2: migration with an estimate of the velocity produces redundant images (here one per
 * offset bin); differences in the position of the same reflector between them measure the error
 * of the velocity model, which is corrected before the data are migrated again and, once the
 * images agree, stacked.  kirchhoff_semblance measures that disagreement for an offset-binned
 * image of plan `p`:
 *     V = sum_b ||w_b I_b - m||^2 / sum_b ||w_b I_b||^2,   m = (1/N) sum_b w_b I_b,
 * the normalised variance of the weighted images across the N bins with w_b > 0 (0 when all
 * agree, 1 - 1/N for images with disjoint supports), and optionally its image gradient
 *     grad[b] = dV/dI_b = (2 w_b / B) ((w_b I_b - m) - V w_b I_b),   B = sum_b ||w_b I_b||^2,
 * so that kirchhoff_velocity_grad(p, ..., image = grad, traces = D, ...) gives dV/d(v0, k) of the
 * images migrated with p.  image: DEVICE FP32 [n_bins][ny][nx][nz]; bin_weight: HOST double
 * [n_bins], >= 0, or NULL for w_b = 1 / (traces of bin b in p's last migrate or gradient call);
 * (only traces the sort kept count: a trace whose midpoint is farther than the aperture from
 * every image column is dropped by the sort and reaches no image point);
 * out: HOST double[3] = (V, D, B), D and B the two sums; grad_image: DEVICE FP32, image-shaped,
 * overwritten, or NULL.  Sums are FP64 in a fixed order (the result does not change from run to
 * run).  Synchronises `cuda_stream`.  Errors: KH_ERR_INVALID_ARG (NULL image/out, negative or
 * non-finite weights, all weights zero, NULL weights before any migration of p). */
KH_API kh_status kirchhoff_semblance(kh_plan p, const float* image, const double* bin_weight, double* out,
                                     float* grad_image, void* cuda_stream);

/* ---------------------------------------------------------------- gridded model v(x, z)
 * Sec. 3 takes T from the high-frequency limit of ray theory, one path per source and image
 * point: the first-arrival time, the solution of the eikonal equation |grad T| = 1/v with T = 0 at
 * the surface location.  For a laterally varying model (KH_VEL_GRID, dim 2) the library solves it
 * on a node grid for every surface location and the migration reads the tables.
 *
 * Node grid (kh_grid): nodes (ox + i h, j h), i < nx, j < nz, z fastest, row 0 at the surface,
 * with h = m dz (m = 1, 2 or 4, to 1e-9 relative) and the image's oz a non-negative multiple of h
 * (to 1e-9), so that image depth iz lies at node row oz/h + iz/m.  The columns must cover every
 * image column and every location; nz >= oz/h + 16 ceil(nz_image / 16) / m + 1 (one node below
 * the deepest depth a migration tile evaluates); nx, nz >= 2, nx nz <= 28000 and
 * 8.125 nx nz + 4 nx <= 232192 bytes (the solver keeps a location's grid in FP64, one bit per node
 * and one FP32 offset per column in one CTA's shared memory).
 *
 * kirchhoff_grid_layout (host only): the smallest such grid for descriptor `d` (vel KH_VEL_GRID)
 * and node spacing multiple m whose columns cover the image and [xmin, xmax] (the locations'
 * range) with `margin` >= 0 spare columns on each side, ox a multiple of h.
 *
 * kirchhoff_grid_tables: for the model v (DEVICE FP32 [grid->nx][grid->nz], m/s, finite, > 0) and
 * nloc >= 1 locations loc_x (DEVICE FP32 [nloc], strictly increasing, inside the grid's columns),
 * builds in the plan one FP32 table per location, on one CTA per location:
 *   - factorisation T = T0 + tau, T0 = s0 |x - x_s| with s0 the slowness at the location (linear
 *     along the surface row), which removes the point-source singularity (additive factor of
 *     Luo and Qian, 2012); constant velocity is reproduced to rounding;
 *   - the Godunov upwind discretisation of |grad T0 + grad tau| = s: with c_x = min(tau_left -
 *     h dT0/dx, tau_right + h dT0/dx) and c_z likewise, tau = min(c_x, c_z) + h s if
 *     |c_x - c_z| >= h s, else (c_x + c_z + sqrt(2 (h s)^2 - (c_x - c_z)^2)) / 2, taken if smaller;
 *   - fast sweeping (Zhao, 2005): Gauss-Seidel passes in the orderings (i up, j up), (i down,
 *     j up), (i down, j down), (i up, j down), each pass as a wavefront of anti-diagonals (the
 *     nodes of one anti-diagonal are independent within a pass, so the result is that of the
 *     sequential pass); rounds of four passes until a round's largest decrease is <= 1e-7 s, at
 *     most 64 rounds; a node is recomputed only after one of its neighbours changed (the same
 *     result with less work);
 *   - the nodes with |x_i - x_s| <= 2 h in rows 0..2 keep the straight-ray time
 *     |x - x_s| (s0 + s(x)) / 2 and are not updated;
 *   - tau, the node equation and the convergence test in FP64 (tau accumulates along every
 *     path), the equation's square root an FP32 estimate refined by one FP64 Newton step; the
 *     shift h grad T0 in FP32 from the FP64 offset x - x_s (relative error below 5e-7, a few
 *     1e-9 s per node); stored as FP32.
 * Synchronises the stream.  Errors: KH_ERR_INVALID_ARG (NULL pointers, a grid that breaks the
 * rules above, v not finite and > 0, locations not increasing or outside the columns, a plan that
 * is not KH_VEL_GRID), KH_ERR_UNSUPPORTED (a location that did not settle in 64 rounds).
 * A later kirchhoff_migrate reads the tables: each trace's source and receiver x must equal one
 * of loc_x exactly; a trace whose position does not is skipped and kirchhoff_sync reports
 * KH_ERR_INVALID_ARG.  Per image tile and location the migration takes the smallest and largest
 * node value the tile interpolates between as the time window's bounds.
 *
 * kirchhoff_grid_read: copies the plan's tables (DEVICE FP32 [nloc][nz][nx], row-major with x
 * fastest, the layout the migration reads; NULL skips) and the
 * rounds each location took (DEVICE int [nloc]; NULL skips); *nloc (HOST, may be NULL) = nloc.
 * Synchronises the stream. */
typedef struct {
    int nx, nz;              /* nodes along x and z */
    double ox, h;            /* x of node column 0, and the node spacing in x and z, metres */
} kh_grid;

KH_API kh_status kirchhoff_grid_layout(const kh_desc* d, int m, double xmin, double xmax, int margin,
                                       kh_grid* out);
KH_API kh_status kirchhoff_grid_tables(kh_plan p, const kh_grid* grid, const float* v, int nloc,
                                       const float* loc_x, void* cuda_stream);
KH_API kh_status kirchhoff_grid_read(kh_plan p, float* tables, int* rounds, int* nloc, void* cuda_stream);

/* ---------------------------------------------------------------- the binning sort
 * Eq. (1)'s delta(X - |x_s - x_r|) assigns each trace to one offset bin, and only traces "close
 * enough" to an image point contribute (Sec. 3 after Eq. 2).  Before every migration and
 * gradient call the library sorts the traces by (offset bin, midpoint cell, original index) on
 * a grid of cells over the image columns widened by the aperture, so that each CTA examines
 * only the cells that meet its tile's aperture disc.  These two calls expose that step.
 *
 * kirchhoff_cell_grid (host only): the grid of descriptor `d` with spatial sorting on (1) or off
 * (0) (see KH_OPT_SPATIAL_SORT for when "on" still gives one cell): ncx x ncy square cells from
 * (gx0, gy0), inv_cell = 1 / cell side in metres.  A trace's
 * cell is cx = floor((m_x - gx0) * inv_cell), cy = floor((m_y - gy0) * inv_cell) (FP64 products
 * of the FP32 midpoint m = (s + r) * 0.5f; cy = 0 for dim 2), its key
 * bin * ncx * ncy + cy * ncx + cx.  Traces without a bin, or whose cell is outside the grid
 * (farther than the aperture from every image column), are dropped.  With no aperture
 * (aperture <= 0) there is one cell (ncx = ncy = 1, inv_cell = 0) and no trace is dropped for
 * its position.  Any output pointer may be NULL.
 *
 * kirchhoff_bin_sort: runs the sort of plan `p` (its KH_OPT_SPATIAL_SORT setting) on the
 * headers and copies out perm_out (DEVICE int [ntr]: the original indices of the kept traces in
 * sorted order, first; the entries past the kept count are unspecified) and key_start_out
 * (DEVICE int [n_bins * ncx * ncy + 1]: the first sorted position of each key; the last entry
 * is the number of kept traces).  The sort is a stable radix sort over all SMs: equal keys keep
 * their original order, and the result is the same on every run. */
KH_API kh_status kirchhoff_cell_grid(const kh_desc* d, int spatial, int* ncx, int* ncy, double* gx0,
                                     double* gy0, double* inv_cell);
KH_API kh_status kirchhoff_bin_sort(kh_plan p, int ntr, const float* sx, const float* sy, const float* rx,
                                    const float* ry, int* perm_out, int* key_start_out, void* cuda_stream);

/* Work count of Eq. (2): number of (image point, trace) pairs with a valid offset bin
 * and the trace midpoint within the aperture of the point's column, computed on the
 * device with the same FP32 aperture test as the migration kernel.  *out_count is a
 * HOST int64; the call synchronises `cuda_stream`. */
KH_API kh_status kirchhoff_count(kh_plan p, int ntr, const float* sx, const float* sy, const float* rx,
                          const float* ry, int64_t* out_count, void* cuda_stream);

/* ---------------------------------------------------------------- batched persistent launch
 * Many independent migrations, each with its own plan (grid, bins, v(z), tile), headers,
 * traces and image, in ONE launch of a persistent kernel (one per ln(1 + rho) polynomial
 * length when linear-v(z) jobs need different lengths).  Each job computes Eq. (1) exactly
 * as kirchhoff_migrate does with the same plan (bit-identical images: the same tile code,
 * traces in the same order).  A job list becomes a device work list of (job, image tile,
 * offset bin) items: jobs by descending estimated cost, each job's bins in order, the items
 * of a bin longest first (cost = tile points x traces of the bin that pass the aperture cull
 * of the tile).  One CTA per SM slot takes items from a single work counter (a scheduler
 * index; no image value is accumulated in global memory), so jobs of very different sizes
 * (Eq. 2: work ~ N_xyz N_tr per job) share the 152 SMs with no launch gap or tail per job.
 * The paper distributes independent images over cluster nodes; it has no single-GPU
 * counterpart of this entry point. */

/* One migration job of a batch. */
typedef struct {
    kh_plan plan;            /* the job's plan (grid, bins, velocity, dtype, KH_OPT_TILE) */
    int ntr;
    const float *sx, *sy, *rx, *ry;   /* device headers, read once by kirchhoff_batched_prepare */
    const void* traces;      /* device [ntr][nt] rows in the plan's trace dtype, read at every launch */
    float* image;            /* device [n_bins][ny][nx][nz], written (fully) at every launch */
} kh_job;

typedef struct kh_batch_s* kh_batch;

/* Plans a batch: validates the jobs, bins each job's headers into the batch's own device
 * buffers, counts culled traces per (tile, bin), builds and uploads the sorted work list and
 * sizes the grid (152 x resident CTAs per SM).  It allocates and synchronises `cuda_stream`;
 * the plans and header arrays may be used for other calls afterwards.  The trace and image
 * pointers are recorded and used by every kirchhoff_migrate_batched() call.
 * All jobs must share the trace dtype, weight, fast-math option and velocity kind (constant,
 * k = 0, or linear v(z)); tables (KH_VEL_TABLE) are refused with KH_ERR_UNSUPPORTED.
 * Wait limits follow jobs[0].plan's KH_OPT_WAIT_POLLS.  Errors: KH_ERR_INVALID_ARG (NULL
 * pointers, plans of another device), KH_ERR_UNSUPPORTED, KH_ERR_OOM, KH_ERR_CUDA. */
KH_API kh_status kirchhoff_batched_prepare(int njobs, const kh_job* jobs, kh_batch* out,
                                           void* cuda_stream);
/* Runs the batch on `cuda_stream`: row padding for jobs whose trace rows are not 16-byte
 * aligned, a reset of the work counter and the persistent kernel.  Stream work only (no
 * allocation, no synchronisation, no host read), so a CUDA graph may capture it; replays
 * read the traces and write the images recorded at prepare.  Two launches of one batch
 * must not overlap (they share the work counter). */
KH_API kh_status kirchhoff_migrate_batched(kh_batch b, void* cuda_stream);
/* Waits for `cuda_stream`; KH_ERR_TIMEOUT if a bounded wait of the batch's kernel ran out. */
KH_API kh_status kirchhoff_batch_sync(kh_batch b, void* cuda_stream);
/* Work items, grid size (CTAs), estimated contributions (culled traces x tile points,
 * summed over items) and launches issued so far; any output pointer may be NULL. */
KH_API kh_status kirchhoff_batch_info(kh_batch b, long long* n_items, int* n_ctas,
                                      double* est_contributions, long long* launches);
/* Frees the batch's device workspace (synchronises the device through cudaFree). */
KH_API kh_status kirchhoff_batch_destroy(kh_batch b);

/* Waits for the plan's work on `cuda_stream` and reports what its kernels flagged since the
 * last call (clearing the flags): KH_ERR_TIMEOUT if a bounded in-kernel wait ran out (results
 * invalid), KH_ERR_INVALID_ARG if a KH_VEL_GRID trace's position had no table (those traces were
 * skipped), KH_ERR_INTERNAL for an internal sizing error, else KH_OK.  The image copies of
 * kirchhoff_migrate_host run on the plan's own stream: join them first (kirchhoff_host_join). */
KH_API kh_status kirchhoff_sync(kh_plan p, void* cuda_stream);

/* Tuning and test options of a plan (kirchhoff_set_option).
 *  KH_OPT_WAIT_POLLS: limit every bounded in-kernel wait to `value` polls (0 restores the
 *                     default, about two seconds of polling).  A test sets 1 to check that
 *                     a wait which runs out returns KH_ERR_TIMEOUT with the context intact.
 *  KH_OPT_FAST_MATH:  1 = hardware approximate square root and reciprocal in the hot loop
 *                     (default), 0 = IEEE-rounded ones; both are parity-tested.
 *  KH_OPT_TILE:       image tile of one CTA, encoded as cx | cy << 10 | cz << 20 (threads per
 *                     CTA along x, y and z-groups, cx*cy*cz == 256, cz <= 16; each thread owns
 *                     16 consecutive z samples of one column); 0 restores the default.
 *  KH_OPT_BATCH_MODE: read from jobs[0].plan by kirchhoff_batched_prepare.  0 (default) = one
 *                     persistent kernel over the work list; 1 = every job's own migration
 *                     kernel on library-owned streams forked from and joined to the caller's
 *                     stream (one graph with parallel branches when captured), so that the
 *                     block scheduler fills one job's tail with the next job's tiles.
 *  KH_OPT_SAMPLE_PAIRS: 1 (default) = kirchhoff_migrate stages FP32 traces of constant or
 *                     linear v(z) plans with nt <= 2460 as (d[i], d[i+1] - d[i]) pairs in plan
 *                     workspace (8 bytes per sample, one pass over the traces), so that each
 *                     interpolated sample takes one shared-memory load; 0 = plain samples.
 *                     The image is bit-identical either way.
 *  KH_OPT_SPATIAL_SORT: 1 (default) = the binning sort orders each offset bin's traces by the
 *                     cell of their midpoint on a grid of about half the aperture (at most 16
 *                     cells per axis), and each CTA of the migration and gradient kernels
 *                     examines only the cells that meet its tile widened by the aperture; the
 *                     grid is used only where a default tile's aperture disc spans at most half
 *                     of its cells (else one cell, as with 0);
 *                     0 = each bin's traces in their original order, every CTA examining its
 *                     whole bin.  Both keep exactly the same (point, trace) pairs; only the
 *                     summation order differs (FP32 rounding).  Without an aperture there is one
 *                     cell either way.  Demigration always sorts by bin alone. */
typedef enum {
    KH_OPT_WAIT_POLLS = 1,
    KH_OPT_FAST_MATH = 2,
    KH_OPT_TILE = 3,
    KH_OPT_BATCH_MODE = 4,
    KH_OPT_SAMPLE_PAIRS = 5,
    KH_OPT_SPATIAL_SORT = 6
} kh_option;
KH_API kh_status kirchhoff_set_option(kh_plan p, kh_option opt, long long value);

/* Profiling: while enabled, CUDA events bracket the main kernel of every migrate /
 * demigrate / gradient call of this plan on the call's stream.  kirchhoff_profile_read()
 * waits for those events and returns the summed main-kernel time in milliseconds and the
 * number of timed launches since the previous read, then resets both. */
KH_API kh_status kirchhoff_profile(kh_plan p, int enable);
KH_API kh_status kirchhoff_profile_read(kh_plan p, double* kernel_ms, long long* timed_launches);

/* Staging statistics of the migration and gradient kernels while profiling is enabled: the
 * traces the staging warps examined (the sorted trace ranges of the offset-bin cells that meet
 * each CTA's aperture-widened tile), those they staged (that passed the aperture cull and have a
 * sample window in the tile), and the CTAs that ran, each summed since the previous read, then
 * reset.  Synchronises `cuda_stream`; all 0 if profiling was never enabled. */
KH_API kh_status kirchhoff_staging_stats(kh_plan p, void* cuda_stream, unsigned long long* examined,
                                         unsigned long long* staged, unsigned long long* ctas);

/* Host-resident migration (no counterpart in the paper: the interface for surveys that live in
 * host memory).  The same operation and result as kirchhoff_migrate, with sx, sy, rx, ry and
 * traces in HOST memory (the layouts of kirchhoff_migrate; sy, ry may be NULL for dim 2) and the
 * image written to HOST memory `image` ([n_bins][ny][nx][nz] FP32).  The call only enqueues: the
 * inputs are copied into one of two plan-owned slots of device buffers on a plan-owned copy
 * stream, migrated on `cuda_stream` once they are in, and the image is copied back on a second
 * plan-owned copy stream once the migration is done.  Consecutive calls use the slots in turn,
 * so call n's inputs travel while call n-1 migrates and call n-1's image travels while call n
 * migrates.  The host buffers belong to the library until the call's image has arrived: make a
 * stream wait for it with kirchhoff_host_join, then synchronise that stream (kirchhoff_sync
 * reports a bounded wait that ran out).  Pinned host memory (cudaHostAlloc / cudaHostRegister)
 * gives the overlap; pageable memory gives the same result with copies that block the caller.
 * Successive calls must use the same `cuda_stream`.  The slots hold two copies of the traces
 * and two images on the device.  Errors: KH_ERR_INVALID_ARG for a NULL plan, image, header or
 * trace array (ntr > 0) or ntr < 0; KH_ERR_CUDA when an allocation, copy or launch fails; every
 * error of kirchhoff_migrate. */
KH_API kh_status kirchhoff_migrate_host(kh_plan p, int ntr, const float* sx, const float* sy,
                                        const float* rx, const float* ry, const void* traces, float* image,
                                        void* cuda_stream);

/* Makes `cuda_stream` wait (on the device) until every image that kirchhoff_migrate_host has
 * enqueued for this plan has arrived in host memory.  Returns without waiting on the host. */
KH_API kh_status kirchhoff_host_join(kh_plan p, void* cuda_stream);

/* Number of kernel launches issued by this plan since creation (for launch accounting). */
KH_API long long kirchhoff_launch_count(kh_plan p);

/* Allocation-free migration (no counterpart in the paper: an interface for callers that
 * cannot allocate device memory, such as services whose HBM is owned by another allocator's
 * pool, or that must not call cudaMalloc after start-up because it can synchronise the
 * device).  Same operation, arguments and result as kirchhoff_migrate, without a plan: the
 * descriptor is validated on every call and the trace-sort scratch is one fixed 2.1 MB
 * __device__ array inside the library, held by every GPU that loads it until the process
 * exits.  Limits: ntr <= 65536, FP32 traces, trace rows 16-byte aligned (nt a multiple of 4).
 * Larger inputs return KH_ERR_INVALID_ARG with a message; nothing is allocated.
 * `status` is an optional DEVICE int: it is zeroed, then bit 0 is set if a bounded in-kernel
 * wait ran out (NULL: a word inside the scratch is used and the outcome is not reported).
 * The first call on each device looks up the scratch's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  The address is kept for the life of the
 * process: it belongs to the device's primary context, so a process that destroys that
 * context (cudaDeviceReset) must not call this entry point on that device afterwards.  All calls on a device share the scratch
 * and it keeps the previous call's contents: calls that overlap on the GPU (for example on
 * two streams) race and must be serialised by the caller. */
KH_API kh_status kirchhoff_migrate_noalloc(const kh_desc* d, int ntr, const float* sx,
                                           const float* sy, const float* rx, const float* ry,
                                           const void* traces, float* image, int* status,
                                           void* cuda_stream);

/* Thread-local message of the last failure ("" if none). */
KH_API const char* kirchhoff_last_error(void);

/* Library version string. */
KH_API const char* kirchhoff_version(void);

#ifdef __cplusplus
}
#endif
#endif /* KIRCHHOFF_H */
