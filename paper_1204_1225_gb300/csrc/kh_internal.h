// Internal declarations shared by the library's translation units (host and device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kirchhoff.h"

namespace kh {

// Each consumer thread owns NZ consecutive z samples of one image column.
constexpr int NZ = 16;
// Consumer warps per CTA (256 threads) plus one producer warp that stages traces.
constexpr int CONSUMER_WARPS = 8;
constexpr int CONSUMERS = CONSUMER_WARPS * 32;
constexpr int THREADS = CONSUMERS + 32;
// Trace staging ring: stages, traces per stage.
constexpr int STAGES = 3;
constexpr int BMAX = 64;
// Bit pattern of 1.5 * 2^23: adding it to |x| < 2^22 leaves round(x) in the low mantissa bits.
constexpr float MAGIC = 12582912.0f;
constexpr int MAGIC_BITS = 0x4B400000;

// The two-leg ln(1 + rho) fit of the linear-velocity delta formulation (rho = U/U_c - 1 of both
// legs): the shortest length of LP_TERMS whose fit meets the error budget over the tile's rho
// bound decides whether a tile is accepted (6 terms for compact tiles of a fine grid, up to 20
// for wide ones).  LP_SHORT is the reference length for tile choice and the template length of
// kernels that evaluate no polynomial.
constexpr int LP_TERMS[] = {6, 8, 10, 12, 20};
constexpr int N_LP_TERMS = 5;
constexpr int LP_SHORT = 12;
constexpr int LP_LONG = 20;
// The kernels evaluate ln(1 + rho) per leg (rho = U/U_c - 1 of one leg, half the range of the
// two-leg rho) and cache or share the source leg's term: lengths up to LG_MONO are monomial in
// rho (no change of variable), longer ones use the shifted variable t.
constexpr int LG_TERMS[] = {4, 5, 6, 8, 12, 20};
constexpr int N_LG_TERMS = 6;
constexpr int LG_MONO = 8;

// An FP32 trace sample and the step to the next one, (d[i], d[i + 1] - d[i]) with d[nt] = 0:
// the staging layout of FP32 traces for the migration kernel, so that one 8-byte shared load
// serves each interpolated sample.  PAIR_MAX_NT is the longest trace whose pair row still fits
// one ring stage; longer traces are staged as plain samples.
struct __align__(8) SamplePair {
    float v, d;
    SamplePair() = default;
    __host__ __device__ explicit SamplePair(float z) : v(z), d(z) {}
};
constexpr int PAIR_MAX_NT = 2460;

// A contribution is valid iff 0 <= tau <= nt - 1 (the oracle's exact rule), decided on the FP32 tau,
// whose rounding (about 1e-5 samples) cannot settle a tau that lies exactly on an edge: the
// kernels accept tau up to EDGE_EPS samples beyond each edge, so that the edge samples themselves
// (tau = 0 and tau = nt - 1 in exact arithmetic) are kept on every path.  Beyond an edge the
// interpolation reads the window's zero or finite neighbour with a weight below EDGE_EPS.
constexpr float EDGE_EPS = 1.0f / 1024.0f;

// Default wait limit: polls of mbarrier.try_wait, each checked against a 2 s wall clock.
constexpr long long WAIT_NS = 2000000000LL;

enum VelKind { VK_CONST = 0, VK_LINEAR = 1, VK_TABLE = 2, VK_PSTM = 3, VK_GRID = 4 };

// Gridded model v(x, z) (KH_VEL_GRID): at most this many nodes, so that the eikonal solver keeps
// a location's grid in one CTA's shared memory (FP64 values and one dirty bit per node).
constexpr int MAX_GRID_NODES = 28000;
// Plan status bits beyond bit 0 (a bounded wait ran out): bit 1 demigration sizing, bit 2 a
// trace position with no traveltime table.
constexpr int STATUS_NO_TABLE = 4;

// RMS velocity of v(z) = v0 + k z down to the two-way vertical time t0: v0^2 (e^{k t0} - 1)/(k t0)
// (v(tau) = v0 e^{k tau} at one-way vertical time tau; the mean of v^2 over [0, t0/2]).
__host__ __device__ inline double vrms2_of(double v0, double k, double t0)
{
    const double x = k * t0;
    if (x < 1e-6 && x > -1e-6) return v0 * v0 * (1.0 + x * (0.5 + x / 6.0));
    return v0 * v0 * expm1(x) / x;
}

// Midpoint cells of the binning sort.  Traces are ordered by (offset bin, cell row cy, cell
// column cx, original index); cell (cx, cy) covers midpoints m with
// floor((m_x - gx0) inv_cs) = cx (FP64), likewise in y.  The grid covers the image columns
// widened by `margin` (a little more than the aperture), so a midpoint outside it is farther
// than the aperture from every column and is dropped with the traces that have no offset bin.
// With a full aperture (margin <= 0) there is one cell and nothing is dropped.
// Bit of the migration kernels' weight template parameter that compiles the operator
// anti-aliasing weight in (constant velocity; kernels without it never evaluate it).
constexpr int W_AA = 4;

// Offset bins the velocity-analysis kernels carry weights for (the plan allows up to 256).
constexpr int MAX_BIN_WEIGHTS = 256;
constexpr int MAX_CELLS_PER_AXIS = 16;
constexpr int MAX_CELL_ROWS = MAX_CELLS_PER_AXIS;
struct CellGrid {
    int ncx = 1, ncy = 1;
    double gx0 = 0.0, gy0 = 0.0;
    double inv_cs = 0.0;     // 1 / cell size
    double margin = 0.0;     // aperture widening of the tile footprint for its cell range
};

// Sorted trace set produced by the binning pass (plan workspace).
struct TraceSet {
    const float4* hdr;      // (sx, sy, rx, ry) in sorted order
    const float2* mid;      // FP32 midpoints (sx + rx) * 0.5f, (sy + ry) * 0.5f
    const int* perm;        // original trace index
    const int* bin_start;   // [n_bins + 1]
    // [n_bins * ncx * ncy + 1]: start of every (bin, cell) key in sorted order (nullptr: the
    // traces of a bin are one range, bin_start[b] .. bin_start[b + 1])
    const int* cell_start = nullptr;
    CellGrid cg{};
};

// Everything a migration-type kernel needs, passed by value.
struct GeomParams {
    int dim, nx, ny, nz, n_bins;
    double ox, oy, oz, dx, dy, dz;
    float fdz;
    // velocity (FP32 constants for the hot loop, FP64 for per-z set-up)
    double v0, k;            // v(z) = v0 + k z (k = 0: constant velocity)
    double kabs;
    double a;                // k^2 / (2 v0): q = a R^2 / (v0 + k z)
    float lp[LP_LONG];       // ln(1 + rho) = rho (1 + rho Q(t)), t = rho lp_s + lp_o,
                             // Q(t) = sum_j lp[j + 1] t^j (Chebyshev-node fit in t on [-1, 1])
    float lpc[LP_LONG];      // lp scaled by C1 + C1lo (host: the tile acceptance fit)
    float lp_s, lp_o;
    int lp_terms;            // one of LP_TERMS; lp[lp_terms..LP_LONG-1] are zero
    float lgc[LP_LONG];      // per-leg fit, scaled by C1 + C1lo: ln(1 + rho) = rho (1 + rho Q),
                             // Q = sum_j lgc[j + 1] / C1 x^j with x = rho (lg_terms <= LG_MONO)
                             // or x = rho lg_s + lg_o; zero beyond lg_terms
    float lg_s, lg_o;
    int lg_terms;            // one of LG_TERMS
    float rho_max;           // |rho| bound the polynomial was fitted for
    float C1, C1lo;          // tau - tau_ref = L * (C1 + C1lo) with L = R_s + R_r (constant v,
                             // tau_ref = -t0/dt) or ln(U/U_c) (linear v); C1lo = FP32 rounding
                             // error of C1
    double c0;               // -t0/dt - 1/2 (the window origin is subtracted per trace)
    // prestack time migration (KH_VEL_PSTM, the VK_PSTM kernels): the image's depth axis is the
    // two-way vertical time t0; each leg is the straight ray of the RMS velocity v_rms(t0) of
    // v(z) = v0 + pk z, T = sqrt(ze^2 + h^2) / v_rms with the equivalent depth ze = v_rms t0 / 2
    // (g.k is 0: nothing of the linear-gradient evaluation applies)
    int pstm;
    double pk;
    // radial traveltime table (KH_VEL_TABLE)
    const void* table;       // [tnh][tnz] nodes, z fastest
    int tnh, tnz;            // nodes along h and z
    int tdt;                 // storage kh_dtype: KH_F32, KH_F16, KH_U16
    float tinv;              // 1 / table_spacing
    float tunz;              // KH_F16: 1 / (tnz - 1), the normalised node depth u_j = j tunz of
                             // the per-row reference c0 + u (c1 + u c2) added to each FP16 residual
    float thmax;             // largest usable h coordinate (tnh - 1 - 1e-3)
    double tza, tsp;         // first z node (the first image depth), h spacing
    int tm;                  // depth nodes every tm image samples (1, 2 or 4)
    float tslack;            // extra window slack (samples) for the interpolation error
    // per-location first-arrival tables of a gridded model (KH_VEL_GRID, dim 2): FP32 seconds
    // [nloc][gnz][gnx] (x fastest) on the nodes (gox + i gh, j gh), read from global memory; the
    // image depth iz lies at node row gzoff + iz / tm.  gbnd: per (location, tile of the launch)
    // the smallest and largest node value over the nodes the tile's points interpolate between.
    const float* gtab;
    long long gstride;       // gnx * gnz
    int gnx, gnz, gzoff;
    double gox, gh;
    const float2* gbnd;
    int gtiles;
    float t0, dt;            // FP32 copies for the window bounds
    double t0d, dtd;         // exact values for the FP64 references
    // weight
    int weight;              // 0 one, 1 obliquity x spreading, 2 true amplitude (constant v)
    double wscale;           // 1 / (2 r0^2)
    // aperture
    int use_aperture;
    float A2;                // (float)(A*A), the exact test
    int use_taper;           // the weight tapers over the outer part of the aperture
    float ap_core, ap_core2; // radius (and its square) up to which the taper is 1
    float ap_invband;        // 1 / width of the taper band
    float aa_c;              // operator anti-aliasing: aa_spacing / (v0 dt) (constant v), aa_spacing / dt
                             // (v0 + k z, k != 0); 0 = off
    float aa_v0sq, aa_v0k, aa_kq;   // v0 + k z: v0^2, v0 k and k^2 / 4 of the legs' slowness factor
    float A2cull;            // enlarged, for the conservative tile cull
    // traces
    int nt;
    long long ld;            // row stride in elements
    int esize;               // bytes per sample
    int tdtype;              // kh_dtype of the traces (F32, F16, BF16)
    int elem_align;          // samples per 16 bytes
    int pairs;               // 1: FP32 traces staged as SamplePair rows (esize 8, ld in pairs)
    int grad;                // 1: the gradient kernel (slope rows d[i+1] - d[i], its own cache)
};

struct TileShape {
    int cx, cy, cz;          // threads along x, y, z-groups (cx*cy*cz == CONSUMERS)
    int tiles_x, tiles_y, tiles_z;
};

struct WaitCfg {
    int* status;             // device status word (bit 0: timeout)
    long long polls;         // 0 = unlimited polls (wall clock only)
    long long ns;
    // optional [3]: traces the staging warps examined and staged, and the staging warps (one per
    // CTA and work item) that reported, summed
    unsigned long long* stats = nullptr;
};

// Launchers (kh_migrate.cu).
cudaError_t launch_migrate(const GeomParams& g, const TileShape& t, const TraceSet& ts,
                           const void* traces, float* image, int vel_kind, int fast_math,
                           const WaitCfg& w, cudaStream_t s);
size_t migrate_smem_bytes(const GeomParams& g);

// One job of a batched persistent launch: its geometry (with the ln(1 + rho) fit of its tile),
// tile shape, binned headers, trace rows (16-byte aligned, row stride g.ld) and image.
struct BatchJob {
    GeomParams g;
    TileShape ts;
    TraceSet tr;
    const void* traces;
    float* image;
};

// The persistent kernel over `n_items` work items (job, tile, bin, -) taken in list order from
// the counter `*next` (zeroed before the launch).  `g_max` sizes the shared-memory ring (its
// nt is the largest of the jobs'); vel_kind/weight/fast/lg_terms/trace dtype are common to
// all jobs of the launch.  `ctas` <= 0 launches nothing: it sets the kernel's shared-memory attribute and returns
// the occupancy-sized grid through `ctas_out` (call it once before launching with that grid).
cudaError_t launch_migrate_batched(const GeomParams& g_max, const BatchJob* jobs, const int4* items,
                                   int n_items, int* next, int vel_kind, int weight, int fast,
                                   int lg_terms, int trace_dtype, const WaitCfg& w, int ctas,
                                   int* ctas_out, cudaStream_t s);
// Velocity gradient: the migration kernel in gradient mode (image as input), per-warp FP64
// partials [gridDim.y * gridDim.x * 8][2], then one fixed-order sum scaled by 1/dt.
cudaError_t launch_vgrad(const GeomParams& g, const TileShape& t, const TraceSet& tr,
                         const void* traces, const float* image, int vel_kind, int fast_math,
                         const WaitCfg& w, double* partial, cudaStream_t s);
cudaError_t launch_vgrad_reduce(const double* partial, long long n, double inv_dt, double* out,
                                cudaStream_t s);

// Demigration (kh_demigrate.cu): trace-stationary kernel over P interleaved image parts, then
// a fixed-order sum of the parts.
struct DmTile {
    int tx, ty, tz;              // tile extent in samples (tx*ty*tz <= 1024, tz <= 64)
    int tiles_x, tiles_y, tiles_z;
    int parts;                   // P
};
constexpr int DM_ROWS_HOST = 96;
cudaError_t launch_demigrate(const GeomParams& g, const DmTile& dt, const TraceSet& tr,
                             const float* image, float* partial, int* status, int max_chunks,
                             int vel_kind, int fast, cudaStream_t s);
cudaError_t launch_dm_reduce(const TraceSet& tr, int n_bins, const float* partial, int parts, int nt,
                             float* out, int ntr, cudaStream_t s);

}  // namespace kh
