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

// Default wait limit: polls of mbarrier.try_wait, each checked against a 2 s wall clock.
constexpr long long WAIT_NS = 2000000000LL;

enum VelKind { VK_CONST = 0, VK_LINEAR = 1, VK_TABLE = 2 };

// Sorted trace set produced by the binning pass (plan workspace).
struct TraceSet {
    const float4* hdr;      // (sx, sy, rx, ry) in bin order
    const float2* mid;      // FP32 midpoints (sx + rx) * 0.5f, (sy + ry) * 0.5f
    const int* perm;        // original trace index
    const int* bin_start;   // [n_bins + 1]
};

// Everything a migration-type kernel needs, passed by value.
struct GeomParams {
    int dim, nx, ny, nz, n_bins;
    double ox, oy, oz, dx, dy, dz;
    float fdz;
    // velocity (FP32 constants for the hot loop, FP64 for per-z set-up)
    double v0, k;            // k already |k| for the hot loop's log form
    double kabs;
    float C1, C0h;           // tau - 1/2 = L * C1 + C0h (L = R_s+R_r or log2 U)
    float t0, dt;
    // weight
    int weight;              // 0 one, 1 obliquity x spreading
    double wscale;           // 1 / (2 r0^2)
    // aperture
    int use_aperture;
    float A2;                // (float)(A*A), the exact test
    float A2cull;            // enlarged, for the conservative tile cull
    // traces
    int nt;
    long long ld;            // row stride in elements
    int esize;               // bytes per sample
    int elem_align;          // samples per 16 bytes
};

struct TileShape {
    int cx, cy, cz;          // threads along x, y, z-groups (cx*cy*cz == CONSUMERS)
    int tiles_x, tiles_y, tiles_z;
};

struct WaitCfg {
    int* status;             // device status word (bit 0: timeout)
    long long polls;         // 0 = unlimited polls (wall clock only)
    long long ns;
};

// Launchers (kh_migrate.cu).
cudaError_t launch_migrate(const GeomParams& g, const TileShape& t, const TraceSet& ts,
                           const void* traces, float* image, int vel_kind, int fast_math,
                           const WaitCfg& w, cudaStream_t s);
size_t migrate_smem_bytes(const GeomParams& g);

}  // namespace kh
