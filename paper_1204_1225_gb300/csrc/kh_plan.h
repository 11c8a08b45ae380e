// The opaque plan behind kh_plan: the descriptor, options and the device workspace it owns.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "kh_internal.h"

struct kh_plan_s {
    kh_desc d;
    int device = 0;
    long long launches = 0;
    long long wait_polls = 0;     // 0 = wall-clock limit only
    int fast_math = 1;
    long long tile_code = 0;      // 0 = default tile for the dimension
    int batch_mode = 0;           // KH_OPT_BATCH_MODE (read from the first job's plan)
    int sample_pairs = 1;         // KH_OPT_SAMPLE_PAIRS
    // device workspace (grown on demand, freed by kirchhoff_destroy)
    int* ws_status = nullptr;     // [2]: bit 0 of [0] = a bounded wait ran out
    int* ws_bin_start = nullptr;  // [MAX_BINS + 1]
    int* ws_bin = nullptr;
    size_t cap_bin = 0;
    int* ws_perm = nullptr;
    size_t cap_perm = 0;
    float4* ws_hdr = nullptr;
    size_t cap_hdr = 0;
    float2* ws_mid = nullptr;
    size_t cap_mid = 0;
    // the binning sort: keys and values (ping-pong), per-block digit counts, (bin, cell) starts
    int* ws_key2 = nullptr;
    size_t cap_key2 = 0;
    int* ws_perm2 = nullptr;
    size_t cap_perm2 = 0;
    int* ws_hist = nullptr;
    size_t cap_hist = 0;
    int* ws_cell_start = nullptr;
    size_t cap_cell_start = 0;
    const int* cur_perm = nullptr;    // the buffer holding the last sort's permutation
    kh::CellGrid cur_cg{};            // and its cell grid
    int spatial_sort = 1;             // KH_OPT_SPATIAL_SORT
    unsigned long long* ws_stats = nullptr;   // [3] staging statistics (while profiling)
    double* ws_semb = nullptr;    // velocity analysis: block partials and (V, D, B)
    unsigned char* ws_pad = nullptr;
    size_t cap_pad = 0;
    long long* ws_count = nullptr;
    size_t cap_count = 0;
    double* ws_partial = nullptr;
    size_t cap_partial = 0;
    float* ws_dm = nullptr;       // demigration partial traces [P][ntr][nt]
    size_t cap_dm = 0;
    // radial traveltime table (KH_VEL_TABLE), rebuilt when a call needs a wider h range
    unsigned char* ws_tab = nullptr;
    size_t cap_tab = 0;
    double* ws_tab64 = nullptr;
    size_t cap_tab64 = 0;
    double* ws_tmm = nullptr;     // [2] table min / max
    unsigned* ws_hmax = nullptr;  // [1] largest horizontal distance (float bits)
    int tab_nh = 0, tab_nz = 0;
    double tab_tmin = 0.0, tab_scale = 1.0;
    // gridded model (KH_VEL_GRID): the node grid, per-location FP32 tables, the locations, the
    // rounds each took, the FP64 slowness s and h s, and per (location, tile) time bounds
    kh_grid grid{};
    int grid_nloc = 0;
    int grid_m = 0;               // depth nodes every grid_m image samples
    int grid_zoff = 0;            // node row of the first image depth
    float* ws_gtab = nullptr;
    size_t cap_gtab = 0;
    float* ws_gloc = nullptr;
    size_t cap_gloc = 0;
    int* ws_grounds = nullptr;
    size_t cap_grounds = 0;
    double* ws_gslow = nullptr;
    size_t cap_gslow = 0;
    float2* ws_gbnd = nullptr;
    size_t cap_gbnd = 0;
    // profiling: event pairs recorded around main kernels while enabled
    int profiling = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_open;
    // host-resident migration (kirchhoff_migrate_host): two slots of device headers ([4][cap_ntr]:
    // sx, sy, rx, ry), traces and image used in turn, a copy stream per direction, and per slot
    // the events of its last inputs-in, migration and image-out
    struct HostSlot {
        float* hdr = nullptr;
        unsigned char* traces = nullptr;
        float* image = nullptr;
        size_t cap_ntr = 0, cap_tr = 0;
        cudaEvent_t in_done = nullptr, mig_done = nullptr, out_done = nullptr;
        bool used = false;
    } host[2];
    cudaStream_t host_in = nullptr, host_out = nullptr;
    int host_next = 0;
};

namespace kh {
kh_status set_error(kh_status s, const char* msg);
kh_status set_cuda_error(cudaError_t e, const char* what);
kh_status ensure_traces_ws(kh_plan_s* p, int ntr);
// Frees the host-resident migration's slots, streams and events (kirchhoff_destroy).
void host_release(kh_plan_s* p);
// Offset bin and midpoint cell per trace, stable multi-CTA radix sort by (bin, cell), the
// (bin, cell) starts and the sorted headers.  `spatial` = false sorts by bin alone (one cell
// per bin; midpoints that reach no column are still dropped).  Sets p->cur_perm, p->cur_cg.
kh_status bin_traces(kh_plan_s* p, int ntr, const float* sx, const float* sy, const float* rx,
                     const float* ry, cudaStream_t s, bool spatial = true);
// The sorted trace set of the last bin_traces call.
TraceSet plan_traces(const kh_plan_s* p);
// Cell grid of a descriptor: one cell with no aperture, else cells of about half the aperture
// (at most 64 per axis) over the image columns widened by the aperture margin.
CellGrid cell_grid_of(const kh_desc& d, bool spatial);
// The radix sort (kh_sort.cu): keys[i] = bin * ncell + cell (n_bins * ncell = no bin or out of
// the grid), vals[i] = i; then stable passes of 8 bits; then the key starts.  Writes the sorted
// permutation into *perm_out (one of the two value buffers) and the starts into cell_start
// [n_bins * ncell + 1] and bin_start [n_bins + 1].
cudaError_t sort_traces(int ntr, const float* sx, const float* sy, const float* rx, const float* ry,
                        int dim, int n_bins, double bin_width, const CellGrid& cg, int* key_a,
                        int* key_b, int* val_a, int* val_b, int* hist, int* cell_start, int* bin_start,
                        const int** perm_out, int* launches, cudaStream_t s);
int sort_hist_entries(int ntr);
// Sorted headers and FP32 midpoints of the first bin_start[n_bins] sorted traces.
cudaError_t launch_gather(int ntr, const int* bin_start, int n_bins, const int* perm, const float* sx,
                          const float* sy, const float* rx, const float* ry, int dim, float4* hdr, float2* mid,
                          cudaStream_t s);
// Brackets a main-kernel launch with profiling events (no-op unless profiling is on).
void prof_begin(kh_plan_s* p, cudaStream_t s);
void prof_end(kh_plan_s* p, cudaStream_t s);
kh_status staged_traces(kh_plan_s* p, int ntr, const void* traces, cudaStream_t s,
                        const void** out, long long* ld);
// Allocation-free path: validation, geometry and tile of a descriptor; binning launches into
// caller-supplied device buffers (bin_start holds n_bins + 1 entries).
kh_status noalloc_prepare(const kh_desc* d, GeomParams* g, TileShape* t);
// Batched launch: a plan's geometry, tile (its KH_OPT_TILE, else the default) and v(z) fit;
// header checks; the row-padding copy of staged_traces into a caller-supplied buffer.
kh_status plan_geometry(const kh_plan_s* p, GeomParams* g, TileShape* t);
kh_status plan_check_headers(const kh_plan_s* p, int ntr, const float* sx, const float* sy,
                             const float* rx, const float* ry);
cudaError_t launch_pad(int ntr, int nt, long long ld, int esize, const void* src, void* dst, cudaStream_t s);
// FP32 rows of nt samples to SamplePair rows of ld (even) pairs.
cudaError_t launch_pairs(int ntr, int nt, int ld, const void* src, void* dst, cudaStream_t s);
// KH_VEL_GRID migration: location indices of the sorted traces and the tile bounds of the
// launch's tiling; fills the table fields of g.
kh_status grid_prepare(kh_plan_s* p, const TileShape& t, GeomParams& g, cudaStream_t s);
cudaError_t noalloc_bin(int ntr, const float* sx, const float* sy, const float* rx, const float* ry,
                        const kh_desc& d, int* bin, int* perm, int* bin_start, float4* hdr,
                        float2* mid, cudaStream_t s);
}  // namespace kh
