// Binning sort of the traces (step before Eq. 1's sum): each trace gets its offset bin (the
// delta(X - |x_s - x_r|) of Eq. 1) and the cell of its midpoint on a coarse grid, and the
// traces are put in (bin, cell row, cell column, original index) order by a stable LSD radix
// sort over all SMs.  The (bin, cell) start table then lets a CTA of the migration walk only
// the cells that meet its tile's aperture disc (the traces near enough to carry the tile's
// reflections, Sec. 3 after Eq. 2) instead of its whole bin, so the staging work per CTA stays proportional to the
// traces it can use as surveys grow to tens of millions of traces (Sec. 2).
//
// Passes (each a few launches, no host synchronisation, no atomics on values, so the order is
// the same on every run):
//   k_cell_key      key = bin * ncell + cell, value = original index (dropped: key = nkeys)
//   k_radix_hist    per block of 4096 items, the counts of one 8-bit digit
//   k_radix_scan    exclusive scan of the counts, digit-major (one CTA)
//   k_radix_scatter stable scatter: items in index order, ranked per warp with match.any
//   k_key_starts    first sorted position of every key, and of every bin
#include "kh_device.cuh"
#include "kh_plan.h"

namespace kh {

constexpr int RX_THREADS = 256;
constexpr int RX_ROUNDS = 16;
constexpr int RX_ITEMS = RX_THREADS * RX_ROUNDS;   // items per block
constexpr int RX_SCAN_THREADS = 1024;

int sort_hist_entries(int ntr) { return 256 * ((ntr + RX_ITEMS - 1) / RX_ITEMS); }

// Offset bin (FP64, as every kernel decides it) and midpoint cell (FP64 of the FP32 midpoint
// the aperture test uses).  Traces with no bin or a midpoint outside the grid get key nkeys.
__global__ void k_cell_key(int ntr, const float* __restrict__ sx, const float* __restrict__ sy,
                           const float* __restrict__ rx, const float* __restrict__ ry, int dim, int n_bins,
                           double w, CellGrid cg, int* __restrict__ key, int* __restrict__ val)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ntr) return;
    const int ncell = cg.ncx * cg.ncy;
    const float a = sx[j], c = rx[j];
    const float b = (dim == 3 && sy) ? sy[j] : 0.f, d = (dim == 3 && ry) ? ry[j] : 0.f;
    const int bin = offset_bin(a, b, c, d, n_bins, w);
    int k = n_bins * ncell;
    if (bin >= 0) {
        int cx = 0, cy = 0;
        if (cg.margin > 0.0) {
            const float mx = __fmul_rn(__fadd_rn(a, c), 0.5f), my = __fmul_rn(__fadd_rn(b, d), 0.5f);
            const double fx = floor(__dmul_rn(__dadd_rn((double)mx, -cg.gx0), cg.inv_cs));
            const double fy = (dim == 3) ? floor(__dmul_rn(__dadd_rn((double)my, -cg.gy0), cg.inv_cs)) : 0.0;
            const bool in_grid = fx >= 0.0 && fx < (double)cg.ncx && fy >= 0.0 && fy < (double)cg.ncy;
            if (in_grid) {
                cx = (int)fx;
                cy = (int)fy;
                k = bin * ncell + cy * cg.ncx + cx;
            }
        } else {
            k = bin * ncell;
        }
    }
    key[j] = k;
    val[j] = j;
}

__global__ void __launch_bounds__(RX_THREADS) k_radix_hist(int n, const int* __restrict__ key, int shift,
                                                           int* __restrict__ hist, int nblocks)
{
    __shared__ int cnt[256];
    const int tid = threadIdx.x;
    cnt[tid] = 0;
    __syncthreads();
    const int base = blockIdx.x * RX_ITEMS;
    for (int r = 0; r < RX_ROUNDS; ++r) {
        const int i = base + r * RX_THREADS + tid;
        if (i < n) atomicAdd(&cnt[(key[i] >> shift) & 255], 1);
    }
    __syncthreads();
    hist[tid * nblocks + blockIdx.x] = cnt[tid];
}

// Exclusive scan of `n` counts in place, one CTA: each thread sums a contiguous chunk, the
// chunk sums are scanned in shared memory, then each thread rewrites its chunk.
__global__ void __launch_bounds__(RX_SCAN_THREADS) k_radix_scan(int* __restrict__ a, int n)
{
    __shared__ int part[RX_SCAN_THREADS];
    const int tid = threadIdx.x;
    const int chunk = (n + RX_SCAN_THREADS - 1) / RX_SCAN_THREADS;
    const int lo = min(n, tid * chunk), hi = min(n, lo + chunk);
    int sum = 0;
    for (int i = lo; i < hi; ++i) sum += a[i];
    part[tid] = sum;
    __syncthreads();
    for (int o = 1; o < RX_SCAN_THREADS; o <<= 1) {   // Hillis-Steele inclusive scan
        const int v = tid >= o ? part[tid - o] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int run = part[tid] - sum;
    for (int i = lo; i < hi; ++i) {
        const int c = a[i];
        a[i] = run;
        run += c;
    }
}

// Stable scatter of one digit: the block's items in index order, 256 per round; within a warp
// the items of equal digit are ranked by lane (match.any), across warps by warp order.
__global__ void __launch_bounds__(RX_THREADS)
    k_radix_scatter(int n, const int* __restrict__ kin, const int* __restrict__ vin, int* __restrict__ kout,
                    int* __restrict__ vout, int shift, const int* __restrict__ offs, int nblocks)
{
    constexpr int WARPS = RX_THREADS / 32;
    __shared__ int base[256];
    __shared__ int wcnt[WARPS][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = offs[tid * nblocks + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RX_ROUNDS; ++r) {
        const int i = blockIdx.x * RX_ITEMS + r * RX_THREADS + tid;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const bool valid = i < n;
        const int k = valid ? kin[i] : 0;
        const int d = valid ? (k >> shift) & 255 : 256;
        const unsigned same = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(same & lt);
        if (valid && rank == 0) wcnt[warp][d] = __popc(same);
        __syncthreads();
        int run = 0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) {
            const int c = wcnt[w][tid];
            wcnt[w][tid] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            const int pos = base[d] + wcnt[warp][d] + rank;
            kout[pos] = k;
            vout[pos] = vin[i];
        }
        __syncthreads();
        base[tid] += run;
    }
}

// start[k] = first sorted position whose key is >= k, for k = 0 .. nkeys (start[nkeys] = number
// of kept traces); bin_start[b] = start[b * ncell].
__global__ void k_key_starts(int n, const int* __restrict__ key, int nkeys, int ncell, int* __restrict__ start,
                             int* __restrict__ bin_start)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
        const int prev = i == 0 ? -1 : min(key[i - 1], nkeys);
        const int cur = i == n ? nkeys : min(key[i], nkeys);
        for (int k = prev + 1; k <= cur; ++k) {
            start[k] = i;
            if (k % ncell == 0) bin_start[k / ncell] = i;
        }
    }
}

cudaError_t sort_traces(int ntr, const float* sx, const float* sy, const float* rx, const float* ry,
                        int dim, int n_bins, double bin_width, const CellGrid& cg, int* key_a,
                        int* key_b, int* val_a, int* val_b, int* hist, int* cell_start, int* bin_start,
                        const int** perm_out, int* launches, cudaStream_t s)
{
    const int ncell = cg.ncx * cg.ncy;
    const int nkeys = n_bins * ncell;
    int bits = 1;
    while ((1LL << bits) <= (long long)nkeys) ++bits;   // keys are 0 .. nkeys
    const int passes = (bits + 7) / 8;
    const int nblocks = (ntr + RX_ITEMS - 1) / RX_ITEMS;
    int *kin = key_a, *kout = key_b, *vin = val_a, *vout = val_b;
    if (ntr > 0) {
        k_cell_key<<<(ntr + 255) / 256, 256, 0, s>>>(ntr, sx, sy, rx, ry, dim, n_bins, bin_width, cg, kin, vin);
        ++*launches;
        for (int p = 0; p < passes; ++p) {
            k_radix_hist<<<nblocks, RX_THREADS, 0, s>>>(ntr, kin, 8 * p, hist, nblocks);
            k_radix_scan<<<1, RX_SCAN_THREADS, 0, s>>>(hist, 256 * nblocks);
            k_radix_scatter<<<nblocks, RX_THREADS, 0, s>>>(ntr, kin, vin, kout, vout, 8 * p, hist, nblocks);
            *launches += 3;
            int* t = kin;
            kin = kout;
            kout = t;
            t = vin;
            vin = vout;
            vout = t;
        }
    }
    const int blocks = std::max(1, std::min((ntr + 256) / 256, 4096));
    k_key_starts<<<blocks, 256, 0, s>>>(ntr, kin, nkeys, ncell, cell_start, bin_start);
    ++*launches;
    *perm_out = vin;
    return cudaGetLastError();
}

}  // namespace kh
