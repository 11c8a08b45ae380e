// Velocity analysis (Sec. 2): migrating with an estimate of the velocity gives redundant images
// of the same reflectors, one per offset bin here; the differences between them measure the
// error of the velocity model, which is corrected and the data migrated again until they agree
// and can be stacked.  The measure is the normalised variance of the weighted offset images
// across the N bins that hold traces,
//     V = sum_b ||w_b I_b - m||^2 / sum_b ||w_b I_b||^2,   m = (1/N) sum_b w_b I_b,
// with w_b = 1 / (traces of bin b) by default, and its image gradient
//     dV/dI_b = (2 w_b / B) ((w_b I_b - m) - V w_b I_b),   B = sum_b ||w_b I_b||^2,
// which the velocity-gradient kernel turns into dV/d(v0, k) = d<dV/dI, L(v0, k) D>/d(v0, k).
//
// Three launches, HBM-bound: per-block FP64 partial sums of D and B over a fixed grid (each
// thread reads one point of every bin: coalesced rows), one fixed-order sum, and the gradient
// image; the result does not depend on the run.
#include <cmath>
#include <vector>

#include "kh_device.cuh"
#include "kh_plan.h"

namespace kh {

constexpr int SEMB_BLOCKS = 1024;
constexpr int SEMB_THREADS = 256;

struct SembArgs {
    int n_bins;
    long long npts;           // image samples per bin
    double inv_n;             // 1 / (bins with traces)
    double w[MAX_BIN_WEIGHTS];
};

__global__ void __launch_bounds__(SEMB_THREADS)
    k_semb_partial(const float* __restrict__ img, SembArgs a, double* __restrict__ part)
{
    __shared__ double sd[SEMB_THREADS], sb[SEMB_THREADS];
    double d = 0.0, bb = 0.0;
    for (long long x = blockIdx.x * (long long)SEMB_THREADS + threadIdx.x; x < a.npts;
         x += (long long)SEMB_BLOCKS * SEMB_THREADS) {
        double s = 0.0;
        for (int b = 0; b < a.n_bins; ++b)
            if (a.w[b] > 0.0) s += a.w[b] * (double)img[b * a.npts + x];
        const double m = s * a.inv_n;
        for (int b = 0; b < a.n_bins; ++b) {
            if (a.w[b] <= 0.0) continue;
            const double v = a.w[b] * (double)img[b * a.npts + x];
            d += (v - m) * (v - m);
            bb += v * v;
        }
    }
    sd[threadIdx.x] = d;
    sb[threadIdx.x] = bb;
    __syncthreads();
    for (int o = SEMB_THREADS / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sd[threadIdx.x] += sd[threadIdx.x + o];
            sb[threadIdx.x] += sb[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sd[0];
        part[2 * blockIdx.x + 1] = sb[0];
    }
}

// out = (V, D, B), the block partials summed in block order by one thread
__global__ void k_semb_reduce(const double* __restrict__ part, double* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double d = 0.0, b = 0.0;
    for (int i = 0; i < SEMB_BLOCKS; ++i) {
        d += part[2 * i];
        b += part[2 * i + 1];
    }
    out[0] = b > 0.0 ? d / b : 0.0;
    out[1] = d;
    out[2] = b;
}

__global__ void __launch_bounds__(SEMB_THREADS)
    k_semb_grad(const float* __restrict__ img, SembArgs a, const double* __restrict__ vdb,
                float* __restrict__ grad)
{
    const double V = vdb[0], B = vdb[2];
    const double c = B > 0.0 ? 2.0 / B : 0.0;
    for (long long x = blockIdx.x * (long long)SEMB_THREADS + threadIdx.x; x < a.npts;
         x += (long long)SEMB_BLOCKS * SEMB_THREADS) {
        double s = 0.0;
        for (int b = 0; b < a.n_bins; ++b)
            if (a.w[b] > 0.0) s += a.w[b] * (double)img[b * a.npts + x];
        const double m = s * a.inv_n;
        for (int b = 0; b < a.n_bins; ++b) {
            const double w = a.w[b];
            float g = 0.f;
            if (w > 0.0) {
                const double v = w * (double)img[b * a.npts + x];
                g = (float)(c * w * ((v - m) - V * v));
            }
            grad[b * a.npts + x] = g;
        }
    }
}

}  // namespace kh

using namespace kh;

extern "C" kh_status kirchhoff_semblance(kh_plan p, const float* image, const double* bin_weight,
                                         double* out, float* grad_image, void* cuda_stream)
{
    if (!p || !image || !out) return set_error(KH_ERR_INVALID_ARG, "kirchhoff_semblance: NULL argument");
    const kh_desc& d = p->d;
    if (d.n_bins > MAX_BIN_WEIGHTS)
        return set_error(KH_ERR_UNSUPPORTED, "kirchhoff_semblance: more offset bins than the kernel's weights");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    SembArgs a;
    a.n_bins = d.n_bins;
    a.npts = (long long)d.ny * d.nx * d.nz;
    std::vector<double> w(d.n_bins, 0.0);
    cudaError_t e = cudaSuccess;
    if (bin_weight) {
        for (int b = 0; b < d.n_bins; ++b) {
            if (!(bin_weight[b] >= 0.0) || !std::isfinite(bin_weight[b]))
                return set_error(KH_ERR_INVALID_ARG, "kirchhoff_semblance: bin weights must be finite and >= 0");
            w[b] = bin_weight[b];
        }
    } else {
        if (!p->cur_perm)
            return set_error(KH_ERR_INVALID_ARG, "kirchhoff_semblance: no bin weights and no migration of this "
                                                 "plan to count the traces per bin from");
        std::vector<int> bs(d.n_bins + 1);
        e = cudaMemcpyAsync(bs.data(), p->ws_bin_start, sizeof(int) * (d.n_bins + 1), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_semblance: bin counts");
        for (int b = 0; b < d.n_bins; ++b) {
            const int n = bs[b + 1] - bs[b];
            w[b] = n > 0 ? 1.0 / n : 0.0;
        }
    }
    int used = 0;
    for (int b = 0; b < MAX_BIN_WEIGHTS; ++b) {
        a.w[b] = b < d.n_bins ? w[b] : 0.0;
        used += (b < d.n_bins && w[b] > 0.0) ? 1 : 0;
    }
    if (used == 0) return set_error(KH_ERR_INVALID_ARG, "kirchhoff_semblance: every bin weight is zero");
    a.inv_n = 1.0 / used;
    if (!p->ws_semb) {
        e = cudaMalloc(reinterpret_cast<void**>(&p->ws_semb), (2 * SEMB_BLOCKS + 3) * sizeof(double));
        if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_semblance: workspace");
    }
    double* part = p->ws_semb;
    double* res = p->ws_semb + 2 * SEMB_BLOCKS;
    k_semb_partial<<<SEMB_BLOCKS, SEMB_THREADS, 0, s>>>(image, a, part);
    k_semb_reduce<<<1, 32, 0, s>>>(part, res);
    p->launches += 2;
    if (grad_image) {
        k_semb_grad<<<SEMB_BLOCKS, SEMB_THREADS, 0, s>>>(image, a, res, grad_image);
        ++p->launches;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_cuda_error(e, "kirchhoff_semblance");
    return KH_OK;
}
