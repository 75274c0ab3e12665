// histogram.cu -- the population statistic of the paper's benchmark (Sec. 5.1:
// a colour cut selecting red galaxies, then a histogram of their r-band
// magnitude), over magnitudes on the device.  The same binning (hist_bin in
// epilogue.cuh) runs fused in the tensor-core path's combine kernel.
#include <cmath>

#include "dsps_internal.cuh"
#include "epilogue.cuh"

namespace dsps {

void set_last_error(const char *msg);

namespace {

// Grid-stride over galaxies; per-block counts in shared memory, flushed with
// one global atomic per non-empty bin.
__global__ void __launch_bounds__(256) hist_kernel(const float *mags, int64_t n, int Q, HistArgs h) {
    extern __shared__ unsigned int sh[];
    for (int b = threadIdx.x; b < h.n_bins; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const float *m = mags + g * Q;
        int bin;
        if (hist_bin(h, m[h.band_a], m[h.band_b], m[h.band_r], bin)) atomicAdd(sh + bin, 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < h.n_bins; b += blockDim.x)
        if (sh[b]) atomicAdd(h.counts + b, (unsigned long long)sh[b]);
}

}  // namespace

int make_hist_args(const dsps_hist_spec *spec, int n_filt, unsigned long long *counts, HistArgs *out) {
    if (!spec || !counts) {
        set_last_error("histogram: null argument");
        return DSPS_ERR_INVALID_ARG;
    }
    const dsps_hist_spec &s = *spec;
    if (s.band_a < 0 || s.band_a >= n_filt || s.band_b < 0 || s.band_b >= n_filt || s.band_r < 0 ||
        s.band_r >= n_filt || s.n_bins < 1 || s.n_bins > DSPS_MAX_HIST_BINS || !std::isfinite(s.lo) ||
        !std::isfinite(s.hi) || !(s.lo < s.hi) || std::isnan(s.cut)) {
        set_last_error("histogram: bad specification");
        return DSPS_ERR_INVALID_ARG;
    }
    HistArgs h;
    h.band_a = s.band_a;
    h.band_b = s.band_b;
    h.band_r = s.band_r;
    h.n_bins = s.n_bins;
    h.cut = s.cut;
    h.lo = s.lo;
    h.hi = s.hi;
    h.scale = (float)((double)s.n_bins / ((double)s.hi - (double)s.lo));
    h.counts = counts;
    *out = h;
    return DSPS_OK;
}

cudaError_t launch_histogram(const float *mags, int64_t n, int Q, const HistArgs &h, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want < 1024 ? want : 1024);
    hist_kernel<<<blocks, 256, (size_t)h.n_bins * sizeof(unsigned int), s>>>(mags, n, Q, h);
    return cudaGetLastError();
}

}  // namespace dsps
