// zsort.cu -- orders a chunk of galaxies by redshift shift s = ln(1+z)/dlnlam
// (counting sort on floor(s * key_scale)) and combines the per-part partial
// filter sums of the tensor-core kernel into magnitudes.
//
// Sorting is a scheduling device only: every galaxy's magnitudes are computed
// from its own row and do not depend on which rows share its tile, so the
// order within a bucket (set by atomics) does not change any result.  With the
// rows of a 128-galaxy tile close in redshift, the tile needs the filter table
// only near one shift (near-broadcast reads) and only the wavelength tiles
// that fall inside the redshifted filter band.
#include <cmath>

#include "dsps_internal.cuh"

namespace dsps {

namespace {

__device__ __forceinline__ int zkey(float z, float inv_dlnlam, float key_scale) {
    if (!(z > 0.f) || !isfinite(z)) return 0;
    int k = (int)(log1pf(z) * inv_dlnlam * key_scale);
    return min(max(k, 0), ZSORT_BUCKETS - 1);
}

__global__ void zsort_hist_kernel(const float *z, int64_t n, float inv_dlnlam, float key_scale, int *hist) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(hist + zkey(z[i], inv_dlnlam, key_scale), 1);
}

// Exclusive scan of ZSORT_BUCKETS counts in one block of 1024 threads.
__global__ void zsort_scan_kernel(int *hist) {
    constexpr int PER = ZSORT_BUCKETS / 1024;
    __shared__ int part[1024];
    const int t = threadIdx.x;
    int v[PER], s = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        v[j] = hist[t * PER + j];
        s += v[j];
    }
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int o = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += o;
        __syncthreads();
    }
    int run = part[t] - s;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        hist[t * PER + j] = run;
        run += v[j];
    }
}

__global__ void zsort_scatter_kernel(const float *z, int64_t n, float inv_dlnlam, float key_scale, int *offsets,
                                     int *perm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[atomicAdd(offsets + zkey(z[i], inv_dlnlam, key_scale), 1)] = (int)i;
}

// Sum of the parts in fixed order, then Sec. 2.2's magnitude; written to the
// galaxy's own (unsorted) row.
__global__ void combine_mags_kernel(const float *partial, int parts, int64_t n, int qs, int Q,
                                    const double *magoff, const double *offq, const int *gidx, float *mags) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t g = gidx[r];
    const double mo = magoff[r];
    for (int q = 0; q < Q; ++q) {
        float acc = 0.f;
        for (int p = 0; p < parts; ++p) acc += partial[((int64_t)p * n + r) * qs + q];
        mags[g * Q + q] = (float)(-2.5 * log10((double)acc) + mo + offq[q]);
    }
}

}  // namespace

float zsort_key_scale(const Ctx &c) {
    const double smax = std::log1p(c.opts.z_max) / c.dlnlam;
    return (float)(ZSORT_BUCKETS / (smax + 1.0));
}

cudaError_t launch_zsort(const Ctx &c, const Workspace &w, const float *z, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const float inv_d = (float)(1.0 / c.dlnlam), ks = zsort_key_scale(c);
    cudaError_t e = cudaMemsetAsync(w.hist, 0, ZSORT_BUCKETS * sizeof(int), s);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    zsort_hist_kernel<<<blocks, 256, 0, s>>>(z, n, inv_d, ks, w.hist);
    zsort_scan_kernel<<<1, 1024, 0, s>>>(w.hist);
    zsort_scatter_kernel<<<blocks, 256, 0, s>>>(z, n, inv_d, ks, w.hist, w.perm);
    return cudaGetLastError();
}

cudaError_t launch_combine(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, int parts, float *mags,
                           cudaStream_t s) {
    (void)c;
    if (n <= 0) return cudaSuccess;
    combine_mags_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w.partial, parts, n, 4 * fs.Q4, fs.Q,
                                                                      w.magoff, fs.d_offq, w.gidx, mags);
    return cudaGetLastError();
}

}  // namespace dsps
