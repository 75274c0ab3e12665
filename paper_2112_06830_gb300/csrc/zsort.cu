// zsort.cu -- orders a chunk of galaxies for the tensor-core kernel (counting
// sort on a two-level key) and combines that kernel's per-part partial filter
// sums into magnitudes.
//
// Key: ZSORT_ZBINS coarse bins of the redshift shift s = ln(1+z)/dlnlam, and
// inside each ZSORT_MUBINS bins of the galaxy's mean metallicity at the middle
// log age.  Rows of one 128-galaxy tile then share a narrow redshift range (the
// tile needs only the wavelength tiles inside the redshifted filter band) and a
// narrow metallicity range (the tile's non-zero weights fill only the K blocks
// of a few metallicity bins).  With a nebular axis the inner key is 8 bins of
// the mean log U times 16 metallicity bins, so that a tile also spans few log U
// sections.  A last pass orders the rows inside each tile by
// redshift, so that the 32 rows of one epilogue warp read the filter table at
// nearby shifts.
// Sorting is a scheduling device only: every galaxy's magnitudes come from its
// own row, and skipped tiles and blocks hold exact zeros for every row, so the
// order within a bucket (set by atomics) changes no result.
#include <climits>
#include <cmath>

#include "dsps_internal.cuh"
#include "epilogue.cuh"

namespace dsps {

namespace {

struct SortKey {
    const float *z, *mu, *slope;   // parameter rows 11, 5, 7 of the chunk
    float inv_dlnlam, zscale;      // s = log1p(z) * inv_dlnlam; z bin = floor(s * zscale)
    float mu_lo, mu_scale;         // mu bin = floor((mua p5 + mub p7 - mu_lo) * mu_scale)
    float mua, mub;                // MDF mean at the middle log age
    const float *um;               // parameter row 12 (nebular axis), or nullptr
    float u_lo, u_scale;           // u bin = floor((u_mean - u_lo) * u_scale), 8 bins
    const float *us;               // parameter row 13 (u_sigma), with um
    const float *uedge;            // [n_u + 1] log U bin edges (+-1e30 outer)
    int n_u;
    int2 *urange;                  // tiles' log U section ranges to preset, or nullptr
};

__device__ __forceinline__ int sort_key(const SortKey &k, int64_t i) {
    const float z = k.z[i];
    int zb = 0;
    if (z > 0.f && isfinite(z)) zb = min(max((int)(log1pf(z) * k.inv_dlnlam * k.zscale), 0), ZSORT_ZBINS - 1);
    const float m = fmaf(k.slope[i], k.mub, k.mua * k.mu[i]);
    int mb = 0;
    if (isfinite(m)) mb = (int)fminf(fmaxf((m - k.mu_lo) * k.mu_scale, 0.f), (float)(ZSORT_MUBINS - 1));
    if (k.um) {
        constexpr int UB = 8, MB = ZSORT_MUBINS / UB;
        const float u = k.um[i];
        int ub = 0;
        if (isfinite(u)) ub = (int)fminf(fmaxf((u - k.u_lo) * k.u_scale, 0.f), (float)(UB - 1));
        mb = ub * MB + mb / UB;
    }
    return zb * ZSORT_MUBINS + mb;
}

// Histogram of the keys; the first threads also reset the per-tile ranges
// and block masks.
__global__ void zsort_hist_kernel(SortKey k, int64_t n, int *hist, int2 *trange, int2 *urange, int n_u,
                                  unsigned *kmask, int n_tiles, int kmw) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_tiles) {
        trange[i] = make_int2(TRANGE_EMPTY_LO, TRANGE_EMPTY_HI);
        urange[i] = make_int2(n_u, -1);
        for (int w = 0; w < kmw; ++w) kmask[i * kmw + w] = 0u;
    }
    if (i < n) atomicAdd(hist + sort_key(k, i), 1);
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

__global__ void zsort_scatter_kernel(SortKey k, int64_t n, int *offsets, int *perm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[atomicAdd(offsets + sort_key(k, i), 1)] = (int)i;
}

// Orders the rows of each 128-row tile by redshift (rank sort in one block per
// tile; ties by position), leaving the tile's set of galaxies unchanged.
__global__ void __launch_bounds__(128) zsort_tile_kernel(SortKey k, int64_t n, int *perm) {
    __shared__ float key[128];
    __shared__ int idx[128];
    const int64_t r0 = (int64_t)blockIdx.x * 128;
    const int t = threadIdx.x;
    const int rows = (int)min((int64_t)128, n - r0);
    __shared__ int ulo, uhi;
    if (t == 0) {
        ulo = k.n_u;
        uhi = -1;
    }
    __syncthreads();
    if (t < rows) {
        idx[t] = perm[r0 + t];
        const float z = k.z[idx[t]];
        key[t] = z > 0.f && isfinite(z) ? z : 0.f;
        if (k.urange) {
            // the log U bins a row can weight (Sec. 3.3, Eq. nebsed: the
            // triweight CDF differences vanish for a bin wholly beyond +-3
            // widths), widened by 1e-3 width against rounding: a superset of
            // the bins the weights kernel finds non-zero
            const float um = k.um[idx[t]], us = k.us[idx[t]];
            if (us > 0.f && isfinite(um) && isfinite(us)) {
                const float isu = 1.f / us;
                int lo = k.n_u, hi = -1;
                for (int b = 0; b < k.n_u; ++b) {
                    const float xl = b == 0 ? -1e30f : (__ldg(k.uedge + b) - um) * isu;
                    const float xh = b == k.n_u - 1 ? 1e30f : (__ldg(k.uedge + b + 1) - um) * isu;
                    if (xl < 3.001f && xh > -3.001f) {
                        lo = min(lo, b);
                        hi = b;
                    }
                }
                if (hi >= lo) {
                    atomicMin(&ulo, lo);
                    atomicMax(&uhi, hi);
                }
            }
        }
    }
    __syncthreads();
    if (k.urange && t == 0) k.urange[blockIdx.x] = make_int2(ulo, uhi);
    if (t < rows) {
        const float kt = key[t];
        int rank = 0;
        for (int j = 0; j < rows; ++j) {
            const float kj = key[j];
            rank += (kj < kt) || (kj == kt && j < t);
        }
        perm[r0 + rank] = idx[t];
    }
}

// Sum of the parts in fixed order, then Sec. 2.2's magnitude (ab_mag),
// written to the galaxy's own (unsorted) row.
template <int Q4>
__global__ void combine_mags_kernel(const float *partial, int parts, int64_t n, int Q, const float *magoff,
                                    const float *offq, const int *gidx, float *mags, HistArgs h) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float acc[4 * Q4];
#pragma unroll
    for (int q = 0; q < 4 * Q4; ++q) acc[q] = 0.f;
    for (int p = 0; p < parts; ++p) {
        const float4 *src = reinterpret_cast<const float4 *>(partial + ((int64_t)p * n + r) * (4 * Q4));
#pragma unroll
        for (int qq = 0; qq < Q4; ++qq) {
            const float4 v = src[qq];
            acc[4 * qq] += v.x;
            acc[4 * qq + 1] += v.y;
            acc[4 * qq + 2] += v.z;
            acc[4 * qq + 3] += v.w;
        }
    }
    const int64_t g = gidx[r];
    const float mo = magoff[r];
    float m[4 * Q4];
#pragma unroll
    for (int q = 0; q < 4 * Q4; ++q) m[q] = q < Q ? ab_mag(acc[q], mo, offq[q]) : 0.f;
    if (h.counts) {
        int bin;
        if (hist_bin(h, m[h.band_a], m[h.band_b], m[h.band_r], bin)) atomicAdd(h.counts + bin, 1ull);
    }
    if (!mags) return;
    float *dst = mags + g * Q;
    if (Q == 4 * Q4) {
#pragma unroll
        for (int qq = 0; qq < Q4; ++qq)
            reinterpret_cast<float4 *>(dst)[qq] = make_float4(m[4 * qq], m[4 * qq + 1], m[4 * qq + 2], m[4 * qq + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < 4 * Q4; ++q)
            if (q < Q) dst[q] = m[q];
    }
}

}  // namespace

cudaError_t launch_zsort(const Ctx &c, const Workspace &w, const float *params, int64_t G_stride, int64_t g_begin,
                         int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    SortKey k;
    k.z = params + 11 * G_stride + g_begin;
    k.mu = params + 5 * G_stride + g_begin;
    k.slope = params + 7 * G_stride + g_begin;
    k.inv_dlnlam = (float)(1.0 / c.dlnlam);
    k.zscale = (float)(ZSORT_ZBINS / (std::log1p(c.opts.z_max) / c.dlnlam + 1.0));
    k.mu_lo = c.sort_mu_lo;
    k.mu_scale = c.sort_mu_scale;
    k.mua = c.sort_mua;
    k.mub = c.sort_mub;
    k.um = c.n_u > 1 ? params + 12 * G_stride + g_begin : nullptr;
    k.u_lo = c.sort_u_lo;
    k.u_scale = c.sort_u_scale;
    // with the nebular axis and tile skipping, the tiles' log U ranges are set
    // here, before the weights, which then write only those sections
    k.us = c.n_u > 1 ? params + 13 * G_stride + g_begin : nullptr;
    k.uedge = c.d_uedge;
    k.n_u = c.n_u;
    k.urange = c.n_u > 1 && c.opts.band_skip ? w.urange : nullptr;
    const int n_tiles = (int)((n + 127) / 128);
    cudaError_t e = cudaMemsetAsync(w.hist, 0, ZSORT_BUCKETS * sizeof(int), s);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((n + 255) / 256);   // n >= n_tiles
    zsort_hist_kernel<<<blocks, 256, 0, s>>>(k, n, w.hist, w.trange, w.urange, c.n_u, w.kmask, n_tiles,
                                             c.kmask_words);
    zsort_scan_kernel<<<1, 1024, 0, s>>>(w.hist);
    zsort_scatter_kernel<<<blocks, 256, 0, s>>>(k, n, w.hist, w.perm);
    zsort_tile_kernel<<<(unsigned)n_tiles, 128, 0, s>>>(k, n, w.perm);
    return cudaGetLastError();
}

cudaError_t launch_combine(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, int parts, float *mags,
                           cudaStream_t s, const HistArgs *hist) {
    (void)c;
    if (n <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    const HistArgs h = hist ? *hist : HistArgs{};
#define DSPS_COMBINE(Q4)                                                                                      \
    combine_mags_kernel<Q4><<<blocks, 256, 0, s>>>(w.partial, parts, n, fs.Q, w.magoff, fs.d_offq, w.gidx, mags, h)
    switch (fs.Q4) {
    case 1: DSPS_COMBINE(1); break;
    case 2: DSPS_COMBINE(2); break;
    case 3: DSPS_COMBINE(3); break;
    default: DSPS_COMBINE(4); break;
    }
#undef DSPS_COMBINE
    return cudaGetLastError();
}

}  // namespace dsps
