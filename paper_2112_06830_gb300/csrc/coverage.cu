// coverage.cu -- the fraction of each filter's response that the SSP grid
// reaches as a galaxy is seen (Sec. 2.2, Eq. restmag: the SED is zero outside
// the grid), a diagnostic that marks the bands measured only through a
// filter's far tail (include/dsps.h: dsps_band_coverage).
//
// For galaxy g and filter q the grid spans ln lam in [a, b] = [ln lam_0,
// ln lam_{N-1}] + ln(1+z) (observer frame; no shift for a rest-frame set).
// With A(x) and B(x) the filter's response left and right of ln lam = x over
// D_q (accumulated on the host from the filter's own table, trapezoids of
// T / lam, FP64), the covered fraction is taken from the side where it is
// small: A(b) - A(a) when the range ends below the point where A reaches 1/2,
// B(a) - B(b) when it starts above it, the two halves' pieces otherwise.
// Inside a table interval A and B are linear in lam.
#include <cmath>

#include "dsps_internal.cuh"

namespace dsps {

void set_last_error(const char *msg);

namespace {

struct CovArgs {
    const float *z;          // parameter row 11 of the chunk
    const double *cov;       // (ln lam, A, B) per table point
    int off[DSPS_MAX_FILTERS + 1], mid[DSPS_MAX_FILTERS];
    int Q, rest;
    double lo, hi;           // ln lam of the first and last grid node
    int64_t n;
    float *out;              // [n][Q]
};

// A (side 1) or B (side 2) at ln lam = x, for the points [p0, p1) of one filter.
__device__ double cum_at(const double *cov, int p0, int p1, double x, int side) {
    if (x <= cov[3 * p0]) return side == 1 ? 0.0 : 1.0;
    if (x >= cov[3 * (p1 - 1)]) return side == 1 ? 1.0 : 0.0;
    int lo = p0, hi = p1 - 1;   // cov[3 lo] <= x < cov[3 hi]
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (cov[3 * m] <= x) lo = m;
        else hi = m;
    }
    const double l0 = exp(cov[3 * lo]), l1 = exp(cov[3 * hi]);
    const double t = (exp(x) - l0) / (l1 - l0);
    return cov[3 * lo + side] + t * (cov[3 * hi + side] - cov[3 * lo + side]);
}

__global__ void band_coverage_kernel(const CovArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n * a.Q) return;
    const int64_t g = i / a.Q;
    const int q = (int)(i - g * a.Q);
    double shift = 0.0;
    if (!a.rest) {
        const float z = a.z[g];
        if (!(z > 0.f) || !isfinite(z)) {
            a.out[i] = __int_as_float(0x7fc00000);
            return;
        }
        shift = log1p((double)z);
    }
    const int p0 = a.off[q], p1 = a.off[q + 1];
    const double xa = fmax(a.lo + shift, a.cov[3 * p0]), xb = fmin(a.hi + shift, a.cov[3 * (p1 - 1)]);
    double c = 0.0;
    if (xb > xa) {
        const double xm = a.cov[3 * a.mid[q]];
        if (xb <= xm) {
            c = cum_at(a.cov, p0, p1, xb, 1) - cum_at(a.cov, p0, p1, xa, 1);
        } else if (xa >= xm) {
            c = cum_at(a.cov, p0, p1, xa, 2) - cum_at(a.cov, p0, p1, xb, 2);
        } else {
            c = (a.cov[3 * a.mid[q] + 1] - cum_at(a.cov, p0, p1, xa, 1)) +
                (a.cov[3 * a.mid[q] + 2] - cum_at(a.cov, p0, p1, xb, 2));
        }
    }
    a.out[i] = (float)fmin(fmax(c, 0.0), 1.0);
}

}  // namespace

}  // namespace dsps

extern "C" int dsps_band_coverage(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t set_id,
                                  float *coverage, dsps_stream_t stream) {
    using namespace dsps;
    DSPS_TRACE("dsps_band_coverage");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || n_gal < 0 || (n_gal > 0 && (!params || !coverage))) {
        set_last_error("dsps_band_coverage: bad argument");
        return DSPS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(c->mu);
    if (set_id < 0 || set_id >= (int)c->sets.size()) {
        set_last_error("dsps_band_coverage: unknown set");
        return DSPS_ERR_INVALID_ARG;
    }
    if (n_gal == 0) return DSPS_OK;
    const FilterSet &fs = c->sets[set_id];
    CovArgs a{};
    a.z = params + 11 * n_gal;
    a.cov = fs.d_cov;
    for (int q = 0; q <= fs.Q; ++q) a.off[q] = fs.cov_off[q];
    for (int q = 0; q < fs.Q; ++q) a.mid[q] = fs.cov_mid[q];
    a.Q = fs.Q;
    a.rest = fs.rest;
    a.lo = c->lnlam0;
    a.hi = c->lnlam0 + (c->n_lam - 1) * c->dlnlam;
    a.n = n_gal;
    a.out = coverage;
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) {
        const int64_t tot = n_gal * fs.Q;
        band_coverage_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return DSPS_ERR_CUDA;
    }
    return DSPS_OK;
}
