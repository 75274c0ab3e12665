// weights.cu -- per-galaxy SSP weights (Sec. 3.1 and 3.2 of Hearin et al. 2021).
//
// One warp per galaxy:
//   1. t_obs(z) and Dmod(z) from the FP64 cosmology table (Sec. 2.2).
//   2. SFR at the uniform cosmic-time nodes (Sec. 3.1), FP32.
//   3. Cumulative formed mass M(t) = int_{t0}^{t} SFR (Eq. mstartot), FP64 warp
//      scan of the trapezoid sums; inside an interval M is the exact integral of
//      the piecewise-linear SFR.
//   4. Age-bin mass fractions P_SFH(i) = [M(t_obs - e_i) - M(t_obs - e_{i+1})]
//      / M(t_obs) (Eq. cspsum and the P_SFH definition), FP64 differencing:
//      the youngest bins are ~1e-5 of the total and lose their digits in FP32.
//   5. Metallicity weights P_met(j | i) as differences of the triweight
//      (Appendix B, Eq. terf) or Gaussian CDF over lgZ bin edges, with the mean
//      moving linearly in log age (Sec. 3.2, Eq. agedep_mdf), FP32.
//   6. Joint weights omega_ij = P_SFH(i) P_met(j | i) (Eq. full_mdf), written as
//      Msun (dsps_weights), FP32 per unit mass (SIMT photometry) or scaled by
//      the SSP row multiplier and split into bf16 hi + lo (tensor photometry).
#include "dsps_internal.cuh"

namespace dsps {

struct WArgs {
    const float *params;
    int64_t G_stride, g_begin, n;
    int n_age, n_z, K, K_pad, n_t, sfh_model, mdf_kernel, n_lut;
    double t0, h, inv_h, dz, zmax, dlnlam;
    const float *logage;
    const double *edges;
    const float *zedge;
    const double *tlut, *glut;
    const float *wmul;
    float *w_msun, *w32;
    __nv_bfloat16 *whi, *wlo;
    float *aux;
    double *magoff;
    unsigned *err;
};

// Sec. 3.1: SFR at cosmic time t [Gyr] (arbitrary normalisation).
__device__ __forceinline__ float sfr_f(int model, const float *p, float t) {
    if (model == DSPS_SFH_DELAYED_TAU) return t * expf(-t / p[0]);
    float lr = logf(t / p[0]);
    float ms = 1.f / (expf(-p[1] * lr) + expf(-p[2] * lr));
    float zq = (t - (p[3] - 0.9f)) * (1.f / 0.3f);
    return ms * exp10f(-p[4] * terf_f(zq));
}

// Triweight / Gaussian CDF in the form S(u) = C(u) for u <= 0 and C(u) - 1 for
// u > 0, so that differences of neighbouring edges keep their relative
// precision in both tails; P = S(u_hi) - S(u_lo) + [u_lo <= 0 < u_hi].
__device__ __forceinline__ float mdf_s(int kernel, float u) {
    const float a = -fabsf(u);
    const float c = kernel == DSPS_MDF_TRIWEIGHT ? terf_f(a) : gauss_cdf_f(a);
    return u > 0.f ? -c : c;
}

__device__ __forceinline__ float mdf_bin(int kernel, float u_lo, float u_hi) {
    float p = mdf_s(kernel, u_hi) - mdf_s(kernel, u_lo);
    if (u_lo <= 0.f && u_hi > 0.f) p += 1.f;
    return p;
}

template <int MODE>
__global__ void __launch_bounds__(256) weights_kernel(WArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const size_t per_warp = ((size_t)a.n_t * 16 + (size_t)(a.n_age + 1) * 8 + (size_t)a.n_age * 4 + 15) & ~(size_t)15;
    unsigned char *base = smem_raw + per_warp * warp;
    double *sfr = reinterpret_cast<double *>(base);
    double *cum = sfr + a.n_t;
    double *phi = cum + a.n_t;
    float *frac = reinterpret_cast<float *>(phi + a.n_age + 1);

    const int64_t gi = (int64_t)blockIdx.x * nwarps + warp;
    if (gi >= a.n) return;
    const int64_t g = a.g_begin + gi;

    float mine = lane < NPAR ? a.params[(int64_t)lane * a.G_stride + g] : 0.f;
    float p[NPAR];
#pragma unroll
    for (int r = 0; r < NPAR; ++r) p[r] = __shfl_sync(0xffffffffu, mine, r);

    const float z = p[11], sig = p[6];
    bool valid = __all_sync(0xffffffffu, isfinite(mine) || lane >= NPAR);
    valid = valid && z > 0.f && (double)z <= a.zmax && sig > 0.f && p[0] > 0.f;

    // 1. cosmology: FP64 table lookup of t_obs; Dmod in FP32 pieces summed in FP64
    double t_obs = 0.0;
    {
        double x = (double)z / a.dz;
        int i = valid ? min((int)x, a.n_lut - 2) : 0;
        double fr = x - i;
        t_obs = a.tlut[i] + fr * (a.tlut[i + 1] - a.tlut[i]);
    }

    // 2. SFR at the time nodes (FP32 evaluation, stored as FP64)
    for (int n = lane; n < a.n_t; n += 32)
        sfr[n] = valid ? (double)sfr_f(a.sfh_model, p, (float)(a.t0 + n * a.h)) : 0.0;
    __syncwarp();

    // 3. FP64 prefix of the trapezoid sums (Eq. mstartot)
    const double hh = 0.5 * a.h;
    const int cnt = (a.n_t + 31) / 32;
    const int b = min(lane * cnt, a.n_t), e = min(b + cnt, a.n_t);
    double tot = 0.0;
    for (int j = b; j < e && j < a.n_t - 1; ++j) tot += sfr[j] + sfr[j + 1];
    double incl = tot;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        double o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
    }
    double run = incl - tot;   // in units of h/2
    for (int j = b; j < e; ++j) {
        cum[j] = run * hh;
        if (j < a.n_t - 1) run += sfr[j] + sfr[j + 1];
    }
    __syncwarp();

    // 4. mass formed before t_obs - e for every age-bin edge, FP64
    const double hinv2 = 0.5 * a.inv_h;
    for (int ei = lane; ei <= a.n_age; ei += 32) {
        const double tau = t_obs - a.edges[ei];
        double M = 0.0;
        if (tau > a.t0) {
            const double x = (tau - a.t0) * a.inv_h;
            const int m = min((int)x, a.n_t - 2);
            const double u = (x - m) * a.h;
            M = cum[m] + u * (sfr[m] + (sfr[m + 1] - sfr[m]) * u * hinv2);
        }
        phi[ei] = M;
    }
    __syncwarp();
    const double Mtot = phi[0];
    valid = valid && Mtot > 0.0 && isfinite(Mtot);
    const float inv_mtot = valid ? 1.f / (float)Mtot : 0.f;
    // bin masses: FP64 differences of the prefix, then FP32
    for (int i = lane; i < a.n_age; i += 32) frac[i] = (float)(phi[i] - phi[i + 1]) * inv_mtot;
    __syncwarp();

    // 5-6. metallicity weights and output, two consecutive k per lane
    const float inv_sig = 1.f / sig;
    const float mass = exp10f(p[10]);
    const int kend = MODE == W_MSUN ? a.K : a.K_pad;
    const int nz = a.n_z;
    const int di = 64 / nz, dj = 64 % nz;
    int k = 2 * lane;
    int i0 = k / nz, j0 = k - i0 * nz;
    for (; k < kend; k += 64) {
        float om[2];
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
            int i = i0, j = j0 + h2;
            if (j >= nz) { j -= nz; ++i; }
            om[h2] = 0.f;
            if (k + h2 < a.K && valid) {
                const float mu_i = fmaf(p[7], __ldg(a.logage + i) - 9.f, p[5]);
                const float u_lo = (__ldg(a.zedge + j) - mu_i) * inv_sig;
                const float u_hi = (__ldg(a.zedge + j + 1) - mu_i) * inv_sig;
                om[h2] = frac[i] * mdf_bin(a.mdf_kernel, u_lo, u_hi);
            }
        }
        if (MODE == W_MSUN) {
            if (k < a.K) a.w_msun[gi * a.K + k] = mass * om[0];
            if (k + 1 < a.K) a.w_msun[gi * a.K + k + 1] = mass * om[1];
        } else if (MODE == W_OMEGA_F32) {
            *reinterpret_cast<float2 *>(a.w32 + gi * a.K_pad + k) = make_float2(om[0], om[1]);
        } else {
            const float2 wm = __ldg(reinterpret_cast<const float2 *>(a.wmul + k));
            const float w0 = om[0] * wm.x, w1 = om[1] * wm.y;
            const __nv_bfloat162 hi = __floats2bfloat162_rn(w0, w1);
            const __nv_bfloat162 lo = __floats2bfloat162_rn(w0 - __low2float(hi), w1 - __high2float(hi));
            *reinterpret_cast<__nv_bfloat162 *>(a.whi + gi * a.K_pad + k) = hi;
            *reinterpret_cast<__nv_bfloat162 *>(a.wlo + gi * a.K_pad + k) = lo;
        }
        i0 += di;
        j0 += dj;
        if (j0 >= nz) { j0 -= nz; ++i0; }
    }

    if (lane == 0) {
        if (!valid) atomicOr(a.err, DERR_PARAM);
        if (MODE != W_MSUN) {
            float *ax = a.aux + gi * AUX_STRIDE;
            ax[0] = -0.4f * 3.32192809488736235f * p[8];
            ax[1] = p[9] - 0.7f;
            ax[2] = valid ? (float)(log1pf(z) / (float)a.dlnlam) : 0.f;
            ax[3] = valid ? 1.f : 0.f;
            ax[4] = p[8];
            ax[5] = p[9];
            ax[6] = 0.f;
            ax[7] = 0.f;
            double magoff = __longlong_as_double(0x7ff8000000000000LL);
            if (valid) {
                double x = (double)z / a.dz;
                int i = min((int)x, a.n_lut - 2);
                double fr = x - i;
                double gz = a.glut[i] + fr * (a.glut[i + 1] - a.glut[i]);
                magoff = -2.5 * (double)p[10] + gz + (double)(5.f * log10f(z)) - (double)(2.5f * log10f(1.f + z));
            }
            a.magoff[gi] = magoff;
        }
    }
}

cudaError_t launch_weights(const Ctx &c, int mode, const float *params, int64_t G_stride,
                           int64_t g_begin, int64_t n, float *w_msun, cudaStream_t s, const Scratch *ws) {
    if (n <= 0) return cudaSuccess;
    WArgs a{};
    a.params = params;
    a.G_stride = G_stride;
    a.g_begin = g_begin;
    a.n = n;
    a.n_age = c.n_age;
    a.n_z = c.n_z;
    a.K = c.K;
    a.K_pad = c.K_pad;
    a.n_t = c.n_t;
    a.sfh_model = c.opts.sfh_model;
    a.mdf_kernel = c.opts.mdf_kernel;
    a.n_lut = c.n_lut;
    a.t0 = c.t0;
    a.h = (c.t1 - c.t0) / (c.n_t - 1);
    a.inv_h = 1.0 / a.h;
    a.dz = c.dz_lut;
    a.zmax = c.opts.z_max;
    a.dlnlam = c.dlnlam;
    a.logage = c.d_logage;
    a.edges = c.d_edges;
    a.zedge = c.d_zedge;
    a.tlut = c.d_tlut;
    a.glut = c.d_glut;
    a.wmul = c.d_wmul;
    a.w_msun = w_msun;
    a.w32 = c.d_w32;
    a.whi = c.d_whi;
    a.wlo = c.d_wlo;
    a.aux = c.d_aux;
    a.magoff = c.d_magoff;
    a.err = c.d_err;
    if (ws) {
        a.w32 = ws->w32;
        a.aux = ws->aux;
        a.magoff = ws->magoff;
    }
    const int threads = 256, warps = threads / 32;
    size_t per_warp = ((size_t)c.n_t * 16 + (size_t)(c.n_age + 1) * 8 + (size_t)c.n_age * 4 + 15) & ~(size_t)15;
    size_t smem = per_warp * warps;
    dim3 grid((unsigned)((n + warps - 1) / warps));
    switch (mode) {
    case W_MSUN:
        cudaFuncSetAttribute(weights_kernel<W_MSUN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        weights_kernel<W_MSUN><<<grid, threads, smem, s>>>(a);
        break;
    case W_OMEGA_F32:
        cudaFuncSetAttribute(weights_kernel<W_OMEGA_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        weights_kernel<W_OMEGA_F32><<<grid, threads, smem, s>>>(a);
        break;
    default:
        cudaFuncSetAttribute(weights_kernel<W_OMEGA_BF16X2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        weights_kernel<W_OMEGA_BF16X2><<<grid, threads, smem, s>>>(a);
        break;
    }
    return cudaGetLastError();
}

}  // namespace dsps
