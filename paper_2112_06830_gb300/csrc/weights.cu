// weights.cu -- per-galaxy SSP weights (Sec. 3.1 and 3.2 of Hearin et al. 2021).
//
// One warp per galaxy:
//   1. t_obs(z) and Dmod(z) from the FP64 cosmology table (Sec. 2.2).
//   2. SFR at the uniform cosmic-time nodes (Sec. 3.1), FP32.
//   3-4. Age-bin masses int_{t_obs - e_{i+1}}^{t_obs - e_i} SFR (the numerator of
//      P_SFH after Eq. cspsum) for the piecewise-linear SFR.  Each bin is
//      integrated directly -- the exact bin width times the mean SFR inside one
//      interval, partial plus whole interval integrals across nodes -- so the
//      youngest bins (down to ~1e-8 of the mass of a quenched galaxy) keep
//      their relative precision in FP32 instead of being the difference of two
//      cumulative masses.  The total M(t_obs) (Eq. mstartot) is accumulated in
//      FP64, and t_obs's position on the time grid is split off in FP64.
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
    double t0, h, inv_h, dz, inv_dz, zmax, dlnlam;
    const float *logage;
    const float *einh;     // [n_age+1] age-bin edge / h
    const float *bwidth;   // [n_age] e_{i+1} - e_i [Gyr]
    const float *zedge;
    const double *tlut, *glut;
    const float *wmul;
    float *w_msun, *w32;
    __nv_bfloat16 *whi, *wlo;
    float *aux;
    double *magoff;
    const int *perm;   // sorted row -> chunk-local galaxy, or nullptr
    int *gidx;         // out: sorted row -> chunk-local galaxy, or nullptr
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
    const float c = kernel == DSPS_MDF_TRIWEIGHT ? terf_lower_f(a) : gauss_cdf_f(a);
    return u > 0.f ? -c : c;
}

__device__ __forceinline__ float mdf_bin(int kernel, float u_lo, float u_hi) {
    float p = mdf_s(kernel, u_hi) - mdf_s(kernel, u_lo);
    if (u_lo <= 0.f && u_hi > 0.f) p += 1.f;
    return p;
}

// Bins spanning more time intervals than this use the FP32 node prefix (their
// mass is a large share of the prefix, so the difference does not cancel).
constexpr int PREFIX_SPAN = 64;

__host__ __device__ inline size_t weights_smem_per_warp(int n_t, int n_age) {
    return (((size_t)n_t * 3 + (size_t)(n_age + 1) * 2 + (size_t)n_age * 2) * 4 + 15) & ~(size_t)15;
}

template <int MODE>
__global__ void __launch_bounds__(256) weights_kernel(WArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const size_t per_warp = weights_smem_per_warp(a.n_t, a.n_age);
    unsigned char *base = smem_raw + per_warp * warp;
    float *sfr = reinterpret_cast<float *>(base);       // [n_t]
    float *itg = sfr + a.n_t;                            // [n_t]
    float *cum = itg + a.n_t;                            // [n_t]
    int *em = reinterpret_cast<int *>(cum + a.n_t);     // [n_age + 1]
    float *er = reinterpret_cast<float *>(em + a.n_age + 1);
    float *bmass = er + a.n_age + 1;                     // [n_age]
    float *frac = bmass + a.n_age;                       // [n_age]

    const int64_t gi = (int64_t)blockIdx.x * nwarps + warp;
    if (gi >= a.n) return;
    const int64_t gl = a.perm ? (int64_t)a.perm[gi] : gi;
    const int64_t g = a.g_begin + gl;

    float mine = lane < NPAR ? a.params[(int64_t)lane * a.G_stride + g] : 0.f;
    float p[NPAR];
#pragma unroll
    for (int r = 0; r < NPAR; ++r) p[r] = __shfl_sync(0xffffffffu, mine, r);

    const float z = p[11], sig = p[6];
    bool valid = __all_sync(0xffffffffu, isfinite(mine) || lane >= NPAR);
    valid = valid && z > 0.f && (double)z <= a.zmax && sig > 0.f && p[0] > 0.f;

    // 1. cosmology: FP64 table lookup of t_obs, and t_obs's position on the
    //    time grid, a = (t_obs - t0)/h = m_obs + f_obs (FP64, split once)
    int m_obs = 0;
    float f_obs = 0.f;
    if (lane == 0 && valid) {
        double x = (double)z * a.inv_dz;
        int i = min((int)x, a.n_lut - 2);
        double fr = x - i;
        const double t_obs = a.tlut[i] + fr * (a.tlut[i + 1] - a.tlut[i]);
        const double apos = (t_obs - a.t0) * a.inv_h;
        if (apos > 0.0) {
            m_obs = min((int)apos, a.n_t - 2);
            f_obs = (float)(apos - m_obs);
        } else {
            m_obs = -1;
        }
    }
    m_obs = __shfl_sync(0xffffffffu, m_obs, 0);
    f_obs = __shfl_sync(0xffffffffu, f_obs, 0);
    valid = valid && m_obs >= 0;

    // 2. SFR at the time nodes (FP32) and the interval integrals I_j
    const float h = (float)a.h;
    for (int n = lane; n < a.n_t; n += 32)
        sfr[n] = valid ? sfr_f(a.sfh_model, p, fmaf((float)n, h, (float)a.t0)) : 0.f;
    __syncwarp();
    for (int j = lane; j < a.n_t - 1; j += 32) itg[j] = 0.5f * h * (sfr[j] + sfr[j + 1]);
    __syncwarp();

    // 3. FP32 prefix of the interval integrals at the nodes, C[j] = sum_{j'<j} I_j'
    //    (used only for bins wider than PREFIX_SPAN intervals, where it does not cancel)
    const int cnt = (a.n_t + 31) / 32;
    const int b = min(lane * cnt, a.n_t), e = min(b + cnt, a.n_t);
    float tot = 0.f;
    for (int j = b; j < e && j < a.n_t - 1; ++j) tot += itg[j];
    float incl = tot;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        float o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
    }
    float run = incl - tot;
    for (int j = b; j < e; ++j) {
        cum[j] = run;
        if (j < a.n_t - 1) run += itg[j];
    }
    // position of every age-bin edge on the time grid: y = f_obs - e/h
    for (int ei = lane; ei <= a.n_age; ei += 32) {
        const float y = f_obs - __ldg(a.einh + ei);
        const float fl = floorf(y);
        em[ei] = m_obs + (int)fl;
        er[ei] = y - fl;
    }
    __syncwarp();

    // 4. age-bin masses (Eq. cspsum's P_SFH numerator) integrated directly from
    //    the piecewise-linear SFR; the total (Eq. mstartot at t_obs) in FP64.
    float lsum = 0.f;
    for (int i = lane; i < a.n_age; i += 32) {
        const int mi = em[i], mo = em[i + 1];
        const float ri = er[i], ro = er[i + 1];
        float B = 0.f;
        if (valid && mi >= 0) {
            const float si = fmaf(sfr[mi + 1] - sfr[mi], ri, sfr[mi]);         // SFR at the younger edge
            const float Pi = 0.5f * h * ri * (sfr[mi] + si);                     // int_{t_mi}^{tau_i}
            if (mo < 0) {
                B = cum[mi] + Pi;
            } else {
                const float so = fmaf(sfr[mo + 1] - sfr[mo], ro, sfr[mo]);     // SFR at the older edge
                const float w = __ldg(a.bwidth + i);                             // tau_i - tau_{i+1}, exact
                if (mi == mo) {
                    B = 0.5f * w * (si + so);
                } else if (mi == mo + 1) {
                    const float yv = h * ri;
                    B = 0.5f * (w - yv) * (so + sfr[mi]) + 0.5f * yv * (sfr[mi] + si);
                } else {
                    const float Qo = 0.5f * h * (1.f - ro) * (so + sfr[mo + 1]);  // int_{tau_o}^{t_mo+1}
                    float mid = 0.f;
                    if (mi - mo <= PREFIX_SPAN) {
                        for (int j = mo + 1; j < mi; ++j) mid += itg[j];
                    } else {
                        mid = cum[mi] - cum[mo + 1];
                    }
                    B = Qo + mid + Pi;
                }
            }
        }
        bmass[i] = B;
        lsum += B;
    }
    double msum = (double)lsum;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) msum += __shfl_xor_sync(0xffffffffu, msum, off);
    valid = valid && msum > 0.0 && isfinite(msum);
    const float inv_mtot = valid ? 1.f / (float)msum : 0.f;
    __syncwarp();
    for (int i = lane; i < a.n_age; i += 32) frac[i] = bmass[i] * inv_mtot;
    __syncwarp();

    // 5-6. metallicity weights and output, four consecutive k per lane.  The
    //      CDF at the upper edge of bin j is the lower edge of bin j+1, and the
    //      outer edges (-inf, +inf) need no evaluation, so each k costs about
    //      one CDF evaluation.
    const float inv_sig = 1.f / sig;
    const float mass = exp10f(p[10]);
    const int kend = MODE == W_MSUN ? a.K : a.K_pad;
    const int nz = a.n_z;
    const int di = 128 / nz, dj = 128 % nz;
    int k = 4 * lane;
    int i0 = k / nz, j0 = k - i0 * nz;
    for (; k < kend; k += 128) {
        float om[4];
        int i = i0, j = j0;
        float mu_i = fmaf(p[7], __ldg(a.logage + min(i, a.n_age - 1)) - 9.f, p[5]);
        float u_lo = (__ldg(a.zedge + j) - mu_i) * inv_sig;
        float s_lo = j == 0 ? 0.f : mdf_s(a.mdf_kernel, u_lo);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            om[c] = 0.f;
            if (k + c < a.K && valid) {
                const bool last = j == nz - 1;
                const float u_hi = last ? 1e30f : (__ldg(a.zedge + j + 1) - mu_i) * inv_sig;
                const float s_hi = last ? 0.f : mdf_s(a.mdf_kernel, u_hi);
                float pj = s_hi - s_lo;
                if (u_lo <= 0.f && u_hi > 0.f) pj += 1.f;
                om[c] = frac[i] * pj;
                s_lo = s_hi;
                u_lo = u_hi;
            }
            if (++j == nz) {   // next age row: its lower edge is -inf
                j = 0;
                ++i;
                mu_i = fmaf(p[7], __ldg(a.logage + min(i, a.n_age - 1)) - 9.f, p[5]);
                u_lo = -1e30f;
                s_lo = 0.f;
            }
        }
        if (MODE == W_MSUN) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (k + c < a.K) a.w_msun[gi * a.K + k + c] = mass * om[c];
        } else if (MODE == W_OMEGA_F32) {
            if (k < a.K_pad)
                *reinterpret_cast<float4 *>(a.w32 + gi * a.K_pad + k) = make_float4(om[0], om[1], om[2], om[3]);
        } else if (k < a.K_pad) {
            const float4 wm = __ldg(reinterpret_cast<const float4 *>(a.wmul + k));
            const float w0 = om[0] * wm.x, w1 = om[1] * wm.y, w2 = om[2] * wm.z, w3 = om[3] * wm.w;
            const __nv_bfloat162 h01 = __floats2bfloat162_rn(w0, w1), h23 = __floats2bfloat162_rn(w2, w3);
            const __nv_bfloat162 l01 = __floats2bfloat162_rn(w0 - __low2float(h01), w1 - __high2float(h01));
            const __nv_bfloat162 l23 = __floats2bfloat162_rn(w2 - __low2float(h23), w3 - __high2float(h23));
            uint2 hv, lv;
            hv.x = *reinterpret_cast<const unsigned *>(&h01);
            hv.y = *reinterpret_cast<const unsigned *>(&h23);
            lv.x = *reinterpret_cast<const unsigned *>(&l01);
            lv.y = *reinterpret_cast<const unsigned *>(&l23);
            *reinterpret_cast<uint2 *>(a.whi + gi * a.K_pad + k) = hv;
            *reinterpret_cast<uint2 *>(a.wlo + gi * a.K_pad + k) = lv;
        }
        i0 += di;
        j0 += dj;
        if (j0 >= nz) { j0 -= nz; ++i0; }
    }

    if (lane == 0) {
        if (!valid) atomicOr(a.err, DERR_PARAM);
        if (a.gidx) a.gidx[gi] = (int)gl;
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
                double x = (double)z * a.inv_dz;
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
                           int64_t g_begin, int64_t n, float *w_msun, cudaStream_t s, const Scratch *ws,
                           bool sorted) {
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
    a.inv_dz = 1.0 / c.dz_lut;
    a.zmax = c.opts.z_max;
    a.dlnlam = c.dlnlam;
    a.logage = c.d_logage;
    a.einh = c.d_einh;
    a.bwidth = c.d_bwidth;
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
    a.perm = sorted ? c.d_perm : nullptr;
    a.gidx = sorted ? c.d_gidx : nullptr;
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
