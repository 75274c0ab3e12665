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
//      cumulative masses.  The whole-interval masses come from a node prefix
//      held as an unevaluated FP32 pair (TwoSum at every addition); the total
//      M(t_obs) (Eq. mstartot) is an FP32 warp tree sum of the bin masses; only
//      t_obs's position on the time grid is split off in FP64 (prep kernel).
//   5. Metallicity weights P_met(j | i) as differences of the triweight
//      (Appendix B, Eq. terf) or Gaussian CDF over lgZ bin edges, with the mean
//      moving linearly in log age (Sec. 3.2, Eq. agedep_mdf), FP32.
//   6. Joint weights omega_ij = P_SFH(i) P_met(j | i) (Eq. full_mdf), times
//      P_neb(u) with a nebular axis (Sec. 3.3, Eq. nebsed: triweight CDF
//      differences over the log U bins), written as Msun (dsps_weights), FP32
//      per unit mass (SIMT photometry) or scaled by the SSP row multiplier and
//      split into bf16 hi + lo (tensor photometry, metallicity-major K, with
//      the per-tile ranges and kz-block masks).
// The kernels are instantiated with and without the nebular axis (NEB), so
// that grids without one run the code of the two-dimensional weights.
#include <cfloat>
#include <climits>
#include <cmath>
#include <type_traits>

#include "dsps_internal.cuh"
#include "f32x2.cuh"

namespace dsps {

struct WArgs {
    const float *params;
    int64_t G_stride, g_begin, n;
    int n_age, n_z, K, K_pad, A_pad, KZ_pad, n_t, sfh_model, mdf_kernel, n_lut, dust_bump, dust_law;
    int n_u, SEC, u_ref, npar;   // nebular axis (n_u = 1: none), section length, reference bin, parameter rows
    int row_sfr, grow_sfr;       // tabulated SFH: parameter rows of the node SFRs and their gradient rows
    int rest;                    // rest-frame magnitudes: no redshift shift, no distance terms
    int urange_pre;              // tiles' log U ranges preset by the sort: write only those sections
    float *fcache_wr;            // out: the age fractions by sorted row [n][n_age] (NaN: invalid), or nullptr
    const float *fcache_rd;      // a one-age launch: its age's fraction from there instead of the SFH, or nullptr
    const float *uedge;          // [n_u + 1] log U bin edges (+-1e30 outer)
    int2 *urange;                // out: per-tile log U bin ranges (atomics), with trange
    int age_lo, age_hi;          // age bins whose weights are written (the others are 0): a dust group
    float dust_T;                // the group's weight of the old-star dust values
    int dust_row_old;            // parameter row of Av_old (delta_old next), or -1: one curve
    int aux_yo;                  // aux gets the young and old dust values (a one-launch contraction of
                                 // every dust group forms each group's curve from them)
    double t0, h, inv_h, dz, inv_dz, zmax, dlnlam;
    float zmax_f;          // largest float <= zmax (z <= zmax_f iff (double)z <= zmax)
    float t0_f, h_f, dlnlam_f;   // FP32 copies used by the per-galaxy warps
    const float *logage;
    const float *mua, *mub;   // [n_age] MDF mean of bin i: mua_i p5 + mub_i p7 (dsps.h: DSPS_MDF_MEAN_*)
    const float *einh;     // [n_age+1] age-bin edge / h
    const float *bwidth;   // [n_age] e_{i+1} - e_i [Gyr]
    const float *zedge;
    const double *tlut;    // [n_lut] t_obs(z) [Gyr]
    const float *glut;     // [n_lut] Dmod(z) - 5 log10 z
    const float *wmul;
    const float *wmul_ab;  // [KA_pad] the age-block order's row multipliers (W_OMEGA_BF16X2_AB)
    int KA_pad;            // row length of the age-block order
    float *w_msun, *w32;
    __nv_bfloat16 *whi, *wlo;
    float *aux;
    float *magoff;
    const int *perm;   // sorted row -> chunk-local galaxy, or nullptr
    int *gidx;         // out: sorted row -> chunk-local galaxy, or nullptr
    int2 *trange;      // out: per-tile redshift-shift ranges (atomics), or nullptr
    unsigned *kmask;   // out: per-tile kz-block masks (atomics), with trange
    int kmw;           // mask words per tile
    GalPrep *prep;     // per-galaxy scalars, chunk order (galaxy_prep_kernel)
    unsigned *err;
};

// Sec. 3.1: SFR at cosmic time t [Gyr] (arbitrary normalisation).  The power
// laws take ln(t / tau) of the correctly rounded ratio, which keeps the
// exponent's absolute error near 1e-7 (the metallicity gradients, sums with
// strong cancellation, see that error through the age-bin fractions).
// The SFH model and the metallicity kernel are template parameters of the
// kernels (SFH = DSPS_SFH_*, MDF = DSPS_MDF_*), so that no evaluation pays
// for the other model's branch.
template <int SFH>
__device__ __forceinline__ float sfr_f(const float *p, float t) {
    if constexpr (SFH == DSPS_SFH_DELAYED_TAU) return t * expf(-t / p[0]);
    float lr = logf(t / p[0]);
    float ms = 1.f / (expf(-p[1] * lr) + expf(-p[2] * lr));
    float zq = (t - (p[3] - 0.9f)) * (1.f / 0.3f);
    return ms * exp10f(-p[4] * terf_f(zq));
}

// Triweight / Gaussian CDF in the form S(u) = C(u) for u <= 0 and C(u) - 1 for
// u > 0, so that differences of neighbouring edges keep their relative
// precision in both tails; P = S(u_hi) - S(u_lo) + [u_lo <= 0 < u_hi].
template <int MDF>
__device__ __forceinline__ float mdf_s(float u) {
    const float a = -fabsf(u);
    float c;
    if constexpr (MDF == DSPS_MDF_TRIWEIGHT) c = terf_lower_f(a);
    else c = gauss_cdf_f(a);
    return u > 0.f ? -c : c;
}

// mdf_s of two edges at once: the triweight's polynomial in paired FP32 ops
// (the same operations in the same order as terf_lower_f, so the same
// numbers), the Gaussian's pair by pair.
template <int MDF>
__device__ __forceinline__ float2 mdf_s2(float2 u) {
    if constexpr (MDF != DSPS_MDF_TRIWEIGHT) {
        return make_float2(mdf_s<MDF>(u.x), mdf_s<MDF>(u.y));
    } else {
        const float2 x = make_float2(-fabsf(u.x) + 3.f, -fabsf(u.y) + 3.f);
        const float2 x2 = mul2(x, x);
        float2 poly = fma2v(x, splat2(-1.f / 7.f), splat2(3.f));
        poly = fma2v(x, poly, splat2(-21.6f));
        poly = fma2v(x, poly, splat2(54.f));
        const float2 c = mul2(mul2(mul2(splat2(35.f / 69984.f), x2), x2), poly);
        const float cx = x.x <= 0.f ? 0.f : c.x, cy = x.y <= 0.f ? 0.f : c.y;
        return make_float2(u.x > 0.f ? -cx : cx, u.y > 0.f ? -cy : cy);
    }
}

__host__ __device__ inline size_t weights_smem_per_warp(int n_t, int n_age) {
    return (((size_t)n_t * 4 + (size_t)(n_age + 1) * 2 + (size_t)n_age * 2) * 4 + 15) & ~(size_t)15;
}

struct SfhSmem {
    float *sfr, *itg;         // [n_t] SFR at nodes, interval integrals
    float *cum_hi, *cum_lo;   // [n_t] node prefix of the interval integrals, unevaluated sum hi + lo
    int *em;                  // [n_age + 1] interval index of each age-bin edge
    float *er;                // [n_age + 1] position of the edge inside its interval
    float *bmass, *frac;      // [n_age] bin masses, fractions of the total
};

__device__ __forceinline__ SfhSmem sfh_smem(unsigned char *base, int n_t, int n_age) {
    SfhSmem m;
    m.sfr = reinterpret_cast<float *>(base);
    m.itg = m.sfr + n_t;
    m.cum_hi = m.itg + n_t;
    m.cum_lo = m.cum_hi + n_t;
    m.em = reinterpret_cast<int *>(m.cum_lo + n_t);
    m.er = reinterpret_cast<float *>(m.em + n_age + 1);
    m.bmass = m.er + n_age + 1;
    m.frac = m.bmass + n_age;
    return m;
}

// Error-free sum: s + e = a + b exactly (Knuth's TwoSum, six FP32 additions).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Stages 2-4 for one galaxy (whole warp), given t_obs's position on the time
// grid (m_obs + f_obs, from galaxy_prep_kernel): SFR at the nodes, the age-bin
// masses and their fractions of the total; returns the galaxy's validity and
// the total formed mass through msum_out.
template <int SFH>
__device__ __noinline__ bool sfh_stage(const WArgs &a, const float *p, int64_t g, bool valid, int m_obs, float f_obs,
                                       int lane, const SfhSmem &sm, float &msum_out) {
    float *sfr = sm.sfr, *itg = sm.itg, *er = sm.er, *bmass = sm.bmass, *frac = sm.frac;
    float *ch = sm.cum_hi, *cl = sm.cum_lo;
    int *em = sm.em;
    valid = valid && m_obs >= 0;

    // 2. SFR at the time nodes (FP32) and the interval integrals I_j; nodes
    //    after t_obs (n > m_obs + 1) bound no age bin and stay 0.  A tabulated
    //    history reads its nodes from its parameter rows (finite, >= 0).
    const float h = a.h_f;
    if constexpr (SFH == DSPS_SFH_TABLE) {
        const float *tab = a.params + (int64_t)a.row_sfr * a.G_stride + g;
        bool bad = false;
        for (int n = lane; n < a.n_t; n += 32) {
            const float v = valid && n <= m_obs + 1 ? tab[(int64_t)n * a.G_stride] : 0.f;
            bad = bad || !(v >= 0.f && v <= FLT_MAX);
            sfr[n] = v;
        }
        valid = valid && !__any_sync(0xffffffffu, bad);
    } else {
        for (int n = lane; n < a.n_t; n += 32)
            sfr[n] = valid && n <= m_obs + 1 ? sfr_f<SFH>(p, fmaf((float)n, h, a.t0_f)) : 0.f;
    }
    __syncwarp();
    for (int j = lane; j < a.n_t - 1; j += 32) itg[j] = 0.5f * h * (sfr[j] + sfr[j + 1]);
    __syncwarp();

    // 3. node prefix C[j] = sum_{j'<j} I_j' as an unevaluated FP32 pair
    //    (TwoSum at every addition): a bin's mass C[mi] - C[mo+1] then keeps
    //    FP32 relative precision however small it is next to C.  Each lane
    //    sums a run of cnt intervals; an inclusive warp scan of the run sums
    //    gives every run's offset.
    const int cnt = (a.n_t + 31) / 32;
    const int b = min(lane * cnt, a.n_t), e = min(b + cnt, a.n_t);
    float th = 0.f, tl = 0.f;
    for (int j = b; j < e && j < a.n_t - 1; ++j) {
        float err;
        two_sum(th, itg[j], th, err);
        tl += err;
    }
    float ih = th, il = tl;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float oh = __shfl_up_sync(0xffffffffu, ih, off), ol = __shfl_up_sync(0xffffffffu, il, off);
        if (lane >= off) {
            float err;
            two_sum(ih, oh, ih, err);
            il = il + ol + err;
        }
    }
    float rh = __shfl_up_sync(0xffffffffu, ih, 1), rl = __shfl_up_sync(0xffffffffu, il, 1);
    if (lane == 0) rh = rl = 0.f;
    for (int j = b; j < e; ++j) {
        ch[j] = rh;
        cl[j] = rl;
        if (j < a.n_t - 1) {
            float err;
            two_sum(rh, itg[j], rh, err);
            rl += err;
        }
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
    //    the piecewise-linear SFR: partial intervals at both edges plus the
    //    whole intervals between them (a difference of the prefix pair); the
    //    total (Eq. mstartot at t_obs) as a warp tree sum.
    float lsum = 0.f;
    for (int i = lane; i < a.n_age; i += 32) {
        const int mi = em[i], mo = em[i + 1];
        const float ri = er[i], ro = er[i + 1];
        float B = 0.f;
        if (valid && mi >= 0) {
            const float si = fmaf(sfr[mi + 1] - sfr[mi], ri, sfr[mi]);         // SFR at the younger edge
            const float Pi = 0.5f * h * ri * (sfr[mi] + si);                     // int_{t_mi}^{tau_i}
            if (mo < 0) {
                B = (ch[mi] + cl[mi]) + Pi;
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
                    const float mid = (ch[mi] - ch[mo + 1]) + (cl[mi] - cl[mo + 1]);
                    B = Qo + mid + Pi;
                }
            }
        }
        bmass[i] = B;
        lsum += B;
    }
    float msum = lsum;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) msum += __shfl_xor_sync(0xffffffffu, msum, off);
    valid = valid && msum > 0.f && isfinite(msum);
    const float inv_mtot = valid ? 1.f / msum : 0.f;
    __syncwarp();
    for (int i = lane; i < a.n_age; i += 32) frac[i] = bmass[i] * inv_mtot;
    __syncwarp();
    msum_out = msum;
    return valid;
}

// Stage 1 (Sec. 2.2), one thread per galaxy: t_obs(z) from the FP64 cosmology
// table and its position on the SFR time grid, (t_obs - t0)/h = m_obs + f_obs
// (split once in FP64), and the magnitude offset -2.5 logM + Dmod(z) - 2.5
// log10(1+z).  Kept apart from the per-galaxy warps of the weights kernels so
// that the FP64 arithmetic (slow on this GPU) runs one galaxy per lane.
__global__ void galaxy_prep_kernel(WArgs a, GalPrep *out) {
    const int64_t gl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gl >= a.n) return;
    const int64_t g = a.g_begin + gl;
    const float z = a.params[11 * a.G_stride + g];
    GalPrep r;
    r.m_obs = -1;
    r.f_obs = 0.f;
    r.magoff = __int_as_float(0x7fc00000);
    r.pad = 0.f;
    if (z > 0.f && z <= a.zmax_f) {
        // FP64 only where the integer part of (t_obs - t0)/h ~ 200 is split
        // off: f_obs keeps its full FP32 precision.
        const double x = (double)z * a.inv_dz;
        const int i = min((int)x, a.n_lut - 2);
        const double fr = x - i;
        const double t_obs = a.tlut[i] + fr * (a.tlut[i + 1] - a.tlut[i]);
        const double apos = (t_obs - a.t0) * a.inv_h;
        if (apos > 0.0) {
            r.m_obs = min((int)apos, a.n_t - 2);
            r.f_obs = (float)(apos - r.m_obs);
        }
        const float frf = (float)fr;
        const float gz = fmaf(frf, a.glut[i + 1] - a.glut[i], a.glut[i]);
        const float lm = a.params[10 * a.G_stride + g];
        // Sec. 2.2: m_q = M'_q + Dmod(z) - 2.5 log10(1+z); rest frame: M_q alone
        r.magoff = a.rest ? -2.5f * lm : fmaf(-2.5f, lm, gz) + (5.f * log10f(z) - 2.5f * log10f(1.f + z));
    }
    out[gl] = r;
}

// Sec. 3.2, Eq. agedep_mdf: mean lgZ of the MDF for age bin i, mua_i p5 +
// mub_i p7 (linear in log age, or the T_erf transition from mu_young to
// mu_old; the per-age coefficients are tabulated per context).
__device__ __forceinline__ float mdf_mean_at(const WArgs &a, const float *p, int i) {
    return fmaf(p[7], __ldg(a.mub + i), __ldg(a.mua + i) * p[5]);
}

// Sec. 3.3, Eq. nebsed: this lane's log U bin probability (lane k < n_u holds
// P_neb(k), the triweight CDF difference over the bin's edges, in the same
// S-form as the metallicity bins), and the galaxy's non-zero range [lo, hi]
// (empty: {n_u, -1}).  An invalid galaxy gets {1, 0, ...} and range {0, 0}.
__device__ __forceinline__ float pneb_lane(const WArgs &a, const float *p, bool valid, int lane, int &lo, int &hi) {
    float pu = 0.f;
    if (!valid) {
        lo = hi = 0;
        return lane == 0 ? 1.f : 0.f;
    }
    if (lane < a.n_u) {
        const float isu = 1.f / p[13];
        const bool first = lane == 0, last = lane == a.n_u - 1;
        const float xl = first ? -1e30f : (__ldg(a.uedge + lane) - p[12]) * isu;
        const float xh = last ? 1e30f : (__ldg(a.uedge + lane + 1) - p[12]) * isu;
        const float sl = first ? 0.f : mdf_s<DSPS_MDF_TRIWEIGHT>(xl);
        const float sh = last ? 0.f : mdf_s<DSPS_MDF_TRIWEIGHT>(xh);
        pu = sh - sl;
        if (xl <= 0.f && xh > 0.f) pu += 1.f;
    }
    const unsigned nzm = __ballot_sync(0xffffffffu, pu != 0.f);
    lo = nzm ? __ffs(nzm) - 1 : a.n_u;
    hi = nzm ? 31 - __clz(nzm) : -1;
    return pu;
}

template <int MODE, int SFH, int MDF, bool NEB>
__global__ void __launch_bounds__(256, NEB ? 3 : 4) weights_kernel(WArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    const size_t per_warp = weights_smem_per_warp(a.n_t, a.n_age);
    const SfhSmem sm = sfh_smem(smem_raw + per_warp * warp, a.n_t, a.n_age);

    const int64_t gi = (int64_t)blockIdx.x * nwarps + warp;
    if (gi >= a.n) return;
    const int64_t gl = a.perm ? (int64_t)a.perm[gi] : gi;
    const int64_t g = a.g_begin + gl;

    constexpr int NP = NEB ? NPAR_MAX : NPAR;
    constexpr int NU = NEB ? MAX_NU : 1;
    float mine = lane < NP ? a.params[(int64_t)lane * a.G_stride + g] : 0.f;
    float p[NP];
#pragma unroll
    for (int r = 0; r < NP; ++r) p[r] = __shfl_sync(0xffffffffu, mine, r);

    const float z = p[11], sig = p[6];
    constexpr bool TAB = SFH == DSPS_SFH_TABLE;   // rows 0..4 unused
    bool valid = __all_sync(0xffffffffu, isfinite(mine) || lane >= NP || (TAB && lane < 5));
    valid = valid && z > 0.f && z <= a.zmax_f && sig > 0.f && (TAB || p[0] > 0.f);
    if constexpr (NEB) valid = valid && p[13] > 0.f;
    const GalPrep gp = a.prep[gl];

    float msum = 0.f;
    float frac1 = 0.f;   // a one-age launch's fraction from the chunk's cache
    if (MODE == W_OMEGA_BF16X2_AGE1 && a.fcache_rd) {
        frac1 = valid ? a.fcache_rd[gi * a.n_age + a.age_lo] : 0.f;
        valid = valid && !isnan(frac1);
    } else {
        valid = sfh_stage<SFH>(a, p, g, valid, gp.m_obs, gp.f_obs, lane, sm, msum);
        if (MODE == W_OMEGA_BF16X2 && a.fcache_wr)
            for (int i = lane; i < a.n_age; i += 32) a.fcache_wr[gi * a.n_age + i] = valid ? sm.frac[i] : __int_as_float(0x7fc00000);
    }
    float *frac = sm.frac;
    // log U bin probabilities, in every lane's registers
    int u_lo = 0, u_hi = 0;
    float pu[NU];
    if constexpr (NEB) {
        const float pu_l = pneb_lane(a, p, valid, lane, u_lo, u_hi);
#pragma unroll
        for (int u = 0; u < NU; ++u) pu[u] = __shfl_sync(0xffffffffu, pu_l, u);
    } else {
        pu[0] = 1.f;
    }

    // 5-6. metallicity weights and output.
    const float inv_sig = 1.f / sig;
    const float mass = exp10f(p[10]);
    // redshift shift in grid steps (none for rest-frame filters)
    const float s_shift = valid && !a.rest ? log1pf(z) / a.dlnlam_f : 0.f;
    const int nz = a.n_z;
    if constexpr (MODE == W_OMEGA_BF16X2 || MODE == W_OMEGA_BF16X2_AGE1 || MODE == W_OMEGA_BF16X2_AB) {
        // AB: the same weights in the age-block order ka = i * KBLOCK + j (the
        // fused age-dependent dust forward), the mask holding one bit per age
        constexpr bool AB = MODE == W_OMEGA_BF16X2_AB;
        uint4 bm = make_uint4(0u, 0u, 0u, 0u);
        const int row_len = AB ? a.KA_pad : a.KZ_pad;
        __nv_bfloat16 *rh = a.whi + gi * row_len, *rl = a.wlo + gi * row_len;
        if constexpr (AB) {
            // Age-block order: lane j takes metallicity bin j (lanes >= n_z write
            // the zero columns) and the warp walks the ages, four at a time
            // (independent).  Lane j evaluates the CDF at its bin's upper edge
            // and takes the lower edge's from lane j - 1 (one CDF per weight, the
            // expressions of the metallicity-major loop below, so every weight is
            // the same number); age i's 32 columns are one coalesced 64-byte
            // store of hi and of lo, and a ballot gives the age's mask bit.
            const int j = lane;
            const bool jin = j < nz;
            const bool first = j == 0, last = j == nz - 1;
            const float ze_lo = jin && !first ? __ldg(a.zedge + j) : 0.f;
            const float ze_hi = jin && !last ? __ldg(a.zedge + j + 1) : 0.f;
            const float isg = valid ? inv_sig : 0.f;
            const int nblk = a.KA_pad / KBLOCK;
            unsigned wbits = 0u;   // mask bits of the current 32 ages (flushed into bm at word ends)
            auto flush = [&](int wi) {
                if (wi == 0) bm.x = wbits;
                else if (wi == 1) bm.y = wbits;
                else if (wi == 2) bm.z = wbits;
                else bm.w = wbits;
                wbits = 0u;
            };
            // two ages at a time in paired FP32 ops (the scalar operations, so the
            // same numbers); nblk is even (KA_pad is a multiple of 64)
            for (int i0 = 0; i0 < nblk; i0 += 4) {
#pragma unroll
                for (int c = 0; c < 4; c += 2) {
                    const int i = i0 + c;
                    if (i >= nblk) break;
                    const float2 fr = make_float2(valid && i < a.n_age ? frac[i] : 0.f,
                                                  valid && i + 1 < a.n_age ? frac[i + 1] : 0.f);
                    float2 mu = splat2(0.f);
                    if (valid) {
                        const int ia = min(i, a.n_age - 1), ib = min(i + 1, a.n_age - 1);
                        mu = fma2v(splat2(p[7]), make_float2(__ldg(a.mub + ia), __ldg(a.mub + ib)),
                                   mul2(make_float2(__ldg(a.mua + ia), __ldg(a.mua + ib)), splat2(p[5])));
                    }
                    const float2 ulv = mul2(sub2(splat2(ze_lo), mu), splat2(isg));
                    const float2 uhv = mul2(sub2(splat2(ze_hi), mu), splat2(isg));
                    const float ul[2] = {first ? -1e30f : ulv.x, first ? -1e30f : ulv.y};
                    const float uh[2] = {last ? 1e30f : uhv.x, last ? 1e30f : uhv.y};
                    float2 sh = mdf_s2<MDF>(make_float2(uh[0], uh[1]));
                    if (last) sh = splat2(0.f);
                    const float2 sl_up = make_float2(__shfl_up_sync(0xffffffffu, sh.x, 1),   // lane j - 1's upper edge
                                                     __shfl_up_sync(0xffffffffu, sh.y, 1));
                    const float2 d = sub2(sh, first ? splat2(0.f) : sl_up);
                    float pj[2] = {d.x, d.y};
#pragma unroll
                    for (int t = 0; t < 2; ++t)
                        if (ul[t] <= 0.f && uh[t] > 0.f) pj[t] += 1.f;
                    const float2 omv = mul2(fr, make_float2(pj[0], pj[1]));
                    const float2 om = jin ? omv : splat2(0.f);
                    // (the multiplier is 0 at the columns j >= n_z, and om finite)
                    const float2 w = mul2(om, make_float2(__ldg(a.wmul_ab + i * KBLOCK + j),
                                                          __ldg(a.wmul_ab + (i + 1) * KBLOCK + j)));
                    const __nv_bfloat162 h = __floats2bfloat162_rn(w.x, w.y);
                    const float2 r = sub2(w, __bfloat1622float2(h));
                    const __nv_bfloat162 l = __floats2bfloat162_rn(r.x, r.y);
                    rh[i * KBLOCK + j] = __low2bfloat16(h);
                    rh[(i + 1) * KBLOCK + j] = __high2bfloat16(h);
                    rl[i * KBLOCK + j] = __low2bfloat16(l);
                    rl[(i + 1) * KBLOCK + j] = __high2bfloat16(l);
                    const unsigned any0 = __ballot_sync(0xffffffffu, om.x != 0.f);
                    const unsigned any1 = __ballot_sync(0xffffffffu, om.y != 0.f);
                    wbits |= ((any0 != 0u ? 1u : 0u) | (any1 != 0u ? 2u : 0u)) << (i & 31);
                    if ((i & 31) == 30) flush(i >> 5);
                }
            }
            if (nblk & 31) flush((nblk - 1) >> 5);
        } else if constexpr (MODE == W_OMEGA_BF16X2_AGE1) {
            // One age bin i: lane j < n_z takes metallicity bin j (both edges'
            // CDFs, the arithmetic of the loop below), and the warp writes, in
            // every section, the 32-wide kz block holding (j, i) -- the weight
            // there, zeros elsewhere.  Those are the only blocks of the row that
            // the contraction reads: every row of the tile writes the same blocks,
            // and the tile's K-block mask holds no other bit.
            const int i = a.age_lo;
            float om = 0.f;
            if (lane < nz) {
                const float isg = valid ? inv_sig : 0.f;
                const float mu = valid ? mdf_mean_at(a, p, i) : 0.f;
                const bool first = lane == 0, last = lane == nz - 1;
                const float ul = first ? -1e30f : (__ldg(a.zedge + lane) - mu) * isg;
                const float uh = last ? 1e30f : (__ldg(a.zedge + lane + 1) - mu) * isg;
                const float sl = first ? 0.f : mdf_s<MDF>(ul);
                const float sh = last ? 0.f : mdf_s<MDF>(uh);
                float pj = sh - sl;
                if (ul <= 0.f && uh > 0.f) pj += 1.f;
                om = valid ? (a.fcache_rd ? frac1 : frac[i]) * pj : 0.f;
                if (om != 0.f) {
                    const int b = (lane * a.A_pad + i) / KBLOCK, wi = b >> 5;
                    const unsigned bit = 1u << (b & 31);
                    bm.x |= wi == 0 ? bit : 0u;
                    bm.y |= wi == 1 ? bit : 0u;
                    bm.z |= wi == 2 ? bit : 0u;
                    bm.w |= wi == 3 ? bit : 0u;
                }
            }
    #pragma unroll
            for (int u = 0; u < NU; ++u) {
                if (NEB && u >= a.n_u) break;
                for (int j = 0; j < nz; ++j) {
                    const float o = __shfl_sync(0xffffffffu, om, j);
                    const int kt = u * a.SEC + j * a.A_pad + i;                 // the weight's column
                    const int kz = u * a.SEC + ((j * a.A_pad + i) & ~(KBLOCK - 1)) + lane;
                    const float w = kz == kt ? (NEB ? o * pu[u] : o) * __ldg(a.wmul + kt) : 0.f;
                    const __nv_bfloat16 h = __float2bfloat16_rn(w);
                    rh[kz] = h;
                    rl[kz] = __float2bfloat16_rn(w - __bfloat162float(h));
                }
            }
        } else {
            // Metallicity-major kz = j * A_pad + i.  Lane g takes the ages 4g ..
            // 4g+3 and walks the metallicity bins upwards, carrying each age's CDF
            // at the bin's lower edge (the previous bin's upper edge): one CDF
            // evaluation per weight, the arithmetic of the age-major loop below.
            // The four weights of one (g, j) are consecutive in kz: one 8-byte
            // store each of hi and lo, a warp writing one contiguous run.
            //
            // An invalid galaxy or a padding age gets fraction 0 and finite
            // standardised edges, so its weights come out exactly 0.  For the
            // triweight, a group whose four bins all lie beyond +-3 standard
            // deviations is exactly 0 without evaluating the CDF (its carried
            // lower-edge value is then 0 below the support, -0 above).
            //
            // Each lane marks, in a 128-bit register mask, the kz blocks (KBLOCK
            // wide) where it wrote a non-zero weight; the warp's OR goes into the
            // tile's mask (grids of more than 128 blocks keep no mask).
            constexpr bool tri = MDF == DSPS_MDF_TRIWEIGHT;
            const float isg = valid ? inv_sig : 0.f;
            // with the nebular axis and preset tile ranges, only the sections
            // the tile's contraction reads are written (the others stay unread)
            const int2 ur = NEB && a.urange_pre ? a.urange[gi >> 7] : make_int2(0, NEB ? a.n_u - 1 : 0);
            for (int gq = lane; 4 * gq < a.A_pad; gq += 32) {
                float mu4[4], fr4[4], ulo[4], slo[4];
    #pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int i = 4 * gq + c;
                    mu4[c] = valid ? mdf_mean_at(a, p, min(i, a.n_age - 1)) : 0.f;
                    fr4[c] = valid && i < a.n_age && i >= a.age_lo && i < a.age_hi ? frac[i] : 0.f;
                    ulo[c] = -1e30f;
                    slo[c] = 0.f;
                }
                // metallicity bin j; LAST: the top bin, whose upper edge is +inf
                // (peeled off so that the other bins carry no selects for it)
                auto bin = [&](int j, auto last_c) {
                    constexpr bool last = decltype(last_c)::value;
                    const float ze = last ? 0.f : __ldg(a.zedge + j + 1);
                    // the four ages in two pairs (paired FP32, the scalar results)
                    float2 uh01 = splat2(1e30f), uh23 = splat2(1e30f);
                    if constexpr (!last) {
                        uh01 = mul2(sub2(splat2(ze), make_float2(mu4[0], mu4[1])), splat2(isg));
                        uh23 = mul2(sub2(splat2(ze), make_float2(mu4[2], mu4[3])), splat2(isg));
                    }
                    const float uh[4] = {uh01.x, uh01.y, uh23.x, uh23.y};
                    const float uh_max = fmaxf(fmaxf(uh[0], uh[1]), fmaxf(uh[2], uh[3]));
                    const float ul_min = fminf(fminf(ulo[0], ulo[1]), fminf(ulo[2], ulo[3]));
                    float om[4] = {0.f, 0.f, 0.f, 0.f};
                    bool nzg = false;
                    if (tri && (uh_max <= -3.f || ul_min >= 3.f)) {
    #pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            slo[c] = uh[c] > 0.f ? -0.f : 0.f;
                            ulo[c] = uh[c];
                        }
                    } else {
                        float2 sh01 = splat2(0.f), sh23 = splat2(0.f);
                        if constexpr (!last) {
                            sh01 = mdf_s2<MDF>(uh01);
                            sh23 = mdf_s2<MDF>(uh23);
                        }
                        const float2 d01 = sub2(sh01, make_float2(slo[0], slo[1]));
                        const float2 d23 = sub2(sh23, make_float2(slo[2], slo[3]));
                        float pj[4] = {d01.x, d01.y, d23.x, d23.y};
    #pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if (ulo[c] <= 0.f && uh[c] > 0.f) pj[c] += 1.f;
                        const float2 om01 = mul2(make_float2(fr4[0], fr4[1]), make_float2(pj[0], pj[1]));
                        const float2 om23 = mul2(make_float2(fr4[2], fr4[3]), make_float2(pj[2], pj[3]));
                        om[0] = om01.x;
                        om[1] = om01.y;
                        om[2] = om23.x;
                        om[3] = om23.y;
                        slo[0] = sh01.x;
                        slo[1] = sh01.y;
                        slo[2] = sh23.x;
                        slo[3] = sh23.y;
    #pragma unroll
                        for (int c = 0; c < 4; ++c) ulo[c] = uh[c];
                        nzg = (om[0] != 0.f) | (om[1] != 0.f) | (om[2] != 0.f) | (om[3] != 0.f);
                    }
                    const int kz = j * a.A_pad + 4 * gq;
                    if (nzg) {
                        const int b = kz / KBLOCK, wi = b >> 5;
                        const unsigned bit = 1u << (b & 31);
                        bm.x |= wi == 0 ? bit : 0u;
                        bm.y |= wi == 1 ? bit : 0u;
                        bm.z |= wi == 2 ? bit : 0u;
                        bm.w |= wi == 3 ? bit : 0u;
                    }
                    // one section per log U bin: omega_ij P_neb(u) at kz + u SEC
    #pragma unroll
                    for (int u = 0; u < NU; ++u) {
                        if (NEB && u >= a.n_u) break;
                        const int kzu = kz + u * a.SEC;
                        if (NEB && (u < ur.x || u > ur.y)) continue;   // a section the tile does not read
                        if (!nzg || (NEB && pu[u] == 0.f)) {   // all four zero, or outside the log U support
                            *reinterpret_cast<uint2 *>(rh + kzu) = make_uint2(0u, 0u);
                            *reinterpret_cast<uint2 *>(rl + kzu) = make_uint2(0u, 0u);
                            continue;
                        }
                        const float4 wm = __ldg(reinterpret_cast<const float4 *>(a.wmul + kzu));
                        float o[4];
    #pragma unroll
                        for (int c = 0; c < 4; ++c) o[c] = NEB ? om[c] * pu[u] : om[c];
                        const float2 w01 = mul2(make_float2(o[0], o[1]), make_float2(wm.x, wm.y));
                        const float2 w23 = mul2(make_float2(o[2], o[3]), make_float2(wm.z, wm.w));
                        const __nv_bfloat162 h01 = __floats2bfloat162_rn(w01.x, w01.y);
                        const __nv_bfloat162 h23 = __floats2bfloat162_rn(w23.x, w23.y);
                        const float2 r01 = sub2(w01, __bfloat1622float2(h01)), r23 = sub2(w23, __bfloat1622float2(h23));
                        const __nv_bfloat162 l01 = __floats2bfloat162_rn(r01.x, r01.y);
                        const __nv_bfloat162 l23 = __floats2bfloat162_rn(r23.x, r23.y);
                        uint2 hv, lv;
                        hv.x = *reinterpret_cast<const unsigned *>(&h01);
                        hv.y = *reinterpret_cast<const unsigned *>(&h23);
                        lv.x = *reinterpret_cast<const unsigned *>(&l01);
                        lv.y = *reinterpret_cast<const unsigned *>(&l23);
                        *reinterpret_cast<uint2 *>(rh + kzu) = hv;
                        *reinterpret_cast<uint2 *>(rl + kzu) = lv;
                    }
                };
                for (int j = 0; j + 1 < nz; ++j) bin(j, std::false_type{});
                bin(nz - 1, std::true_type{});
            }
            // padding columns [n_z * A_pad, SEC) of every written section but
            // the last, then [(n_u - 1) * SEC + n_z * A_pad, KZ_pad)
            for (int u = ur.x; u + 1 < (NEB ? a.n_u : 1) && u <= ur.y; ++u)
                for (int kz = u * a.SEC + nz * a.A_pad + 4 * lane; kz < (u + 1) * a.SEC; kz += 128) {
                    *reinterpret_cast<uint2 *>(rh + kz) = make_uint2(0u, 0u);
                    *reinterpret_cast<uint2 *>(rl + kz) = make_uint2(0u, 0u);
                }
            if (ur.y >= (NEB ? a.n_u : 1) - 1)
                for (int kz = ((NEB ? a.n_u : 1) - 1) * a.SEC + nz * a.A_pad + 4 * lane; kz < a.KZ_pad; kz += 128) {
                    *reinterpret_cast<uint2 *>(rh + kz) = make_uint2(0u, 0u);
                    *reinterpret_cast<uint2 *>(rl + kz) = make_uint2(0u, 0u);
                }
        }
        bm.x = __reduce_or_sync(0xffffffffu, bm.x);
        bm.y = __reduce_or_sync(0xffffffffu, bm.y);
        bm.z = __reduce_or_sync(0xffffffffu, bm.z);
        bm.w = __reduce_or_sync(0xffffffffu, bm.w);
        if (a.trange && valid) {
            const int64_t t = gi >> 7;
            if (lane < a.kmw && a.kmw <= 4) {
                const unsigned v = lane == 0 ? bm.x : lane == 1 ? bm.y : lane == 2 ? bm.z : bm.w;
                if (v) atomicOr(a.kmask + t * a.kmw + lane, v);
            }
            if (lane == 0) {
                const int i0 = (int)floorf(s_shift);
                atomicMin(&a.trange[t].x, i0);
                atomicMax(&a.trange[t].y, i0);
                atomicMin(&a.urange[t].x, u_lo);
                atomicMax(&a.urange[t].y, u_hi);
            }
        }
    } else if constexpr (NEB) {
        // Age-major k = (i * n_z + j) * n_u + u: each lane takes (i, j) pairs,
        // the metallicity bin probability from its two edges' CDFs, and writes
        // its n_u log U bins.
        for (int ij = lane; ij < a.n_age * nz; ij += 32) {
            const int i = ij / nz, j = ij - i * nz;
            float om = 0.f;
            if (valid) {
                const float mu_i = mdf_mean_at(a, p, i);
                const float ul = (__ldg(a.zedge + j) - mu_i) * inv_sig;
                const float uh = j == nz - 1 ? 1e30f : (__ldg(a.zedge + j + 1) - mu_i) * inv_sig;
                const float sl = j == 0 ? 0.f : mdf_s<MDF>(ul);
                const float sh = j == nz - 1 ? 0.f : mdf_s<MDF>(uh);
                float pj = sh - sl;
                if (ul <= 0.f && uh > 0.f) pj += 1.f;
                om = i >= a.age_lo && i < a.age_hi ? frac[i] * pj : 0.f;
            }
#pragma unroll
            for (int u = 0; u < NU; ++u) {
                if (u >= a.n_u) break;
                const int k = ij * a.n_u + u;
                if (MODE == W_MSUN) a.w_msun[gi * a.K + k] = mass * (om * pu[u]);
                else a.w32[gi * a.K_pad + k] = om * pu[u];
            }
        }
        if (MODE != W_MSUN)
            for (int k = a.K + lane; k < a.K_pad; k += 32) a.w32[gi * a.K_pad + k] = 0.f;
    } else {
        // Age-major k, four consecutive k per lane.  The CDF at the upper edge
        // of bin j is the lower edge of bin j+1, and the outer edges (-inf,
        // +inf) need no evaluation, so each k costs about one CDF evaluation.
        const int kend = MODE == W_MSUN ? a.K : a.K_pad;
        const int di = 128 / nz, dj = 128 % nz;
        int k = 4 * lane;
        int i0 = k / nz, j0 = k - i0 * nz;
        for (; k < kend; k += 128) {
            float om[4];
            int i = i0, j = j0;
            float mu_i = mdf_mean_at(a, p, min(i, a.n_age - 1));
            float u_lo = (__ldg(a.zedge + j) - mu_i) * inv_sig;
            float s_lo = j == 0 ? 0.f : mdf_s<MDF>(u_lo);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                om[c] = 0.f;
                if (k + c < a.K && valid) {
                    const bool last = j == nz - 1;
                    const float u_hi = last ? 1e30f : (__ldg(a.zedge + j + 1) - mu_i) * inv_sig;
                    const float s_hi = last ? 0.f : mdf_s<MDF>(u_hi);
                    float pj = s_hi - s_lo;
                    if (u_lo <= 0.f && u_hi > 0.f) pj += 1.f;
                    om[c] = i >= a.age_lo && i < a.age_hi ? frac[i] * pj : 0.f;
                    s_lo = s_hi;
                    u_lo = u_hi;
                }
                if (++j == nz) {   // next age row: its lower edge is -inf
                    j = 0;
                    ++i;
                    mu_i = mdf_mean_at(a, p, min(i, a.n_age - 1));
                    u_lo = -1e30f;
                    s_lo = 0.f;
                }
            }
            if (MODE == W_MSUN) {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (k + c < a.K) a.w_msun[gi * a.K + k + c] = mass * om[c];
            } else if (k < a.K_pad) {
                *reinterpret_cast<float4 *>(a.w32 + gi * a.K_pad + k) = make_float4(om[0], om[1], om[2], om[3]);
            }
            i0 += di;
            j0 += dj;
            if (j0 >= nz) { j0 -= nz; ++i0; }
        }
    }

    if (lane == 0) {
        if (a.gidx) a.gidx[gi] = (int)gl;
        if (MODE == W_OMEGA_F32 && a.trange && valid) {   // the FP32 form's band ranges (no K masks)
            const int i0 = (int)floorf(s_shift);
            atomicMin(&a.trange[gi >> 7].x, i0);
            atomicMax(&a.trange[gi >> 7].y, i0);
        }
        // the dust of this call: rows 8, 9, or with age-dependent dust the
        // group's Av = (1 - T) Av_young + T Av_old, delta likewise (Sec. 3.4.1)
        float Av = p[8], dl = p[9];
        if (a.dust_row_old >= 0 && MODE != W_MSUN) {
            const float avo = a.params[(int64_t)a.dust_row_old * a.G_stride + g];
            const float dlo = a.params[(int64_t)(a.dust_row_old + 1) * a.G_stride + g];
            if (!isfinite(avo) || !isfinite(dlo)) valid = false;
            Av = group_dust_value(a.dust_T, p[8], avo);
            dl = group_dust_value(a.dust_T, p[9], dlo);
        }
        if (!valid) atomicOr(a.err, DERR_PARAM);
        if (MODE == W_OMEGA_BF16X2_AB || a.aux_yo) {
            // the young and old dust values; each group's curve is formed from
            // them in the one-launch contraction (agedep_tc.cu, phot_simt.cu)
            float *ax = a.aux + gi * AUX_STRIDE;
            ax[0] = p[8];
            ax[1] = p[9];
            ax[2] = s_shift;
            ax[3] = valid ? 1.f : 0.f;
            ax[4] = a.dust_row_old >= 0 ? a.params[(int64_t)a.dust_row_old * a.G_stride + g] : p[8];
            ax[5] = a.dust_row_old >= 0 ? a.params[(int64_t)(a.dust_row_old + 1) * a.G_stride + g] : p[9];
            ax[6] = ax[7] = 0.f;
            a.magoff[gi] = valid ? gp.magoff : __int_as_float(0x7fc00000);
        } else if (MODE != W_MSUN) {
            float *ax = a.aux + gi * AUX_STRIDE;
            store_dust_aux(ax, Av, dl, a.dust_law, a.dust_bump);
            ax[2] = s_shift;
            ax[3] = valid ? 1.f : 0.f;
            a.magoff[gi] = valid ? gp.magoff : __int_as_float(0x7fc00000);
        }
    }
}


// ---------------------------------------------------------------------------
// Adjoint of the weights (reverse of stages 6 .. 2).  Input: What[r][k], the
// adjoint contraction against the metallicity-differenced SSP block (scaled
// by 2^-E'_k in the tensor form: multiplied back by wmul_d here).  Output:
// param_bar rows 0..7 (SFH, mdf_mu, mdf_sigma, slope).
// ---------------------------------------------------------------------------

// Sec. 3.1: dSFR/dp_k at time t (same parametrisation as sfr_f), k = 0..4.
template <int SFH>
__device__ __forceinline__ void sfr_grad_f(const float *p, float t, float (&gr)[5]) {
#pragma unroll
    for (int k = 0; k < 5; ++k) gr[k] = 0.f;
    if constexpr (SFH == DSPS_SFH_DELAYED_TAU) {
        const float sv = t * expf(-t / p[0]);
        gr[0] = sv * t / (p[0] * p[0]);
        return;
    }
    const float lr = logf(t / p[0]);
    const float ra = expf(-p[1] * lr), rf = expf(-p[2] * lr);
    const float ms = 1.f / (ra + rf);
    const float invD2 = ms * ms;
    const float zq = (t - (p[3] - 0.9f)) * (1.f / 0.3f);
    const float P = terf_f(zq);
    const float fq = exp10f(-p[4] * P);
    gr[0] = -(p[1] * ra + p[2] * rf) / p[0] * invD2 * fq;
    gr[1] = lr * ra * invD2 * fq;
    gr[2] = lr * rf * invD2 * fq;
    gr[3] = ms * fq * p[4] * 2.302585093f * triweight_f(zq) * (1.f / 0.3f);
    gr[4] = -ms * fq * 2.302585093f * P;
}

// mdf_pdf of two points at once: the triweight in paired FP32 ops, z / 3
// taken as z times the FP32 1/3 (within 1.5 ulp of the quotient, against a
// correctly rounded division's dozen instructions), the Gaussian pair by pair.
template <int MDF>
__device__ __forceinline__ float mdf_pdf(float u);

template <int MDF>
__device__ __forceinline__ float2 mdf_pdf2(float2 z) {
    if constexpr (MDF != DSPS_MDF_TRIWEIGHT) {
        return make_float2(mdf_pdf<MDF>(z.x), mdf_pdf<MDF>(z.y));
    } else {
        const float2 q = mul2(z, splat2(1.f / 3.f));
        const float2 t = fma2v(make_float2(-q.x, -q.y), q, splat2(1.f));
        const float2 d = mul2(mul2(mul2(splat2(35.f / 96.f), t), t), t);
        return make_float2(z.x <= -3.f || z.x >= 3.f ? 0.f : d.x, z.y <= -3.f || z.y >= 3.f ? 0.f : d.y);
    }
}

template <int MDF>
__device__ __forceinline__ float mdf_pdf(float u) {
    if constexpr (MDF == DSPS_MDF_TRIWEIGHT) return triweight_f(u);
    else return gauss_pdf_f(u);
}

__host__ __device__ inline size_t weights_vjp_smem_per_warp(int n_t, int n_age) {
    return weights_smem_per_warp(n_t, n_age) + ((((size_t)n_t + (size_t)n_age) * 4 + 15) & ~(size_t)15);
}

template <int SFH, int MDF, bool NEB>
__global__ void __launch_bounds__(256, NEB ? 2 : 4) weights_vjp_kernel(WArgs a, const float *what, int scaled, float *pbar) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    unsigned char *base = smem_raw + weights_vjp_smem_per_warp(a.n_t, a.n_age) * warp;
    const SfhSmem sm = sfh_smem(base, a.n_t, a.n_age);
    float *fracbar = reinterpret_cast<float *>(base + weights_smem_per_warp(a.n_t, a.n_age));   // [n_age]
    float *sbar = fracbar + a.n_age;                                                            // [n_t]

    const int64_t gi = (int64_t)blockIdx.x * nwarps + warp;
    if (gi >= a.n) return;
    const int64_t gl = a.perm ? (int64_t)a.perm[gi] : gi;
    const int64_t g = a.g_begin + gl;
    constexpr int NP = NEB ? NPAR_MAX : NPAR;
    float mine = lane < NP ? a.params[(int64_t)lane * a.G_stride + g] : 0.f;
    float p[NP];
#pragma unroll
    for (int r = 0; r < NP; ++r) p[r] = __shfl_sync(0xffffffffu, mine, r);
    const float z = p[11], sig = p[6];
    constexpr bool TAB = SFH == DSPS_SFH_TABLE;   // rows 0..4 unused
    bool valid = __all_sync(0xffffffffu, isfinite(mine) || lane >= NP || (TAB && lane < 5));
    valid = valid && z > 0.f && z <= a.zmax_f && sig > 0.f && (TAB || p[0] > 0.f);
    if constexpr (NEB) valid = valid && p[13] > 0.f;
    const GalPrep gp = a.prep[gl];
    float msum = 0.f;
    valid = sfh_stage<SFH>(a, p, g, valid, gp.m_obs, gp.f_obs, lane, sm, msum);
    const float *frac = sm.frac;
    for (int i = lane; i < a.n_age; i += 32) fracbar[i] = 0.f;
    for (int n = lane; n < a.n_t; n += 32) sbar[n] = 0.f;
    __syncwarp();

    // reverse of stages 5-6, by parts: with dw_(i,e) = dLoss/domega_(i,e) -
    // dLoss/domega_(i,e-1) (dw_(i,0) = dLoss/domega_(i,0)) from the adjoint
    // contraction against the differenced block,
    //   dLoss/dfrac_i = sum_e dw_(i,e) P(Z >= edge e | i)
    //   dLoss/dmu_i   = frac_i / sigma sum_{e>=1} dw_(i,e) pdf(u_e)
    //   dLoss/dsigma  = sum_i frac_i / sigma sum_{e>=1} dw_(i,e) pdf(u_e) u_e
    // (the MDF bin probabilities are CDF differences, Sec. 3.2 / Appendix B),
    // and dLoss/dp5, dLoss/dp7 = sum_i dLoss/dmu_i (mua_i, mub_i).
    const float inv_sig = 1.f / sig;
    const int nz = a.n_z;
    float mu_bar = 0.f, sig_bar = 0.f, slope_bar = 0.f;
    // Metallicity-major What (kz = e * A_pad + i): lane g takes the ages 4g ..
    // 4g+3 and walks the edges e upwards with one float4 load per edge, each
    // age's dLoss/dfrac in a register.  Beyond the triweight's support the
    // terms are exact: above it (u >= 3 for the four ages, and so for every
    // higher edge) P(Z >= edge) and the density vanish, so the walk stops;
    // below it (u <= -3) P(Z >= edge) = 1 and the density vanishes.
    constexpr bool tri = MDF == DSPS_MDF_TRIWEIGHT;
    const float *wrow = what + gi * a.KZ_pad;
    float ubar_mean = 0.f, ubar_sig = 0.f;
    if constexpr (NEB) {
        // With a nebular axis the adjoint rows are (section u, edge e, age i):
        // D2_u = D_u - D_ref for u != u_ref and D_ref itself, D_u the
        // metallicity difference of dLoss/domega in log U bin u.  The walk
        // takes D_u = D2_u + D2_ref over the galaxy's log U support, uses
        // dw = sum_u P_u D_u where the MDF adjoint used dw, and accumulates
        //   hd_u = sum_i frac_i sum_e P(Z >= edge e | i) D2_(u, e, i)
        //        = dLoss/dP_u - dLoss/dP_ref,
        // which gives the log U gradients (the P_u sum to 1, so the reference
        // bin drops out of sum_u dLoss/dP_u dP_u/dtheta).
        int u_lo, u_hi;
        const float pu_l = pneb_lane(a, p, valid, lane, u_lo, u_hi);
        float pu[MAX_NU], hd[MAX_NU];
#pragma unroll
        for (int u = 0; u < MAX_NU; ++u) {
            pu[u] = __shfl_sync(0xffffffffu, pu_l, u);
            hd[u] = 0.f;
        }
        const int uref = a.u_ref;
        auto ld4 = [&](int kz) {
            float4 v = *reinterpret_cast<const float4 *>(wrow + kz);
            if (scaled) {
                const float4 m = __ldg(reinterpret_cast<const float4 *>(a.wmul + kz));
                v.x *= m.x;
                v.y *= m.y;
                v.z *= m.z;
                v.w *= m.w;
            }
            return v;
        };
        for (int gq = lane; 4 * gq < a.A_pad && valid; gq += 32) {
            float mu4[4], xl4[4], xa4[4], fr4[4], fb4[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int i = 4 * gq + c;
                xa4[c] = __ldg(a.mua + min(i, a.n_age - 1));
                xl4[c] = __ldg(a.mub + min(i, a.n_age - 1));
                mu4[c] = fmaf(p[7], xl4[c], xa4[c] * p[5]);
                fr4[c] = i < a.n_age ? frac[i] : 0.f;
                fb4[c] = 0.f;
            }
            for (int e = 0; e < nz; ++e) {
                const int kz = e * a.A_pad + 4 * gq;
                float u[4], se[4];   // standardised edge, P(Z >= edge e | i)
                bool dens = false;   // some age's density may be non-zero at the edge
                if (e == 0) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) u[c] = se[c] = 1.f;
                } else {
                    const float ze = __ldg(a.zedge + e);
#pragma unroll
                    for (int c = 0; c < 4; ++c) u[c] = (ze - mu4[c]) * inv_sig;
                    if (tri && fminf(fminf(u[0], u[1]), fminf(u[2], u[3])) >= 3.f) break;
                    if (tri && fmaxf(fmaxf(u[0], u[1]), fmaxf(u[2], u[3])) <= -3.f) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) se[c] = 1.f;
                    } else {
                        dens = true;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float sv = mdf_s<MDF>(u[c]);
                            se[c] = u[c] > 0.f ? -sv : 1.f - sv;
                        }
                    }
                }
                // every section's load issued before any is used (the loads
                // are independent; one after another they leave the warp
                // waiting on memory latency once per section)
                const float4 r = ld4(uref * a.SEC + kz);
                float4 vs[MAX_NU];
#pragma unroll
                for (int uu = 0; uu < MAX_NU; ++uu) {
                    const bool live = uu < a.n_u && uu >= u_lo && uu <= u_hi && uu != uref;
                    vs[uu] = live ? *reinterpret_cast<const float4 *>(wrow + uu * a.SEC + kz)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                float dw[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int uu = 0; uu < MAX_NU; ++uu) {
                    if (uu >= a.n_u) break;
                    if (uu < u_lo || uu > u_hi) continue;
                    if (uu == uref) {
                        dw[0] = fmaf(pu[uu], r.x, dw[0]);
                        dw[1] = fmaf(pu[uu], r.y, dw[1]);
                        dw[2] = fmaf(pu[uu], r.z, dw[2]);
                        dw[3] = fmaf(pu[uu], r.w, dw[3]);
                        continue;
                    }
                    float4 v = vs[uu];
                    if (scaled) {
                        const float4 m = __ldg(reinterpret_cast<const float4 *>(a.wmul + uu * a.SEC + kz));
                        v.x *= m.x;
                        v.y *= m.y;
                        v.z *= m.z;
                        v.w *= m.w;
                    }
                    dw[0] = fmaf(pu[uu], v.x + r.x, dw[0]);
                    dw[1] = fmaf(pu[uu], v.y + r.y, dw[1]);
                    dw[2] = fmaf(pu[uu], v.z + r.z, dw[2]);
                    dw[3] = fmaf(pu[uu], v.w + r.w, dw[3]);
                    hd[uu] = fmaf(fr4[0] * se[0], v.x,
                                  fmaf(fr4[1] * se[1], v.y, fmaf(fr4[2] * se[2], v.z, fmaf(fr4[3] * se[3], v.w, hd[uu]))));
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) fb4[c] = fmaf(dw[c], se[c], fb4[c]);
                if (!dens) continue;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float t = fr4[c] * dw[c] * mdf_pdf<MDF>(u[c]) * inv_sig;
                    mu_bar = fmaf(t, xa4[c], mu_bar);
                    sig_bar = fmaf(t, u[c], sig_bar);
                    slope_bar = fmaf(t, xl4[c], slope_bar);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (4 * gq + c < a.n_age) fracbar[4 * gq + c] = fb4[c];
        }
        // dP_u/du_mean = -(pdf(x_hi) - pdf(x_lo)) / u_sigma, dP_u/du_sigma =
        // -(pdf(x_hi) x_hi - pdf(x_lo) x_lo) / u_sigma over the bin's edges
        // (outer edges at +-infinity contribute nothing)
        const float isu = valid ? 1.f / p[13] : 0.f;
#pragma unroll
        for (int uu = 0; uu < MAX_NU; ++uu) {
            float h = hd[uu];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) h += __shfl_xor_sync(0xffffffffu, h, off);
            if (uu >= a.n_u || uu == uref) continue;
            const bool first = uu == 0, last = uu == a.n_u - 1;
            const float xl = first ? 0.f : (__ldg(a.uedge + uu) - p[12]) * isu;
            const float xh = last ? 0.f : (__ldg(a.uedge + uu + 1) - p[12]) * isu;
            const float dl = first ? 0.f : triweight_f(xl), dh = last ? 0.f : triweight_f(xh);
            ubar_mean = fmaf(h, -(dh - dl) * isu, ubar_mean);
            ubar_sig = fmaf(h, -(dh * xh - dl * xl) * isu, ubar_sig);
        }
    }
    for (int gq = lane; !NEB && 4 * gq < a.A_pad && valid; gq += 32) {
        float mu4[4], xl4[4], xa4[4], fr4[4], fb4[4];   // xa4, xl4: d mu_i / d p5, d p7
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = 4 * gq + c;
            xa4[c] = __ldg(a.mua + min(i, a.n_age - 1));
            xl4[c] = __ldg(a.mub + min(i, a.n_age - 1));
            mu4[c] = fmaf(p[7], xl4[c], xa4[c] * p[5]);
            fr4[c] = i < a.n_age ? frac[i] : 0.f;
            fb4[c] = 0.f;
        }
        // the next edge's adjoint row entries (and multipliers) are loaded one
        // edge ahead, so that the loads overlap the current edge's arithmetic
        float4 wv_next = *reinterpret_cast<const float4 *>(wrow + 4 * gq);
        float4 m_next = scaled ? __ldg(reinterpret_cast<const float4 *>(a.wmul + 4 * gq)) : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int e = 0; e < nz; ++e) {
            const int kz = e * a.A_pad + 4 * gq;
            float4 wv = wv_next;
            const float4 m = m_next;
            if (e + 1 < nz) {
                wv_next = *reinterpret_cast<const float4 *>(wrow + kz + a.A_pad);
                if (scaled) m_next = __ldg(reinterpret_cast<const float4 *>(a.wmul + kz + a.A_pad));
            }
            float2 u01 = splat2(0.f), u23 = splat2(0.f);   // the four ages in two pairs
            if (e > 0) {
                const float ze = __ldg(a.zedge + e);
                u01 = mul2(sub2(splat2(ze), make_float2(mu4[0], mu4[1])), splat2(inv_sig));
                u23 = mul2(sub2(splat2(ze), make_float2(mu4[2], mu4[3])), splat2(inv_sig));
                if (tri && fminf(fminf(u01.x, u01.y), fminf(u23.x, u23.y)) >= 3.f) break;
            }
            const float u[4] = {u01.x, u01.y, u23.x, u23.y};
            if (scaled) {
                wv.x *= m.x;
                wv.y *= m.y;
                wv.z *= m.z;
                wv.w *= m.w;
            }
            const float dw[4] = {wv.x, wv.y, wv.z, wv.w};
            if (e == 0 || (tri && fmaxf(fmaxf(u[0], u[1]), fmaxf(u[2], u[3])) <= -3.f)) {
#pragma unroll
                for (int c = 0; c < 4; ++c) fb4[c] += dw[c];
                continue;
            }
            const float2 sv01 = mdf_s2<MDF>(u01), sv23 = mdf_s2<MDF>(u23);
            const float2 om01 = sub2(splat2(1.f), sv01), om23 = sub2(splat2(1.f), sv23);
            const float2 se01 = make_float2(u01.x > 0.f ? -sv01.x : om01.x, u01.y > 0.f ? -sv01.y : om01.y);
            const float2 se23 = make_float2(u23.x > 0.f ? -sv23.x : om23.x, u23.y > 0.f ? -sv23.y : om23.y);
            const float2 fb01 = fma2v(make_float2(dw[0], dw[1]), se01, make_float2(fb4[0], fb4[1]));
            const float2 fb23 = fma2v(make_float2(dw[2], dw[3]), se23, make_float2(fb4[2], fb4[3]));
            fb4[0] = fb01.x;
            fb4[1] = fb01.y;
            fb4[2] = fb23.x;
            fb4[3] = fb23.y;
            const float2 t01 = mul2(mul2(mul2(make_float2(fr4[0], fr4[1]), make_float2(dw[0], dw[1])), mdf_pdf2<MDF>(u01)),
                                    splat2(inv_sig));
            const float2 t23 = mul2(mul2(mul2(make_float2(fr4[2], fr4[3]), make_float2(dw[2], dw[3])), mdf_pdf2<MDF>(u23)),
                                    splat2(inv_sig));
            const float t[4] = {t01.x, t01.y, t23.x, t23.y};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                mu_bar = fmaf(t[c], xa4[c], mu_bar);
                sig_bar = fmaf(t[c], u[c], sig_bar);
                slope_bar = fmaf(t[c], xl4[c], slope_bar);
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (4 * gq + c < a.n_age) fracbar[4 * gq + c] = fb4[c];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        mu_bar += __shfl_xor_sync(0xffffffffu, mu_bar, off);
        sig_bar += __shfl_xor_sync(0xffffffffu, sig_bar, off);
        slope_bar += __shfl_xor_sync(0xffffffffu, slope_bar, off);
    }
    __syncwarp();

    // reverse of the normalisation frac_i = B_i / sum_i B_i
    float dot = 0.f;
    for (int i = lane; i < a.n_age; i += 32) dot = fmaf(fracbar[i], frac[i], dot);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, off);
    const float inv_m = valid ? 1.f / msum : 0.f;

    // reverse of stages 3-4: each bin integral is linear in the node SFRs.
    //  (a) the partial intervals at each bin's two edges (a few shared atomics
    //      per bin);
    //  (b) the whole intervals strictly inside bin i, em[i+1] < m < em[i]:
    //      each lane finds the bin of each of its intervals by bisection on
    //      the non-increasing em[], and each node takes half of the weight of
    //      both intervals it bounds.
    const float h = a.h_f;
    float *bbin = sm.bmass;   // dLoss/dB_i (the bin masses are not needed again)
    float *cf = sm.itg;       // weight of each whole interval (likewise)
    for (int i = lane; i < a.n_age; i += 32) {
        const float bb = valid ? (fracbar[i] - dot) * inv_m : 0.f;
        bbin[i] = bb;
        const int mi = sm.em[i], mo = sm.em[i + 1];
        const float ri = sm.er[i], ro = sm.er[i + 1];
        if (!valid || mi < 0 || bb == 0.f) continue;
        auto add = [&](int m, float len, float rbar) {
            atomicAdd(sbar + m, bb * len * (1.f - rbar));
            atomicAdd(sbar + m + 1, bb * len * rbar);
        };
        if (mo < 0) {
            add(mi, ri * h, 0.5f * ri);
        } else if (mi == mo) {
            add(mi, __ldg(a.bwidth + i), 0.5f * (ri + ro));
        } else {
            add(mo, mi == mo + 1 ? __ldg(a.bwidth + i) - ri * h : (1.f - ro) * h, 0.5f * (ro + 1.f));
            add(mi, ri * h, 0.5f * ri);
        }
    }
    __syncwarp();
    for (int m = lane; m < a.n_t - 1; m += 32) {
        float v = 0.f;
        if (valid) {
            int lo = 0, hi = a.n_age + 1;   // first edge with em <= m
            while (lo < hi) {
                const int md = (lo + hi) >> 1;
                if (sm.em[md] <= m) hi = md;
                else lo = md + 1;
            }
            if (lo > 0 && lo <= a.n_age && sm.em[lo] < m) v = bbin[lo - 1] * h;
        }
        cf[m] = v;
    }
    __syncwarp();
    for (int n = lane; n < a.n_t; n += 32)
        sbar[n] += 0.5f * ((n > 0 ? cf[n - 1] : 0.f) + (n < a.n_t - 1 ? cf[n] : 0.f));
    __syncwarp();

    // reverse of stage 2: the SFR parameters (nodes after t_obs have no
    // adjoint), or for a tabulated history the node SFRs themselves
    float tb[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if constexpr (TAB) {
        const float nan = __int_as_float(0x7fc00000);
        for (int n = lane; n < a.n_t; n += 32)
            pbar[(int64_t)(a.grow_sfr + n) * a.G_stride + g] = valid ? (n <= gp.m_obs + 1 ? sbar[n] : 0.f) : nan;
    } else {
        for (int n = lane; n <= gp.m_obs + 1 && n < a.n_t && valid; n += 32) {
            float gr[5];
            sfr_grad_f<SFH>(p, fmaf((float)n, h, a.t0_f), gr);
#pragma unroll
            for (int q = 0; q < 5; ++q) tb[q] = fmaf(sbar[n], gr[q], tb[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) tb[q] += __shfl_xor_sync(0xffffffffu, tb[q], off);

    if (lane == 0) {
        const float nan = __int_as_float(0x7fc00000);
        const float out[8] = {tb[0], tb[1], tb[2], tb[3], tb[4], mu_bar, sig_bar, slope_bar};
#pragma unroll
        for (int q = 0; q < 8; ++q) pbar[(int64_t)q * a.G_stride + g] = valid ? out[q] : nan;
        if constexpr (NEB) {
            pbar[(int64_t)11 * a.G_stride + g] = valid ? ubar_mean : nan;
            pbar[(int64_t)12 * a.G_stride + g] = valid ? ubar_sig : nan;
        }
    }
}

WArgs make_wargs(const Ctx &c, const Workspace &w, const float *params, int64_t G_stride, int64_t g_begin, int64_t n) {
    WArgs a{};
    a.params = params;
    a.G_stride = G_stride;
    a.g_begin = g_begin;
    a.n = n;
    a.n_age = c.n_age;
    a.n_z = c.n_z;
    a.age_lo = 0;
    a.age_hi = c.n_age;
    a.dust_T = 0.f;
    a.dust_row_old = -1;
    a.n_u = c.n_u;
    a.SEC = c.SEC;
    a.u_ref = c.u_ref;
    a.npar = c.npar;
    a.row_sfr = c.row_sfr;
    a.grow_sfr = c.grow_sfr;
    a.rest = w.rest;
    a.uedge = c.d_uedge;
    a.K = c.K;
    a.K_pad = c.K_pad;
    a.A_pad = c.A_pad;
    a.KZ_pad = c.KZ_pad;
    a.n_t = c.n_t;
    a.sfh_model = c.opts.sfh_model;
    a.mdf_kernel = c.opts.mdf_kernel;
    a.dust_bump = c.opts.dust_bump;
    a.dust_law = c.opts.dust_law;
    a.n_lut = c.n_lut;
    a.t0 = c.t0;
    a.h = (c.t1 - c.t0) / (c.n_t - 1);
    a.inv_h = 1.0 / a.h;
    a.dz = c.dz_lut;
    a.inv_dz = 1.0 / c.dz_lut;
    a.zmax = c.opts.z_max;
    a.dlnlam = c.dlnlam;
    a.t0_f = (float)a.t0;
    a.h_f = (float)a.h;
    a.dlnlam_f = (float)a.dlnlam;
    a.logage = c.d_logage;
    a.mua = c.d_mua;
    a.mub = c.d_mub;
    a.einh = c.d_einh;
    a.bwidth = c.d_bwidth;
    a.zedge = c.d_zedge;
    a.tlut = c.d_tlut;
    a.glut = c.d_glut;
    a.wmul = c.d_wmul;
    a.wmul_ab = c.d_wmul_ab;
    a.KA_pad = c.KA_pad;
    a.w32 = w.w32;
    a.whi = w.whi;
    a.wlo = w.wlo;
    a.aux = w.aux;
    a.magoff = w.magoff;
    a.prep = w.prep;
    a.zmax_f = (float)c.opts.z_max;
    if ((double)a.zmax_f > c.opts.z_max) a.zmax_f = std::nextafter(a.zmax_f, -INFINITY);
    a.err = c.d_err;
    return a;
}

namespace {

// Launches K<SFH, MDF, NEB> for the context's model pair and grid.
template <template <int, int, bool> class L, bool NEB, typename... Args>
cudaError_t launch_models_n(const Ctx &c, Args... args) {
    const int sfh = c.opts.sfh_model, mdf = c.opts.mdf_kernel;
    if (sfh == DSPS_SFH_DELAYED_TAU)
        return mdf == DSPS_MDF_TRIWEIGHT ? L<DSPS_SFH_DELAYED_TAU, DSPS_MDF_TRIWEIGHT, NEB>::run(args...)
                                         : L<DSPS_SFH_DELAYED_TAU, DSPS_MDF_GAUSSIAN, NEB>::run(args...);
    if (sfh == DSPS_SFH_TABLE)
        return mdf == DSPS_MDF_TRIWEIGHT ? L<DSPS_SFH_TABLE, DSPS_MDF_TRIWEIGHT, NEB>::run(args...)
                                         : L<DSPS_SFH_TABLE, DSPS_MDF_GAUSSIAN, NEB>::run(args...);
    return mdf == DSPS_MDF_TRIWEIGHT ? L<DSPS_SFH_DPL_QUENCH, DSPS_MDF_TRIWEIGHT, NEB>::run(args...)
                                     : L<DSPS_SFH_DPL_QUENCH, DSPS_MDF_GAUSSIAN, NEB>::run(args...);
}
template <template <int, int, bool> class L, typename... Args>
cudaError_t launch_models(const Ctx &c, Args... args) {
    return c.n_u > 1 ? launch_models_n<L, true>(c, args...) : launch_models_n<L, false>(c, args...);
}

template <int SFH, int MDF, bool NEB>
struct VjpLaunch {
    static cudaError_t run(const WArgs &a, const float *what, int scaled, float *pbar, unsigned grid, size_t smem,
                           cudaStream_t s) {
        cudaFuncSetAttribute(weights_vjp_kernel<SFH, MDF, NEB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        weights_vjp_kernel<SFH, MDF, NEB><<<grid, 256, smem, s>>>(a, what, scaled, pbar);
        return cudaGetLastError();
    }
};

template <int MODE>
struct WeightsLaunch {
    template <int SFH, int MDF, bool NEB>
    struct L {
        static cudaError_t run(const WArgs &a, unsigned grid, size_t smem, cudaStream_t s) {
            cudaFuncSetAttribute(weights_kernel<MODE, SFH, MDF, NEB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
            weights_kernel<MODE, SFH, MDF, NEB><<<grid, 256, smem, s>>>(a);
            return cudaGetLastError();
        }
    };
};

}  // namespace

// The adjoint reads the per-galaxy scalars (w.prep) of the forward weights
// launch that preceded it on the same chunk.
cudaError_t launch_weights_vjp(const Ctx &c, const Workspace &w, const float *params, int64_t G_stride,
                               int64_t g_begin, int64_t n, bool sorted, bool scaled, float *param_bar,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    WArgs a = make_wargs(c, w, params, G_stride, g_begin, n);
    a.perm = sorted ? w.perm : nullptr;
    a.wmul = c.d_wmul_d;
    const int warps = 8;
    const size_t smem = weights_vjp_smem_per_warp(c.n_t, c.n_age) * warps;
    return launch_models<VjpLaunch>(c, a, static_cast<const float *>(w.w32), scaled ? 1 : 0, param_bar,
                                    (unsigned)((n + warps - 1) / warps), smem, s);
}

cudaError_t launch_weights(const Ctx &c, const Workspace &w, int mode, const float *params, int64_t G_stride,
                           int64_t g_begin, int64_t n, float *w_msun, cudaStream_t s, bool sorted,
                           const DustGroup *group, bool aux_yo) {
    if (n <= 0) return cudaSuccess;
    WArgs a = make_wargs(c, w, params, G_stride, g_begin, n);
    if (group) {
        a.age_lo = group->i0;
        a.age_hi = group->i1;
        a.dust_T = group->T;
        a.dust_row_old = c.row_dust_old;
    }
    if (mode == W_OMEGA_BF16X2_AB || aux_yo) a.dust_row_old = c.row_dust_old;   // both dust values into aux
    a.aux_yo = aux_yo ? 1 : 0;
    a.w_msun = w_msun;
    a.perm = sorted ? w.perm : nullptr;
    a.gidx = sorted ? w.gidx : nullptr;
    a.trange = sorted && mode != W_MSUN ? w.trange : nullptr;
    a.urange = w.urange;
    a.kmask = w.kmask;
    a.kmw = c.kmask_words;
    const int warps = 8;
    const size_t smem = weights_smem_per_warp(c.n_t, c.n_age) * warps;
    galaxy_prep_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, w.prep);
    const unsigned grid = (unsigned)((n + warps - 1) / warps);
    a.urange_pre = mode == W_OMEGA_BF16X2 && sorted && c.n_u > 1 && c.opts.band_skip ? 1 : 0;
    // a one-age dust group writes only its age's K blocks, which are all the
    // contraction reads when it skips by the tiles' K-block masks
    if (mode == W_OMEGA_BF16X2 && group && group->i1 - group->i0 == 1 && sorted && c.kmask_words <= 4 &&
        c.opts.band_skip)
        mode = W_OMEGA_BF16X2_AGE1;
    // the chunk's age fractions: cached by a multi-age group, read by one-age ones
    a.fcache_wr = w.fcache && w.fcache_mode == 1 && mode == W_OMEGA_BF16X2 && sorted ? w.fcache : nullptr;
    a.fcache_rd = w.fcache && w.fcache_mode == 2 && mode == W_OMEGA_BF16X2_AGE1 ? w.fcache : nullptr;
    switch (mode) {
    case W_MSUN: return launch_models<WeightsLaunch<W_MSUN>::L>(c, a, grid, smem, s);
    case W_OMEGA_F32: return launch_models<WeightsLaunch<W_OMEGA_F32>::L>(c, a, grid, smem, s);
    case W_OMEGA_BF16X2_AGE1: return launch_models<WeightsLaunch<W_OMEGA_BF16X2_AGE1>::L>(c, a, grid, smem, s);
    case W_OMEGA_BF16X2_AB:
        if (c.n_u > 1 || !c.KA_pad) return cudaErrorInvalidValue;
        return launch_models_n<WeightsLaunch<W_OMEGA_BF16X2_AB>::L, false>(c, a, grid, smem, s);
    default: return launch_models<WeightsLaunch<W_OMEGA_BF16X2>::L>(c, a, grid, smem, s);
    }
}

}  // namespace dsps
