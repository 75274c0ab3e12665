// epilogue.cuh -- per-element photometry epilogue shared by the FP32 SIMT and
// the tcgen05 contraction kernels.
//
// For galaxy g and rest-frame wavelength node n with composite luminosity
// S_gn (Eq. full_mdf, per unit formed mass):
//   u    = (lam_n / 5500 A)^(delta - 0.7)             power-law attenuation curve
//   c    = u + e D0_n                                  with the UV bump (Eq. uvbump):
//          D0_n the unit Drude profile at lam_n, e = (0.85 - 1.9 delta) / 4.05
//   F    = 10^(-0.4 Av c)                              Eq. (attenuation)
//   v_n  = S_gn F c_n / lam_n                          rest-grid trapezoid of dlam/lam
//   N_q += v_n T_q((1+z) lam_n)                        Eq. (restmag) in the observer frame
// The filters are tabulated on the SSP grid's ln-lambda spacing, so the
// observer-frame position of node n is grid index n + s, s = ln(1+z)/dlnlam,
// i0 = floor(s), f = s - i0, and T_q there is the 4-point Lagrange
// interpolation  sum_{d=-1..2} w_d(f) T[n + i0 + d]  (error O(dlnlam^4)).
// Regrouping the sum by grid index m gives
//   N_q = sum_m T_q[m] y_m,  y_m = sum_d w_d v_{m - i0 - d},
// which the kernels evaluate over a contiguous run of nodes [a, b) with the
// last three v kept in registers; at node n the row m = n + i0 - 1 is complete,
// and three closing rows b + i0 - 1, b + i0, b + i0 + 1 end the run.
// Table row t holds grid index m = t - 1 (one leading row for m = -1).
#pragma once
#include <cmath>

#include "dsps_internal.cuh"
#include "f32x2.cuh"

namespace dsps {

struct RowConst {
    float alpha, beta;
    float w[4];   // Lagrange weights of grid indices i0-1, i0, i0+1, i0+2
    int i0;
    bool valid;
    float e, ed;  // UV-bump amplitude / 4.05 and its delta derivative (0 without the bump)
};

__device__ __forceinline__ RowConst load_row_const(const float *aux, int64_t row, int64_t n_rows) {
    RowConst rc{0.f, 0.f, {0.f, 1.f, 0.f, 0.f}, 0, false, 0.f, 0.f};
    if (row < n_rows) {
        const float *ax = aux + row * AUX_STRIDE;
        rc.alpha = ax[0];
        rc.beta = ax[1];
        const float s = ax[2];
        const float fl = floorf(s);
        rc.i0 = (int)fl;
        const float f = s - fl;
        rc.w[0] = -f * (f - 1.f) * (f - 2.f) * (1.f / 6.f);
        rc.w[1] = (f + 1.f) * (f - 1.f) * (f - 2.f) * 0.5f;
        rc.w[2] = -(f + 1.f) * f * (f - 2.f) * 0.5f;
        rc.w[3] = (f + 1.f) * f * (f - 1.f) * (1.f / 6.f);
        rc.valid = ax[3] != 0.f;
        rc.e = ax[6];
        rc.ed = ax[7];
    }
    return rc;
}

// Sliding state of a run: the last three v (v_{n-1}, v_{n-2}, v_{n-3}).
struct Slide {
    float v1 = 0.f, v2 = 0.f, v3 = 0.f;
};

struct ColConst {
    float ell0, dell;          // log2(lam_n / 5500) = ell0 + n dell
    float kap0, kapmid, kapN;  // trapezoid weight / lambda at n = 0, interior, N-1
    int N;
    const float *bump;         // [N_pad] unit Drude profile D0(lam_n), or nullptr (no UV bump)
    const float *k0;           // [N_pad] k0(lam_n) / 4.05 (Eq. kzero), or nullptr (power-law stand-in)
};

// The tilted term of the attenuation curve at node n (ell = log2(lam_n / 5500)):
// k0_n / 4.05 (lam_n / lam_V)^delta with the paper's starburst curve (Eq.
// salim; rc.beta = delta), or the stand-in (lam_n / lam_V)^(delta - 0.7)
// (rc.beta = delta - 0.7).  Its delta derivative is the term times ell ln 2.
__device__ __forceinline__ float dust_pow(const ColConst &cc, const RowConst &rc, float ell, int n) {
    const float p = exp2f(rc.beta * ell);
    return cc.k0 ? __ldg(cc.k0 + n) * p : p;
}

// Attenuation curve A_lambda / Av at node n: u, plus the UV bump when on.
__device__ __forceinline__ float dust_curve(const ColConst &cc, const RowConst &rc, float u, int n) {
    return cc.bump ? fmaf(rc.e, __ldg(cc.bump + n), u) : u;
}

// Host: column constants of the context's wavelength grid (phot_simt.cu).
ColConst make_col_const(const Ctx &c);

__device__ __forceinline__ float col_kappa(const ColConst &cc, int n) {
    return n == 0 ? cc.kap0 : (n == cc.N - 1 ? cc.kapN : cc.kapmid);
}

// acc[q] += y T_q(row m) for the filters two at a time (paired FMAs: the
// scalar fmaf results, half the instructions)
__device__ __forceinline__ void acc_pair4(float *acc, float y, const float4 &t) {
    const float2 a = fma2v(splat2(y), make_float2(t.x, t.y), make_float2(acc[0], acc[1]));
    const float2 b = fma2v(splat2(y), make_float2(t.z, t.w), make_float2(acc[2], acc[3]));
    acc[0] = a.x;
    acc[1] = a.y;
    acc[2] = b.x;
    acc[3] = b.y;
}

template <int Q4>
__device__ __forceinline__ void acc_row(float (&acc)[4 * Q4], const float4 *__restrict__ tab, int m, float y) {
    const float4 *tp = tab + (size_t)m * Q4;
#pragma unroll
    for (int qq = 0; qq < Q4; ++qq) acc_pair4(acc + 4 * qq, y, __ldg(tp + qq));
}

// One node of the sliding sum: completes grid row m = n + i0 - 1 (table row n + i0).
template <int Q4>
__device__ __forceinline__ void epi_node(float (&acc)[4 * Q4], Slide &sl, float S, int n, const RowConst &rc,
                                         const ColConst &cc, const float4 *__restrict__ tab, int m_last) {
    const float ell = fmaf((float)n, cc.dell, cc.ell0);
    const float u = dust_pow(cc, rc, ell, n);
    const float F = exp2f(rc.alpha * dust_curve(cc, rc, u, n));
    const float v = S * F * col_kappa(cc, n);
    const float y = fmaf(rc.w[0], v, fmaf(rc.w[1], sl.v1, fmaf(rc.w[2], sl.v2, rc.w[3] * sl.v3)));
    sl.v3 = sl.v2;
    sl.v2 = sl.v1;
    sl.v1 = v;
    acc_row<Q4>(acc, tab, min(n + rc.i0, m_last), y);
}

// Nodes n and n + 1 (n even within a run of columns): the operations of two
// epi_node calls, paired where they do not depend on each other (f32x2.cuh:
// the same numbers); the two filter rows are then added in node order.
template <int Q4>
__device__ __forceinline__ void epi_node2(float (&acc)[4 * Q4], Slide &sl, float S0, float S1, int n,
                                          const RowConst &rc, const ColConst &cc, const float4 *__restrict__ tab,
                                          int m_last) {
    const float2 ell = fma2v(make_float2((float)n, (float)(n + 1)), splat2(cc.dell), splat2(cc.ell0));
    const float2 be = mul2(splat2(rc.beta), ell);
    float2 u = make_float2(exp2f(be.x), exp2f(be.y));
    if (cc.k0) u = mul2(make_float2(__ldg(cc.k0 + n), __ldg(cc.k0 + n + 1)), u);
    if (cc.bump) u = fma2v(splat2(rc.e), make_float2(__ldg(cc.bump + n), __ldg(cc.bump + n + 1)), u);
    const float2 ac = mul2(splat2(rc.alpha), u);
    const float2 F = make_float2(exp2f(ac.x), exp2f(ac.y));
    const float2 v = mul2(mul2(make_float2(S0, S1), F), make_float2(col_kappa(cc, n), col_kappa(cc, n + 1)));
    // y_n = w0 v_n + w1 v_n-1 + w2 v_n-2 + w3 v_n-3 and y_n+1 likewise, innermost term first
    float2 y = mul2(splat2(rc.w[3]), make_float2(sl.v3, sl.v2));
    y = fma2v(splat2(rc.w[2]), make_float2(sl.v2, sl.v1), y);
    y = fma2v(splat2(rc.w[1]), make_float2(sl.v1, v.x), y);
    y = fma2v(splat2(rc.w[0]), v, y);
    sl.v3 = sl.v1;
    sl.v2 = v.x;
    sl.v1 = v.y;
    acc_row<Q4>(acc, tab, min(n + rc.i0, m_last), y.x);
    acc_row<Q4>(acc, tab, min(n + 1 + rc.i0, m_last), y.y);
}

// The attenuation of node n, F = 10^(-0.4 Av c_n) (Eq. attenuation) with the
// curve of rc (c_n = u + e D0_n).
__device__ __forceinline__ float dust_factor(const ColConst &cc, const RowConst &rc, int n) {
    const float ell = fmaf((float)n, cc.dell, cc.ell0);
    const float u = dust_pow(cc, rc, ell, n);
    return exp2f(rc.alpha * dust_curve(cc, rc, u, n));
}

// One node of the sliding sum for a spectrum already attenuated (age-dependent
// dust: each group's curve applied before the groups are summed).
template <int Q4>
__device__ __forceinline__ void epi_node_plain(float (&acc)[4 * Q4], Slide &sl, float S, int n, const RowConst &rc,
                                               const ColConst &cc, const float4 *__restrict__ tab, int m_last) {
    const float v = S * col_kappa(cc, n);
    const float y = fmaf(rc.w[0], v, fmaf(rc.w[1], sl.v1, fmaf(rc.w[2], sl.v2, rc.w[3] * sl.v3)));
    sl.v3 = sl.v2;
    sl.v2 = sl.v1;
    sl.v1 = v;
    acc_row<Q4>(acc, tab, min(n + rc.i0, m_last), y);
}

// epi_node_plain for nodes n and n + 1, paired like epi_node2.
template <int Q4>
__device__ __forceinline__ void epi_node_plain2(float (&acc)[4 * Q4], Slide &sl, float S0, float S1, int n,
                                                const RowConst &rc, const ColConst &cc,
                                                const float4 *__restrict__ tab, int m_last) {
    const float2 v = mul2(make_float2(S0, S1), make_float2(col_kappa(cc, n), col_kappa(cc, n + 1)));
    float2 y = mul2(splat2(rc.w[3]), make_float2(sl.v3, sl.v2));
    y = fma2v(splat2(rc.w[2]), make_float2(sl.v2, sl.v1), y);
    y = fma2v(splat2(rc.w[1]), make_float2(sl.v1, v.x), y);
    y = fma2v(splat2(rc.w[0]), v, y);
    sl.v3 = sl.v1;
    sl.v2 = v.x;
    sl.v1 = v.y;
    acc_row<Q4>(acc, tab, min(n + rc.i0, m_last), y.x);
    acc_row<Q4>(acc, tab, min(n + 1 + rc.i0, m_last), y.y);
}

// Closing rows of a run that ended at node b-1 (grid rows b+i0-1 .. b+i0+1).
template <int Q4>
__device__ __forceinline__ void epi_close(float (&acc)[4 * Q4], const Slide &sl, int b, const RowConst &rc,
                                          const float4 *__restrict__ tab, int m_last) {
    acc_row<Q4>(acc, tab, min(b + rc.i0, m_last), fmaf(rc.w[1], sl.v1, fmaf(rc.w[2], sl.v2, rc.w[3] * sl.v3)));
    acc_row<Q4>(acc, tab, min(b + rc.i0 + 1, m_last), fmaf(rc.w[2], sl.v1, rc.w[3] * sl.v2));
    acc_row<Q4>(acc, tab, min(b + rc.i0 + 2, m_last), rc.w[3] * sl.v1);
}

// Gradient mode: besides N_q (acc[0]) the same sliding sums accumulate
//   A_q = sum_n v_n c_n T_q                    (acc[1]),  d N_q / d Av    = -0.4 ln10 A_q
//   D_q = sum_n v_n (u_n l_n + e' D0_n) T_q    (acc[2]),  d N_q / d delta = -0.4 ln10 Av D_q
// with l_n = ln(lam_n / 5500 A) and e' = de/ddelta, since dF/dAv = -0.4 ln10 c F
// and dc/ddelta = u l_n + e' D0_n (Sec. 3.4, Eqs. attenuation, uvbump).
template <int Q4>
__device__ __forceinline__ void acc_row3(float (&acc)[3][4 * Q4], const float4 *__restrict__ tab, int m,
                                         float y0, float y1, float y2) {
    const float4 *tp = tab + (size_t)m * Q4;
#pragma unroll
    for (int qq = 0; qq < Q4; ++qq) {
        const float4 t = __ldg(tp + qq);
        acc_pair4(acc[0] + 4 * qq, y0, t);
        acc_pair4(acc[1] + 4 * qq, y1, t);
        acc_pair4(acc[2] + 4 * qq, y2, t);
    }
}

template <int Q4>
__device__ __forceinline__ void epi_node_grad(float (&acc)[3][4 * Q4], Slide (&sl)[3], float S, int n,
                                              const RowConst &rc, const ColConst &cc,
                                              const float4 *__restrict__ tab, int m_last) {
    const float ell = fmaf((float)n, cc.dell, cc.ell0);
    const float u = dust_pow(cc, rc, ell, n);
    const float d0 = cc.bump ? __ldg(cc.bump + n) : 0.f;
    const float cn = fmaf(rc.e, d0, u);
    const float F = exp2f(rc.alpha * cn);
    const float v = S * F * col_kappa(cc, n);
    const float vv[3] = {v, v * cn, v * fmaf(u, ell * 0.69314718055994531f, rc.ed * d0)};
    float y[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        y[r] = fmaf(rc.w[0], vv[r], fmaf(rc.w[1], sl[r].v1, fmaf(rc.w[2], sl[r].v2, rc.w[3] * sl[r].v3)));
        sl[r].v3 = sl[r].v2;
        sl[r].v2 = sl[r].v1;
        sl[r].v1 = vv[r];
    }
    acc_row3<Q4>(acc, tab, min(n + rc.i0, m_last), y[0], y[1], y[2]);
}

template <int Q4>
__device__ __forceinline__ void epi_close_grad(float (&acc)[3][4 * Q4], const Slide (&sl)[3], int b,
                                               const RowConst &rc, const float4 *__restrict__ tab, int m_last) {
    float y[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) y[r] = fmaf(rc.w[1], sl[r].v1, fmaf(rc.w[2], sl[r].v2, rc.w[3] * sl[r].v3));
    acc_row3<Q4>(acc, tab, min(b + rc.i0, m_last), y[0], y[1], y[2]);
#pragma unroll
    for (int r = 0; r < 3; ++r) y[r] = fmaf(rc.w[2], sl[r].v1, rc.w[3] * sl[r].v2);
    acc_row3<Q4>(acc, tab, min(b + rc.i0 + 1, m_last), y[0], y[1], y[2]);
#pragma unroll
    for (int r = 0; r < 3; ++r) y[r] = rc.w[3] * sl[r].v1;
    acc_row3<Q4>(acc, tab, min(b + rc.i0 + 2, m_last), y[0], y[1], y[2]);
}

// Columns (in 32-wide blocks [kb0, kb1)) of the adjoint Shat[g, n] that can be
// non-zero for the 128-row galaxy tile mt: Shat_n uses grid indices n + i0 - 1
// .. n + i0 + 2, so it vanishes unless n + i0 lies in [m_nz_lo - 2, m_nz_hi + 1]
// for some i0 of the tile (trange x .. y, over its valid rows).  At
// least one block is kept.
struct VjpBand {
    int on, m_nz_lo, m_nz_hi, Q;
};

__device__ __forceinline__ void vjp_band(const VjpBand &b, const int2 *trange, int mt, int N_pad, int &kb0,
                                         int &kb1) {
    kb0 = 0;
    kb1 = N_pad / 32;
    if (!b.on) return;
    const int2 r = trange[mt];
    const int n_lo = r.y < r.x ? 0 : max(b.m_nz_lo - r.y - 2, 0);
    const int n_hi = r.y < r.x ? -1 : min(b.m_nz_hi - r.x + 1, N_pad - 1);
    if (b.m_nz_hi < b.m_nz_lo || n_hi < n_lo) {
        kb0 = 0;
        kb1 = 1;
        return;
    }
    kb0 = n_lo / 32;
    kb1 = n_hi / 32 + 1;
}

VjpBand make_vjp_band(const Ctx &c, const FilterSet &fs, bool band);

// m_q = -2.5 log10(N_q) + 2.5 log10(AB0 D_q) - 2.5 logM + Dmod - 2.5 log10(1+z),
// in FP32 (the offsets, ~20-50 mag, carry ~4e-6 mag of rounding).
__device__ __forceinline__ float ab_mag(float flux, float magoff, float offq) {
    return -2.5f * log10f(flux) + (magoff + offq);
}

// The benchmark's colour cut and magnitude bin (dsps.h: dsps_hist_spec), in
// FP32; NaN magnitudes fail every comparison and are not counted.
__device__ __forceinline__ bool hist_bin(const HistArgs &h, float ma, float mb, float mr, int &bin) {
    const float colour = ma - mb;
    if (!(colour > h.cut) || !(mr >= h.lo) || !(mr < h.hi)) return false;
    bin = min((int)((mr - h.lo) * h.scale), h.n_bins - 1);
    return true;
}

template <int Q4>
__device__ __forceinline__ void write_mags(const float (&acc)[4 * Q4], int Q, float magoff,
                                           const float *__restrict__ offq, float *out) {
#pragma unroll
    for (int q = 0; q < 4 * Q4; ++q)
        if (q < Q) out[q] = ab_mag(acc[q], magoff, offq[q]);
}

}  // namespace dsps
