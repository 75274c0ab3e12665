// epilogue.cuh -- per-element photometry epilogue shared by the FP32 SIMT and
// the tcgen05 contraction kernels.
//
// For galaxy g and rest-frame wavelength node n with composite luminosity
// S_gn (Eq. full_mdf, per unit formed mass):
//   u    = (lam_n / 5500 A)^(delta - 0.7)             power-law attenuation curve
//   F    = 10^(-0.4 Av u)                              Eq. (attenuation)
//   v_n  = S_gn F c_n / lam_n                          rest-grid trapezoid of dlam/lam
//   N_q += v_n T_q((1+z) lam_n)                        Eq. (restmag) in the observer frame
// The filters are tabulated on the SSP grid's ln-lambda spacing, so the
// observer-frame position of node n is table index n + s, s = ln(1+z)/dlnlam,
// and T_q there is (1-f) T[n+i0] + f T[n+i0+1] with i0 = floor(s), f = s - i0.
// Regrouping the sum by table row m gives
//   N_q = sum_m T_q[m] y_m,  y_m = (1-f) v_{m-i0} + f v_{m-i0-1},
// which the kernels evaluate over a contiguous run of nodes [a, b) as a
// sliding pair (v_prev) plus one closing term f v_{b-1} T[b+i0].
#pragma once
#include <cmath>

#include "dsps_internal.cuh"

namespace dsps {

struct RowConst {
    float alpha, beta, f, omf;
    int i0;
    bool valid;
};

__device__ __forceinline__ RowConst load_row_const(const float *aux, int64_t row, int64_t n_rows) {
    RowConst rc{0.f, 0.f, 0.f, 1.f, 0, false};
    if (row < n_rows) {
        const float *ax = aux + row * AUX_STRIDE;
        rc.alpha = ax[0];
        rc.beta = ax[1];
        float s = ax[2];
        float fl = floorf(s);
        rc.i0 = (int)fl;
        rc.f = s - fl;
        rc.omf = 1.f - rc.f;
        rc.valid = ax[3] != 0.f;
    }
    return rc;
}

struct ColConst {
    float ell0, dell;          // log2(lam_n / 5500) = ell0 + n dell
    float kap0, kapmid, kapN;  // trapezoid weight / lambda at n = 0, interior, N-1
    int N;
};

// Host: column constants of the context's wavelength grid (phot_simt.cu).
ColConst make_col_const(const Ctx &c);

__device__ __forceinline__ float col_kappa(const ColConst &cc, int n) {
    return n == 0 ? cc.kap0 : (n == cc.N - 1 ? cc.kapN : cc.kapmid);
}

template <int Q4>
__device__ __forceinline__ void acc_row(float (&acc)[4 * Q4], const float4 *__restrict__ tab, int m, float y) {
    const float4 *tp = tab + (size_t)m * Q4;
#pragma unroll
    for (int qq = 0; qq < Q4; ++qq) {
        float4 t = __ldg(tp + qq);
        acc[4 * qq + 0] = fmaf(y, t.x, acc[4 * qq + 0]);
        acc[4 * qq + 1] = fmaf(y, t.y, acc[4 * qq + 1]);
        acc[4 * qq + 2] = fmaf(y, t.z, acc[4 * qq + 2]);
        acc[4 * qq + 3] = fmaf(y, t.w, acc[4 * qq + 3]);
    }
}

// One node of the sliding sum.
template <int Q4>
__device__ __forceinline__ void epi_node(float (&acc)[4 * Q4], float &vprev, float S, int n,
                                         const RowConst &rc, const ColConst &cc,
                                         const float4 *__restrict__ tab, int m_last) {
    float ell = fmaf((float)n, cc.dell, cc.ell0);
    float u = exp2f(rc.beta * ell);
    float F = exp2f(rc.alpha * u);
    float v = S * F * col_kappa(cc, n);
    float y = fmaf(rc.omf, v, rc.f * vprev);
    vprev = v;
    acc_row<Q4>(acc, tab, min(n + rc.i0, m_last), y);
}

// Closing term of a run that ended at node b-1.
template <int Q4>
__device__ __forceinline__ void epi_close(float (&acc)[4 * Q4], float vprev, int b, const RowConst &rc,
                                          const float4 *__restrict__ tab, int m_last) {
    acc_row<Q4>(acc, tab, min(b + rc.i0, m_last), rc.f * vprev);
}

// m_q = -2.5 log10(N_q) + 2.5 log10(AB0 D_q) - 2.5 logM + Dmod - 2.5 log10(1+z)
template <int Q4>
__device__ __forceinline__ void write_mags(const float (&acc)[4 * Q4], int Q, double magoff,
                                           const double *__restrict__ offq, float *out) {
#pragma unroll
    for (int q = 0; q < 4 * Q4; ++q)
        if (q < Q) out[q] = (float)(-2.5 * log10((double)acc[q]) + magoff + offq[q]);
}

}  // namespace dsps
