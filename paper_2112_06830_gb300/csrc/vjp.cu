// vjp.cu -- adjoint of the photometry (Sec. 2.1: the gradient of the SED with
// respect to the parameters follows from the gradients of the SSP weights;
// Sec. 3.4 for dust).  Given mag_bar = dLoss/dm[g][q]:
//
//   Nbar_q  = mag_bar_q * (-2.5 / ln 10) / N_q                (Sec. 2.2 magnitudes)
//   Av_bar  = sum_q Nbar_q (-0.4 ln 10) A_q,   delta_bar = sum_q Nbar_q (-0.4 ln 10 Av) D_q
//   logM_bar = -2.5 sum_q mag_bar_q
//   Shat[g, n] = kappa_n F_gn sum_q Nbar_q T_q((1+z_g) lam_n)  (= dLoss/dS[g, n])
//   What[g, kz] = sum_n Shat[g, n] Ld[kz, n]
// with Ld the metallicity-differenced SSP block (prep.cu; metallicity-major
// rows kz = j * A_pad + i), so What holds
// dLoss/domega[g, (i, 0)] and the differences dLoss/domega[g, (i, j)] -
// dLoss/domega[g, (i, j-1)]; the weights adjoint (weights.cu) follows.  A_q, D_q come from the
// forward kernels' gradient mode, so no spectrum is ever stored.
#include <cmath>

#include "dsps_internal.cuh"
#include "epilogue.cuh"
#include "simt_common.cuh"
#include "f32x2.cuh"

namespace dsps {

namespace {

__global__ void combine_grad_kernel(const float *partial, int parts, int64_t n, int qs, int Q, const float *magoff,
                                    const float *offq, const int *gidx, const float *aux, const float *mag_bar,
                                    float *mags, float *param_bar, int64_t G_stride, int64_t g_begin, float *cq) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t g = gidx ? (int64_t)gidx[r] : r;
    const bool valid = aux[r * AUX_STRIDE + 3] != 0.f;
    const float Av = aux[r * AUX_STRIDE + 4];
    const float mo = magoff[r];
    const float k10 = -2.5f / 2.302585092994046f;
    const float kd = -0.4f * 2.302585092994046f;
    float av_bar = 0.f, d_bar = 0.f, lm_bar = 0.f;
    for (int q = 0; q < Q; ++q) {
        float N = 0.f, A = 0.f, D = 0.f;
        for (int p = 0; p < parts; ++p) {
            const float *src = partial + ((int64_t)p * n + r) * (3 * qs);
            N += src[q];
            A += src[qs + q];
            D += src[2 * qs + q];
        }
        const float mb = mag_bar[g * Q + q];
        // a band without flux (filter off the SSP grid at this z): m = +inf, no gradient term
        const float nb = valid && N > 0.f ? mb * k10 / N : 0.f;
        av_bar = fmaf(nb * kd, A, av_bar);
        d_bar = fmaf(nb * kd * Av, D, d_bar);
        if (N > 0.f) lm_bar = fmaf(-2.5f, mb, lm_bar);
        cq[r * QSTRIDE_MAX + q] = nb;
        if (mags) mags[g * Q + q] = ab_mag(N, mo, offq[q]);
    }
    const float nan = __int_as_float(0x7fc00000);
    param_bar[8 * G_stride + g_begin + g] = valid ? av_bar : nan;
    param_bar[9 * G_stride + g_begin + g] = valid ? d_bar : nan;
    param_bar[10 * G_stride + g_begin + g] = valid ? lm_bar : nan;
}

// One warp per (sorted) row: Shat over the row's band columns [32 kb0, 32 kb1)
// (without DUST the factor F is left out: the part all dust curves share).
template <int Q4, bool BF16, bool DUST = true>
__global__ void __launch_bounds__(256) shat_kernel(const float *aux, const int2 *trange, const float *cq,
                                                   const float4 *tab, int m_last, ColConst cc, int64_t n, int N_pad,
                                                   VjpBand band, float *out32,
                                                   __nv_bfloat16 *out_hi, __nv_bfloat16 *out_lo) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    int kb0, kb1;
    vjp_band(band, trange, (int)(r / 128), N_pad, kb0, kb1);
    const RowConst rc = load_row_const(aux, r, n);
    float nb[4 * Q4];
#pragma unroll
    for (int q = 0; q < 4 * Q4; ++q) nb[q] = q < band.Q ? cq[r * QSTRIDE_MAX + q] : 0.f;
    // Grid indices col + i0 - 1 .. col + i0 + 2 are table rows col + i0 .. col +
    // i0 + 3.  One pass covers 64 columns, for which the warp needs 67
    // consecutive rows: lane l reduces rows col0 + l and col0 + 32 + l (its two
    // chains as paired FP32 operations; consecutive lanes read consecutive
    // rows) and lanes 0..2 rows col0 + 64 .. 66; the 67 sums go through a
    // per-warp shared buffer, from which lane l takes the stencils of columns
    // col0 + 2l and col0 + 2l + 1.  The two columns' attenuation and stencil are
    // paired FP32 operations (f32x2.cuh: each column gets the numbers of the
    // scalar operations), and their bf16 halves one 4-byte store each.
    __shared__ __align__(16) float srow_all[8][68];
    float *srow = srow_all[(threadIdx.x >> 5) & 7];
    auto reduce_row = [&](int row) {
        const float4 *tr = tab + (size_t)min(row, m_last) * Q4;
        float v = 0.f;
#pragma unroll
        for (int qq = 0; qq < Q4; ++qq) {
            const float4 t = __ldg(tr + qq);
            v = fmaf(nb[4 * qq + 0], t.x, fmaf(nb[4 * qq + 1], t.y, fmaf(nb[4 * qq + 2], t.z, fmaf(nb[4 * qq + 3], t.w, v))));
        }
        return v;
    };
    auto reduce_row2 = [&](int row_a, int row_b) {
        const float4 *ta = tab + (size_t)min(row_a, m_last) * Q4;
        const float4 *tb = tab + (size_t)min(row_b, m_last) * Q4;
        float2 v = splat2(0.f);
#pragma unroll
        for (int qq = 0; qq < Q4; ++qq) {
            const float4 a4 = __ldg(ta + qq), b4 = __ldg(tb + qq);
            v = fma2v(splat2(nb[4 * qq + 3]), make_float2(a4.w, b4.w), v);
            v = fma2v(splat2(nb[4 * qq + 2]), make_float2(a4.z, b4.z), v);
            v = fma2v(splat2(nb[4 * qq + 1]), make_float2(a4.y, b4.y), v);
            v = fma2v(splat2(nb[4 * qq + 0]), make_float2(a4.x, b4.x), v);
        }
        return v;
    };
    // Shat at columns c0, c0 + 1 from their stencil rows (cmd: row + d of each)
    auto shat2 = [&](int c0, float2 cm0, float2 cm1, float2 cm2, float2 cm3) {
        const float2 ell = fma2v(make_float2((float)c0, (float)(c0 + 1)), splat2(cc.dell), splat2(cc.ell0));
        float2 F = splat2(1.f);
        if constexpr (DUST && BF16) {
            // split to bf16 hi + lo (16 significant bits): ex2.approx (relative
            // error below 2^-22) for the power law and the attenuation
            const float2 bl = mul2(splat2(rc.beta), ell);
            float2 pw;
            asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(pw.x) : "f"(bl.x));
            asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(pw.y) : "f"(bl.y));
            float2 u = cc.k0 ? mul2(make_float2(__ldg(cc.k0 + c0), __ldg(cc.k0 + c0 + 1)), pw) : pw;
            if (cc.bump) u = fma2v(splat2(rc.e), make_float2(__ldg(cc.bump + c0), __ldg(cc.bump + c0 + 1)), u);
            const float2 ar = mul2(splat2(rc.alpha), u);
            asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(F.x) : "f"(ar.x));
            asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(F.y) : "f"(ar.y));
        } else if constexpr (DUST) {
            F.x = exp2f(rc.alpha * dust_curve(cc, rc, dust_pow(cc, rc, ell.x, c0), c0));
            F.y = exp2f(rc.alpha * dust_curve(cc, rc, dust_pow(cc, rc, ell.y, c0 + 1), c0 + 1));
        }
        float2 t = mul2(splat2(rc.w[3]), cm3);
        t = fma2v(splat2(rc.w[2]), cm2, t);
        t = fma2v(splat2(rc.w[1]), cm1, t);
        t = fma2v(splat2(rc.w[0]), cm0, t);
        return mul2(mul2(make_float2(col_kappa(cc, c0), col_kappa(cc, c0 + 1)), F), t);
    };
    auto store2 = [&](int c0, float2 sh) {
        if (BF16) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(sh.x, sh.y);
            const float2 rr = sub2(sh, __bfloat1622float2(h));
            *reinterpret_cast<__nv_bfloat162 *>(out_hi + r * N_pad + c0) = h;
            *reinterpret_cast<__nv_bfloat162 *>(out_lo + r * N_pad + c0) = __floats2bfloat162_rn(rr.x, rr.y);
        } else {
            *reinterpret_cast<float2 *>(out32 + r * N_pad + c0) = sh;
        }
    };
    const int cend = kb1 * 32;
    for (int col0 = kb0 * 32; col0 < cend; col0 += 64) {
        const bool two = col0 + 32 < cend;
        const int c0 = col0 + 2 * lane;
        float2 R = splat2(0.f);
        float ve = 0.f;
        if (rc.valid) {
            R = reduce_row2(col0 + lane + rc.i0, col0 + 32 + lane + rc.i0);
            if (two && lane < 3) ve = reduce_row(col0 + 64 + lane + rc.i0);
        }
        __syncwarp();   // the previous pass's reads are done
        srow[lane] = R.x;
        srow[32 + lane] = R.y;
        if (lane < 3) srow[64 + lane] = ve;
        __syncwarp();
        const float2 p01 = *reinterpret_cast<const float2 *>(srow + 2 * lane);
        const float2 p23 = *reinterpret_cast<const float2 *>(srow + 2 * lane + 2);
        const float p4 = srow[2 * lane + 4];
        if (c0 < cend)
            store2(c0, rc.valid ? shat2(c0, p01, make_float2(p01.y, p23.x), p23, make_float2(p23.y, p4))
                                : splat2(0.f));
    }
}

// What[r][k] = sum_n A[r][n] B[k][n]: both operands K-contiguous (A = Shat,
// B = the FP32 differenced SSP block), register-tiled like the forward SIMT kernel.
constexpr int BM = 128, BN = 128, BK = 16, THREADS = 256, AS_LD = BM + 4;

__global__ void __launch_bounds__(THREADS, 2) vjp_simt_kernel(const float *A, const float *B, int64_t n, int K_pad,
                                                              int N_pad, int col0, int col1, const int2 *trange,
                                                              VjpBand band, float *C) {
    __shared__ __align__(16) float As[2][BK][AS_LD];
    __shared__ __align__(16) float Bs[2][BK][AS_LD];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int k0c = blockIdx.y * BN;   // output column block (SSP index k)
    float c[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) c[i][j] = 0.f;
    float4 ra[2], rb[2];
    auto gload = [&](int kk) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int idx = tid + t * THREADS;
            const int row = idx >> 2, q = (idx & 3) * 4;
            const int64_t gr = m0 + row;
            ra[t] = gr < n ? *reinterpret_cast<const float4 *>(A + gr * N_pad + kk + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            const int kr = k0c + row;
            rb[t] = kr < K_pad ? *reinterpret_cast<const float4 *>(B + (int64_t)kr * N_pad + kk + q)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int idx = tid + t * THREADS;
            const int row = idx >> 2, q = (idx & 3) * 4;
            As[buf][q + 0][row] = ra[t].x;
            As[buf][q + 1][row] = ra[t].y;
            As[buf][q + 2][row] = ra[t].z;
            As[buf][q + 3][row] = ra[t].w;
            Bs[buf][q + 0][row] = rb[t].x;
            Bs[buf][q + 1][row] = rb[t].y;
            Bs[buf][q + 2][row] = rb[t].z;
            Bs[buf][q + 3][row] = rb[t].w;
        }
    };
    // contraction over the Shat columns [col0, col1) (multiples of BK), and over
    // the row tile's band only when it has one (Shat is zero outside it)
    if (band.on) {
        int kb0, kb1;
        vjp_band(band, trange, blockIdx.x, N_pad, kb0, kb1);
        col0 = max(col0, kb0 * 32);
        col1 = min(col1, kb1 * 32);
        if (col1 < col0) col1 = col0;
    }
    const int KT = (col1 - col0) / BK;
    gload(col0);
    sstore(0);
    __syncthreads();
    for (int kt = 0; kt < KT; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < KT) gload(col0 + (kt + 1) * BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][k][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; j += 2) simt::fma2(c[i][j], c[i][j + 1], av[i], bv[j], bv[j + 1]);
        }
        if (kt + 1 < KT) sstore(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (r >= n) continue;
#pragma unroll
        for (int j = 0; j < 8; j += 4) {
            const int col = k0c + (j < 4 ? tx * 4 : 64 + tx * 4);
            if (col < K_pad)
                *reinterpret_cast<float4 *>(C + r * K_pad + col) =
                    make_float4(c[i][j], c[i][j + 1], c[i][j + 2], c[i][j + 3]);
        }
    }
}

}  // namespace

VjpBand make_vjp_band(const Ctx &c, const FilterSet &fs, bool band) {
    VjpBand b;
    b.on = band ? 1 : 0;
    b.m_nz_lo = fs.m_nz_lo;
    b.m_nz_hi = fs.m_nz_hi;
    b.Q = fs.Q;
    return b;
}

cudaError_t launch_combine_grad(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, int parts,
                                bool sorted, const float *mag_bar, float *mags, float *param_bar, int64_t G_stride,
                                int64_t g_begin, cudaStream_t s) {
    (void)c;
    if (n <= 0) return cudaSuccess;
    combine_grad_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        w.partial, parts, n, 4 * fs.Q4, fs.Q, w.magoff, fs.d_offq, sorted ? w.gidx : nullptr, w.aux, mag_bar,
        mags, param_bar, G_stride, g_begin, w.cq);
    return cudaGetLastError();
}

cudaError_t launch_shat(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, bool bf16, bool band,
                        cudaStream_t s, bool dust) {
    if (n <= 0) return cudaSuccess;
    const VjpBand b = make_vjp_band(c, fs, band);
    const ColConst cc = make_col_const(c);
    const auto *tab = reinterpret_cast<const float4 *>(fs.d_tab);
    const int m_last = fs.m_rows - 1;
    float *o32 = reinterpret_cast<float *>(w.shat);
    auto *ohi = reinterpret_cast<__nv_bfloat16 *>(w.shat);
    __nv_bfloat16 *olo = ohi + (size_t)w.cap * c.N_pad;
    const unsigned blocks = (unsigned)((n * 32 + 255) / 256);
#define DSPS_SHAT(Q4)                                                                                              \
    if (!dust)                                                                                                     \
        shat_kernel<Q4, false, false><<<blocks, 256, 0, s>>>(w.aux, w.trange, w.cq, tab, m_last, cc, n, c.N_pad, b,\
                                                             o32, ohi, olo);                                       \
    else if (bf16)                                                                                                 \
        shat_kernel<Q4, true><<<blocks, 256, 0, s>>>(w.aux, w.trange, w.cq, tab, m_last, cc, n, c.N_pad, b, o32,   \
                                                     ohi, olo);                                                    \
    else                                                                                                           \
        shat_kernel<Q4, false><<<blocks, 256, 0, s>>>(w.aux, w.trange, w.cq, tab, m_last, cc, n, c.N_pad, b, o32,  \
                                                      ohi, olo);
    switch (fs.Q4) {
    case 1: DSPS_SHAT(1) break;
    case 2: DSPS_SHAT(2) break;
    case 3: DSPS_SHAT(3) break;
    default: DSPS_SHAT(4) break;
    }
#undef DSPS_SHAT
    return cudaGetLastError();
}

cudaError_t launch_vjp_simt(const Ctx &c, const Workspace &w, int64_t n, cudaStream_t s, int col0, int col1,
                            const FilterSet *fs) {
    if (n <= 0) return cudaSuccess;
    if (col1 < 0) col1 = c.N_pad;
    if (col0 < 0 || col1 > c.N_pad || col0 % BK || col1 % BK || col1 <= col0) return cudaErrorInvalidValue;
    const VjpBand b = fs ? make_vjp_band(c, *fs, c.opts.band_skip != 0) : VjpBand{0, 0, -1, 0};
    dim3 grid((unsigned)((n + BM - 1) / BM), (unsigned)((c.KZ_pad + BN - 1) / BN));
    vjp_simt_kernel<<<grid, THREADS, 0, s>>>(reinterpret_cast<const float *>(w.shat), c.d_Ld32, n, c.KZ_pad,
                                             c.N_pad, col0, col1, w.trange, b, w.w32);
    return cudaGetLastError();
}

}  // namespace dsps
