// agedep.cu -- age-dependent dust attenuation (Sec. 3.4.1, Eq.
// agedep_dust_csp): age bin i is attenuated by its own curve, with
// Av_i = (1 - T_i) Av_young + T_i Av_old and delta_i likewise,
// T_i = T_erf((log10 age_i - x0) / h) (Appendix B).
//
// The contraction no longer factorises into one GEMM followed by one
// attenuation, but it does by groups of age bins that share a curve: the young
// bins with T = 0, each bin of the transition, and the old bins with T = 1
// (Ctx::dust_groups).  Each group runs the ordinary fused path -- weights of
// the group's ages only, with the group's dust constants, then the tensor-core
// (or FP32) contraction with its fused epilogue, both on the chunk's sorted
// rows -- and the groups' filter sums
// are added in a fixed order before the magnitudes are formed.  Every group
// keeps the chunk's sort, so rows line up; skipped K blocks (ages outside the
// group) hold exact zeros.
//
// Gradient: the filter sums of the dust derivatives are accumulated per group
// with the weights (1 - T, T) of the young and old values; the adjoint of the
// weights runs the adjoint contraction once per group, with the group's
// attenuation in Shat (its dust constants rewritten in aux; the weights are
// not needed again), keeps the adjoint rows of the group's ages, and then
// runs the weights adjoint once on the merged rows.
#include "dsps_internal.cuh"
#include "epilogue.cuh"

namespace dsps {

void set_last_error(const char *msg);

namespace {

constexpr int QS = QSTRIDE_MAX;

// Tile ranges and masks back to empty before the next group's weights (the
// chunk's sort is kept; the log U ranges depend on the log U parameters alone
// and stay -- with the nebular axis they are preset by the sort).
__global__ void tile_reset_kernel(int2 *trange, unsigned *kmask, int kmw, int n_tiles) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tiles) return;
    trange[i] = make_int2(TRANGE_EMPTY_LO, TRANGE_EMPTY_HI);
    for (int w = 0; w < kmw; ++w) kmask[(size_t)i * kmw + w] = 0u;
}

// Adds one group's filter sums (its parts in a fixed order) to
// gacc[r] = {N, A_young, A_old, D_young, D_old} (QS floats each), with
// A_* weighted by (1 - T, T) and D_* by (1 - T, T) Av_group (the delta
// derivative of the flux carries the group's Av).
__global__ void group_acc_kernel(const float *partial, int parts, int nr, int64_t n, int qs, int Q, float T,
                                 const float *aux, bool grad, bool first, float *gacc) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float Av = aux[r * AUX_STRIDE + 4];
    float *ga = gacc + r * 5 * QS;
    for (int q = 0; q < Q; ++q) {
        float N = 0.f, A = 0.f, D = 0.f;
        for (int p = 0; p < parts; ++p) {
            const float *src = partial + ((int64_t)p * n + r) * (nr * qs);
            N += src[q];
            if (grad) {
                A += src[qs + q];
                D += src[2 * qs + q];
            }
        }
        const float v[5] = {N, (1.f - T) * A, T * A, (1.f - T) * Av * D, T * Av * D};
        for (int k = 0; k < (grad ? 5 : 1); ++k) ga[k * QS + q] = first ? v[k] : ga[k * QS + q] + v[k];
    }
}

struct FinalArgs {
    const float *gacc;
    int64_t n, G_stride, g_begin;
    int Q, grow_old;          // gradient row of Av_old (delta_old next)
    const float *magoff, *offq, *aux;
    const int *gidx;          // sorted row -> chunk galaxy, or nullptr
    float *mags;              // [G][Q] of the chunk, or nullptr
    HistArgs hist;
    const float *mag_bar;     // [G][Q] of the chunk (gradient), or nullptr
    float *cq;                // [n][QS] Nbar (gradient)
    float *param_bar;         // [ngrad][G_stride] (gradient)
    int dust_rows;            // write the dust rows from gacc's A and D sums (else left to agedep_dust_rows_kernel)
};

// Magnitudes (or histogram counts) from the summed fluxes; with the gradient,
// Nbar_q and the dust and mass rows of param_bar.
__global__ void agedep_final_kernel(FinalArgs a) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n) return;
    const int64_t g = a.gidx ? (int64_t)a.gidx[r] : r;
    const float *ga = a.gacc + r * 5 * QS;
    const float mo = a.magoff[r];
    float m[DSPS_MAX_FILTERS];
    for (int q = 0; q < a.Q; ++q) m[q] = ab_mag(ga[q], mo, a.offq[q]);
    if (a.hist.counts) {
        int bin;
        if (hist_bin(a.hist, m[a.hist.band_a], m[a.hist.band_b], m[a.hist.band_r], bin))
            atomicAdd(a.hist.counts + bin, 1ull);
    }
    if (a.mags)
        for (int q = 0; q < a.Q; ++q) a.mags[g * a.Q + q] = m[q];
    if (!a.mag_bar) return;
    const bool valid = a.aux[r * AUX_STRIDE + 3] != 0.f;
    const float k10 = -2.5f / 2.302585092994046f, kd = -0.4f * 2.302585092994046f;
    float avy = 0.f, avo = 0.f, dly = 0.f, dlo = 0.f, lm = 0.f;
    for (int q = 0; q < a.Q; ++q) {
        const float mb = a.mag_bar[g * a.Q + q];
        const float nb = valid && ga[q] > 0.f ? mb * k10 / ga[q] : 0.f;   // no flux: no gradient term
        a.cq[r * QS + q] = nb;
        avy = fmaf(nb * kd, ga[QS + q], avy);
        avo = fmaf(nb * kd, ga[2 * QS + q], avo);
        dly = fmaf(nb * kd, ga[3 * QS + q], dly);
        dlo = fmaf(nb * kd, ga[4 * QS + q], dlo);
        if (ga[q] > 0.f) lm = fmaf(-2.5f, mb, lm);
    }
    const float nan = __int_as_float(0x7fc00000);
    const int64_t col = a.g_begin + g;
    a.param_bar[10 * a.G_stride + col] = valid ? lm : nan;
    if (!a.dust_rows) return;
    a.param_bar[8 * a.G_stride + col] = valid ? avy : nan;
    a.param_bar[9 * a.G_stride + col] = valid ? dly : nan;
    a.param_bar[(int64_t)a.grow_old * a.G_stride + col] = valid ? avo : nan;
    a.param_bar[(int64_t)(a.grow_old + 1) * a.G_stride + col] = valid ? dlo : nan;
}

// The dust rows of param_bar from the one-launch gradient pass
// (launch_phot_tc_groups with G): per sorted row, the parts' sums (fixed
// order) of sum_g (1 - T_g) s_g, T_g s_g, (1 - T_g) Av_g t_g and T_g Av_g t_g,
// s_g = sum_n G_n c_g,n F_g,n S_g,n and t_g with dc_g/ddelta, times
// -0.4 ln 10 (dF/dAv = -0.4 ln10 c F, Eq. attenuation): dLoss/dAv_young,
// dLoss/dAv_old, dLoss/ddelta_young, dLoss/ddelta_old.
__global__ void agedep_dust_rows_kernel(const float *dpart, int parts, int64_t n, const float *aux, const int *gidx,
                                        int64_t G_stride, int64_t g_begin, int grow_old, float *param_bar) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    for (int p = 0; p < parts; ++p) {
        const float4 v = *reinterpret_cast<const float4 *>(dpart + ((int64_t)p * n + r) * 4);
        s[0] += v.x;
        s[1] += v.y;
        s[2] += v.z;
        s[3] += v.w;
    }
    const bool valid = aux[r * AUX_STRIDE + 3] != 0.f;
    const float kd = -0.4f * 2.302585092994046f, nan = __int_as_float(0x7fc00000);
    const int64_t col = g_begin + (gidx ? (int64_t)gidx[r] : r);
    param_bar[8 * G_stride + col] = valid ? kd * s[0] : nan;
    param_bar[(int64_t)grow_old * G_stride + col] = valid ? kd * s[1] : nan;
    param_bar[9 * G_stride + col] = valid ? kd * s[2] : nan;
    param_bar[(int64_t)(grow_old + 1) * G_stride + col] = valid ? kd * s[3] : nan;
}

// Keeps, in the merged adjoint rows, the columns of the group's ages
// (kz = u SEC + j A_pad + i with i in [i0, i1)); the first group also zeroes
// the padding columns.  A thread decodes four consecutive columns once and
// walks a strip of rows, touching memory only where one of its columns is
// kept or (first group) zeroed: a one-age group moves about 1 % of the rows.
__global__ void merge_rows_kernel(const float *__restrict__ src, float *__restrict__ dst, int64_t n, int rows,
                                  int KZ_pad, int SEC, int A_pad, int nzA, int n_u, int n_age, int i0, int i1,
                                  bool first) {
    const int kz0 = 4 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (kz0 >= KZ_pad) return;
    unsigned keep = 0u, zero = 0u;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int kz = kz0 + c;
        const int u = kz / SEC, rr = kz - u * SEC;
        const bool pad = u >= n_u || rr >= nzA;
        const int i = pad ? -1 : rr % A_pad;
        if (!pad && i >= i0 && i < i1) keep |= 1u << c;
        else if (first && (pad || i >= n_age)) zero |= 1u << c;
    }
    if (!(keep | zero)) return;
    const int64_t r0 = (int64_t)blockIdx.y * rows;
    const int64_t r1 = r0 + rows < n ? r0 + rows : n;
#pragma unroll 4
    for (int64_t r = r0; r < r1; ++r) {
        const int64_t o = r * KZ_pad + kz0;
        float4 v = keep ? *reinterpret_cast<const float4 *>(src + o) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (!(keep & 1u)) v.x = 0.f;
        if (!(keep & 2u)) v.y = 0.f;
        if (!(keep & 4u)) v.z = 0.f;
        if (!(keep & 8u)) v.w = 0.f;
        if ((keep | zero) == 0xFu) {
            *reinterpret_cast<float4 *>(dst + o) = v;
        } else {
            const unsigned m = keep | zero;
            if (m & 1u) dst[o] = v.x;
            if (m & 2u) dst[o + 1] = v.y;
            if (m & 4u) dst[o + 2] = v.z;
            if (m & 8u) dst[o + 3] = v.w;
        }
    }
}

// Adjoint rows of the one-age groups (age bin i each) written straight into
// the merged rows: for each group, section u and metallicity bin j,
//   What[r, u SEC + j A_pad + i] = sum_n G[r, n] F_g[r, n] Ld[u SEC + j A_pad + i, n]
// over the row tile's band, with G the dust-free Shat (FP32, one pass for all
// one-age groups) and F_g the group's attenuation -- FP32 products in place
// of an adjoint contraction over every K column of which a group keeps n_z.
// Stored divided by wmul_d (a power of two) when the weights adjoint expects
// the tensor form's scaled rows.  One block per (256-row tile, group,
// section): the group's dust constants of each row come from its parameters
// (Sec. 3.4.1), the band is walked in 16-column chunks with the next chunk's
// G and Ld loaded into registers while the current one is contracted; thread t
// stages row t's 16 columns of G F_g (the power law stepped from column to
// column, one ex2 per column for F_g) and the group's n_z rows of Ld are
// staged beside them in shared memory; thread t accumulates rows t / 4 + 64 h
// (h < 4) over the metallicity bins j = (t & 3) + 4 m, m < MAXM / 2, in
// increasing column order.  The groups (and sections) are the grid's fastest
// index, so a tile's blocks run together and share its G in L2.
constexpr int A1_ROWS = 256, A1_CHUNK = 16, A1_THREADS = 256, A1_LD = A1_CHUNK + 4, A1_MAXG = 64;
constexpr int A1_RPT = A1_ROWS / 64;   // rows per thread in the contraction

// 2^x in one MUFU instruction (PTX ex2.approx, relative error below 2^-22).
__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct Age1Set {
    int n;                   // one-age groups (<= A1_MAXG per launch)
    int age[A1_MAXG];        // their age bins
    float T[A1_MAXG];        // their weights of the old-star dust values
};

struct Age1Args {
    const float *G, *params, *Ld, *wmul_d;
    const int *gidx;
    const int2 *trange;
    VjpBand band;
    ColConst cc;
    int64_t n, G_stride, g_begin;
    int N_pad, KZ_pad, SEC, A_pad, n_z, n_u, row_old, dust_law, bump, scaled;
    int col0, col1;          // contracted columns, or (col1 <= col0) each row tile's band
    float *out;
};

template <int MAXM>
__global__ void __launch_bounds__(A1_THREADS, 3) age1_adjoint_kernel(const Age1Args a, const Age1Set set) {
    __shared__ __align__(16) float As[A1_ROWS][A1_LD];    // G F_g, [row][column]
    __shared__ __align__(16) float Bs[2 * MAXM][A1_LD];   // Ld rows of the group's columns, [j][column]
    constexpr int LPT = (2 * MAXM * A1_CHUNK + A1_THREADS - 1) / A1_THREADS;   // Ld values per thread
    static_assert(A1_ROWS == A1_THREADS && A1_CHUNK == 16, "staging: one row of 16 columns per thread");
    const int tid = threadIdx.x, mt = blockIdx.y;
    const int gi = blockIdx.x / a.n_u, u = blockIdx.x - gi * a.n_u;
    const int i_age = set.age[gi];
    const float T = set.T[gi];
    const int64_t r0 = (int64_t)mt * A1_ROWS;
    for (int e = tid; e < 2 * MAXM * A1_LD; e += A1_THREADS) (&Bs[0][0])[e] = 0.f;   // rows j >= n_z stay 0
    // staging role: row tid of the tile, with the row's group curve in registers
    const int64_t sr = r0 + tid;
    float alpha = 0.f, beta = 0.f, eb = 0.f;
    if (sr < a.n) {
        float ax[AUX_STRIDE] = {};
        const int64_t g = a.g_begin + (a.gidx ? a.gidx[sr] : sr);
        const float avy = a.params[8 * a.G_stride + g], dly = a.params[9 * a.G_stride + g];
        const float avo = a.params[(int64_t)a.row_old * a.G_stride + g];
        const float dlo = a.params[(int64_t)(a.row_old + 1) * a.G_stride + g];
        store_dust_aux(ax, group_dust_value(T, avy, avo), group_dust_value(T, dly, dlo), a.dust_law, a.bump);
        alpha = ax[0];
        beta = ax[1];
        eb = ax[6];
    }
    const float ustep = exp2f(beta * a.cc.dell);
    // the bands of the block's two 128-row tiles (G is written over each
    // tile's band only: a row reads zeros outside its own)
    static_assert(A1_ROWS == 256, "two 128-row tiles per block");
    int kb0, kb1, ob0, ob1;
    vjp_band(a.band, a.trange, 2 * mt, a.N_pad, kb0, kb1);
    ob0 = kb0;
    ob1 = kb1;
    if ((int64_t)(2 * mt + 1) * 128 < a.n) {
        int kc0, kc1;
        vjp_band(a.band, a.trange, 2 * mt + 1, a.N_pad, kc0, kc1);
        if (tid >= 128) {
            ob0 = kc0;
            ob1 = kc1;
        }
        kb0 = min(kb0, kc0);
        kb1 = max(kb1, kc1);
    }
    const int colz = u * a.SEC + i_age;   // column of metallicity bin 0 in this section
    // the band in columns (vjp_band counts 32-column blocks), or the given range
    const bool given = a.col1 > a.col0;
    const int cbeg = given ? a.col0 : kb0 * 32, cend = given ? a.col1 : kb1 * 32;
    const int own0 = given ? a.col0 : ob0 * 32, own1 = given ? a.col1 : ob1 * 32;
    float4 gv[4];
    float lv[LPT];
    auto load = [&](int c0) {
        const bool in = sr < a.n && c0 >= own0 && c0 < own1;   // chunks and bands are 16-aligned
        const float4 *src = reinterpret_cast<const float4 *>(a.G + sr * a.N_pad + c0);
#pragma unroll
        for (int s = 0; s < 4; ++s) gv[s] = in ? src[s] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int t = 0; t < LPT; ++t) {
            const int e = tid + t * A1_THREADS, j = e / A1_CHUNK, k = e % A1_CHUNK;
            lv[t] = j < a.n_z ? __ldg(a.Ld + (size_t)(colz + j * a.A_pad) * a.N_pad + c0 + k) : 0.f;
        }
    };
    auto stage = [&](int c0) {
        // (lam_n / lam_V)^beta at the chunk's first column, then stepped
        float uc = exp2f(beta * fmaf((float)c0, a.cc.dell, a.cc.ell0));
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float g4[4] = {gv[s].x, gv[s].y, gv[s].z, gv[s].w};
            float o4[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int col = c0 + 4 * s + c;
                const float cp = a.cc.k0 ? uc * __ldg(a.cc.k0 + col) : uc;
                const float cn = a.cc.bump ? fmaf(eb, __ldg(a.cc.bump + col), cp) : cp;
                o4[c] = g4[c] * fast_exp2(alpha * cn);
                uc *= ustep;
            }
            *reinterpret_cast<float4 *>(&As[tid][4 * s]) = make_float4(o4[0], o4[1], o4[2], o4[3]);
        }
#pragma unroll
        for (int t = 0; t < LPT; ++t) {
            const int e = tid + t * A1_THREADS, j = e / A1_CHUNK, k = e % A1_CHUNK;
            if (j < 2 * MAXM) Bs[j][k] = lv[t];
        }
    };
    constexpr int M2 = MAXM / 2;
    const int row = tid >> 2, qt = tid & 3;   // rows row + 64 h; bins qt + 4 m
    float acc[A1_RPT][M2];
#pragma unroll
    for (int h = 0; h < A1_RPT; ++h)
#pragma unroll
        for (int m = 0; m < M2; ++m) acc[h][m] = 0.f;
    if (cbeg < cend) load(cbeg);
    for (int c0 = cbeg; c0 < cend; c0 += A1_CHUNK) {
        __syncthreads();   // the previous chunk's reads are done
        stage(c0);
        __syncthreads();
        if (c0 + A1_CHUNK < cend) load(c0 + A1_CHUNK);
#pragma unroll
        for (int k = 0; k < A1_CHUNK; k += 4) {
            float4 x[A1_RPT];
#pragma unroll
            for (int h = 0; h < A1_RPT; ++h) x[h] = *reinterpret_cast<const float4 *>(&As[row + 64 * h][k]);
#pragma unroll
            for (int m = 0; m < M2; ++m) {
                const float4 y = *reinterpret_cast<const float4 *>(&Bs[qt + 4 * m][k]);
#pragma unroll
                for (int h = 0; h < A1_RPT; ++h)
                    acc[h][m] = fmaf(x[h].w, y.w, fmaf(x[h].z, y.z, fmaf(x[h].y, y.y, fmaf(x[h].x, y.x, acc[h][m]))));
            }
        }
    }
#pragma unroll
    for (int h = 0; h < A1_RPT; ++h) {
        const int64_t r = r0 + row + 64 * h;
        if (r >= a.n) break;
#pragma unroll
        for (int m = 0; m < M2; ++m) {
            const int j = qt + 4 * m;
            if (j >= a.n_z) break;
            const int kz = colz + j * a.A_pad;
            a.out[r * a.KZ_pad + kz] = a.scaled ? acc[h][m] / __ldg(a.wmul_d + kz) : acc[h][m];
        }
    }
}

// The group's dust constants in aux, for the chunk's sorted rows: the
// adjoint passes need the group's curve but not its weights.
__global__ void group_aux_kernel(const float *params, int64_t G_stride, int64_t g_begin, const int *gidx, int64_t n,
                                 int row_old, float T, int dust_law, int bump, float *aux) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t g = g_begin + gidx[r];
    const float avy = params[8 * G_stride + g], dly = params[9 * G_stride + g];
    const float avo = params[(int64_t)row_old * G_stride + g], dlo = params[(int64_t)(row_old + 1) * G_stride + g];
    store_dust_aux(aux + r * AUX_STRIDE, group_dust_value(T, avy, avo), group_dust_value(T, dly, dlo), dust_law,
                   bump);
}

cudaError_t launch_tile_reset(const Ctx &c, const Workspace &w, int64_t n, cudaStream_t s) {
    const int n_tiles = (int)((n + 127) / 128);
    tile_reset_kernel<<<(n_tiles + 255) / 256, 256, 0, s>>>(w.trange, w.kmask, c.kmask_words, n_tiles);
    return cudaGetLastError();
}

cudaError_t launch_group_acc(const Workspace &w, const FilterSet &fs, int64_t n, int parts, int nr, float T,
                             bool grad, bool first, cudaStream_t s) {
    group_acc_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w.partial, parts, nr, n, 4 * fs.Q4, fs.Q, T, w.aux,
                                                                 grad, first, w.gacc);
    return cudaGetLastError();
}

cudaError_t launch_final(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, bool sorted, float *mags,
                         const HistArgs *hist, const float *mag_bar, float *param_bar, int64_t G_stride,
                         int64_t g_begin, cudaStream_t s, bool dust_rows = true) {
    FinalArgs a{};
    a.dust_rows = dust_rows ? 1 : 0;
    a.gacc = w.gacc;
    a.n = n;
    a.G_stride = G_stride;
    a.g_begin = g_begin;
    a.Q = fs.Q;
    a.grow_old = c.grow_dust_old;
    a.magoff = w.magoff;
    a.offq = fs.d_offq;
    a.aux = w.aux;
    a.gidx = sorted ? w.gidx : nullptr;
    a.mags = mags;
    if (hist) a.hist = *hist;
    a.mag_bar = mag_bar;
    a.cq = w.cq;
    a.param_bar = param_bar;
    agedep_final_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_group_aux(const Ctx &c, const Workspace &w, const float *params, int64_t G_stride,
                             int64_t g_begin, int64_t n, const DustGroup &gr, cudaStream_t s) {
    group_aux_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(params, G_stride, g_begin, w.gidx, n,
                                                                 c.row_dust_old, gr.T, c.opts.dust_law,
                                                                 c.opts.dust_bump, w.aux);
    return cudaGetLastError();
}

int fail_cuda(cudaError_t e) {
    set_last_error(cudaGetErrorString(e));
    return DSPS_ERR_CUDA;
}

// Forward of one chunk over all dust groups, leaving the summed fluxes (and,
// with grad, the dust-derivative sums) in w.gacc.
cudaError_t groups_forward(Ctx *c, const Workspace &w, int64_t n_gal, int64_t g0, int64_t n, const float *params,
                           const FilterSet &fs, bool tc, bool grad, cudaStream_t s, bool prof) {
    cudaError_t e = cudaSuccess;
    {
        ProfScope ps(*c, 0, s, prof);
        e = launch_zsort(*c, w, params, n_gal, g0, n, s);
    }
    // split-bf16: the first multi-age group's weights cache the galaxies' age
    // fractions in w32 (unused until the adjoint; [n][n_age] <= [cap][KZ_pad]),
    // and the one-age groups after it read theirs instead of recomputing the SFH
    bool cached = false;
    for (size_t k = 0; k < c->dust_groups.size() && e == cudaSuccess; ++k) {
        const DustGroup &gr = c->dust_groups[k];
        Workspace wk = w;
        const bool multi = gr.i1 - gr.i0 > 1;
        if (tc && (cached || multi)) {
            wk.fcache = w.w32;
            wk.fcache_mode = cached ? 2 : 1;
        }
        {
            ProfScope ps(*c, 0, s, prof);
            if (tc && k > 0) e = launch_tile_reset(*c, w, n, s);
            if (e == cudaSuccess)
                e = launch_weights(*c, wk, tc ? W_OMEGA_BF16X2 : W_OMEGA_F32, params, n_gal, g0, n, nullptr, s, true,
                                   &gr);
        }
        cached = cached || wk.fcache_mode == 1;
        int parts = 1;
        if (e == cudaSuccess) {
            ProfScope ps(*c, tc ? 2 : 1, s, prof);
            // the FP32 form's sums come from its gradient mode (N, A, D per filter)
            e = tc ? launch_phot_tc(*c, w, fs, n, &parts, s, grad)
                   : launch_phot_simt(*c, w, fs, n, nullptr, s, true, true, &gr, &parts);
        }
        if (e == cudaSuccess) {
            ProfScope ps(*c, 0, s, prof);
            e = launch_group_acc(w, fs, n, parts, (tc && !grad) ? 1 : 3, gr.T, grad, k == 0, s);
        }
    }
    return e;
}

}  // namespace

bool age1_direct(const Ctx &c, const DustGroup &gr) { return gr.i1 - gr.i0 == 1 && c.n_z <= 32; }

cudaError_t launch_age1_adjoint(const Ctx &c, const Workspace &w, const FilterSet *fs, const float *params,
                                int64_t G_stride, int64_t g_begin, int64_t n, bool scaled, cudaStream_t s,
                                const float *G, int col0, int col1, const DustGroup *only) {
    if (n <= 0) return cudaSuccess;
    if ((n + A1_ROWS - 1) / A1_ROWS > 65535) return cudaErrorInvalidValue;   // row tiles are the grid's y
    Age1Args a{};
    a.G = G ? G : reinterpret_cast<const float *>(w.shat);
    a.params = params;
    a.Ld = c.d_Ld32;
    a.wmul_d = c.d_wmul_d;
    a.gidx = G ? nullptr : w.gidx;
    a.trange = w.trange;
    a.band = fs ? make_vjp_band(c, *fs, c.opts.band_skip != 0) : VjpBand{0, 0, -1, 0};
    a.col0 = col0;
    a.col1 = col1;
    a.cc = make_col_const(c);
    a.n = n;
    a.G_stride = G_stride;
    a.g_begin = g_begin;
    a.N_pad = c.N_pad;
    a.KZ_pad = c.KZ_pad;
    a.SEC = c.SEC;
    a.A_pad = c.A_pad;
    a.n_z = c.n_z;
    a.n_u = c.n_u;
    a.row_old = c.row_dust_old;
    a.dust_law = c.opts.dust_law;
    a.bump = c.opts.dust_bump;
    a.scaled = scaled ? 1 : 0;
    a.out = w.what2;
    const int mm = (c.n_z + 1) / 2;
    Age1Set set{};
    size_t k = 0;
    while (true) {
        set.n = 0;
        for (; k < c.dust_groups.size() && set.n < A1_MAXG; ++k)
            if (age1_direct(c, c.dust_groups[k]) && (!only || &c.dust_groups[k] == only)) {
                set.age[set.n] = c.dust_groups[k].i0;
                set.T[set.n] = c.dust_groups[k].T;
                ++set.n;
            }
        if (set.n == 0) break;
        const dim3 grid((unsigned)(set.n * c.n_u), (unsigned)((n + A1_ROWS - 1) / A1_ROWS));
        if (mm <= 4) age1_adjoint_kernel<4><<<grid, A1_THREADS, 0, s>>>(a, set);
        else if (mm <= 8) age1_adjoint_kernel<8><<<grid, A1_THREADS, 0, s>>>(a, set);
        else if (mm <= 12) age1_adjoint_kernel<12><<<grid, A1_THREADS, 0, s>>>(a, set);
        else age1_adjoint_kernel<16><<<grid, A1_THREADS, 0, s>>>(a, set);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_merge_rows(const Ctx &c, const Workspace &w, int64_t n, const DustGroup &gr, bool first,
                         cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int rows = 64;
    while ((n + rows - 1) / rows > 65535) rows *= 2;
    const dim3 grid((unsigned)((c.KZ_pad / 4 + 127) / 128), (unsigned)((n + rows - 1) / rows));
    merge_rows_kernel<<<grid, 128, 0, s>>>(w.w32, w.what2, n, rows, c.KZ_pad, c.SEC, c.A_pad, c.n_z * c.A_pad, c.n_u,
                                          c.n_age, gr.i0, gr.i1, first);
    return cudaGetLastError();
}

int run_photometry_agedep_ws(Ctx *c, const Workspace &w0, int64_t n_gal, const float *params, const FilterSet &fs,
                             int32_t precision, float *mags, cudaStream_t s, bool profile, const HistArgs *hist) {
    Workspace w = w0;
    w.rest = fs.rest;
    w.stats = (profile && c->prof) ? c->d_stats : nullptr;
    const bool prof = profile && c->prof;
    const bool tc = precision == DSPS_PREC_BF16X3;
    // every group in one launch: split-bf16 (agedep_tc.cu) where the grid
    // allows, FP32 (phot_simt.cu) up to AGEDEP_MAX_GROUPS groups
    const bool fused = c->opts.agedep_fused &&
                       (tc ? agedep_fused_ok(*c) : (int)c->dust_groups.size() <= AGEDEP_MAX_GROUPS);
    for (int64_t g0 = 0; g0 < n_gal; g0 += w.cap) {
        const int64_t n = n_gal - g0 < w.cap ? n_gal - g0 : w.cap;
        cudaError_t e = cudaSuccess;
        if (fused) {
            int parts = 0;
            {
                ProfScope ps(*c, 0, s, prof);
                e = launch_zsort(*c, w, params, n_gal, g0, n, s);
                if (e == cudaSuccess)
                    e = tc ? launch_weights(*c, w, W_OMEGA_BF16X2_AB, params, n_gal, g0, n, nullptr, s, true)
                           : launch_weights(*c, w, W_OMEGA_F32, params, n_gal, g0, n, nullptr, s, true, nullptr, true);
            }
            if (e == cudaSuccess) {
                ProfScope ps(*c, tc ? 2 : 1, s, prof);
                e = tc ? launch_phot_tc_groups(*c, w, fs, n, &parts, s) : launch_phot_simt_groups(*c, w, fs, n, &parts, s);
            }
            if (e == cudaSuccess) {
                ProfScope ps(*c, 0, s, prof);
                e = launch_combine(*c, w, fs, n, parts, hist ? nullptr : mags + g0 * fs.Q, s, hist);
            }
        } else {
            e = groups_forward(c, w, n_gal, g0, n, params, fs, tc, false, s, prof);
            if (e == cudaSuccess) {
                ProfScope ps(*c, 0, s, prof);
                e = launch_final(*c, w, fs, n, true, hist ? nullptr : mags + g0 * fs.Q, hist, nullptr, nullptr, n_gal,
                                 g0, s);
            }
        }
        if (e != cudaSuccess) return fail_cuda(e);
    }
    return DSPS_OK;
}

int run_photometry_vjp_agedep_ws(Ctx *c, const Workspace &w0, int64_t n_gal, const float *params,
                                 const FilterSet &fs, int32_t precision, const float *mag_bar, float *mags,
                                 float *param_bar, cudaStream_t s, bool profile) {
    Workspace w = w0;
    w.rest = fs.rest;
    w.stats = (profile && c->prof) ? c->d_stats : nullptr;
    const bool prof = profile && c->prof;
    const bool tc = precision == DSPS_PREC_BF16X3;
    // split-bf16 with the one-launch forward: the fluxes from that launch, the
    // dust rows from its gradient pass over the dust-free adjoint spectrum
    const bool fused = tc && c->opts.agedep_fused && agedep_fused_ok(*c);
    for (int64_t g0 = 0; g0 < n_gal; g0 += w.cap) {
        const int64_t n = n_gal - g0 < w.cap ? n_gal - g0 : w.cap;
        cudaError_t e = cudaSuccess;
        int parts = 0;
        if (fused) {
            {
                ProfScope ps(*c, 0, s, prof);
                e = launch_zsort(*c, w, params, n_gal, g0, n, s);
                if (e == cudaSuccess)
                    e = launch_weights(*c, w, W_OMEGA_BF16X2_AB, params, n_gal, g0, n, nullptr, s, true);
            }
            if (e == cudaSuccess) {
                ProfScope ps(*c, 2, s, prof);
                e = launch_phot_tc_groups(*c, w, fs, n, &parts, s);
            }
            if (e == cudaSuccess) {
                ProfScope ps(*c, 0, s, prof);
                e = launch_group_acc(w, fs, n, parts, 1, 0.f, false, true, s);
            }
        } else {
            e = groups_forward(c, w, n_gal, g0, n, params, fs, tc, true, s, prof);
        }
        if (e == cudaSuccess) {
            ProfScope ps(*c, 3, s, prof);
            e = launch_final(*c, w, fs, n, true, mags ? mags + g0 * fs.Q : nullptr, nullptr, mag_bar + g0 * fs.Q,
                             param_bar, n_gal, g0, s, !fused);
        }
        // adjoint of the weights, merged over the groups (the group's curve in
        // aux; the tile ranges depend on z alone and stay): padding columns
        // zeroed once; the one-age groups from one dust-free Shat, their n_z
        // columns each; the other groups by an adjoint contraction each,
        // keeping their ages' columns
        bool any1 = false;
        for (const DustGroup &gr : c->dust_groups) any1 = any1 || age1_direct(*c, gr);
        if (e == cudaSuccess) {
            ProfScope ps(*c, 3, s, prof);
            e = launch_merge_rows(*c, w, n, DustGroup{0, 0, 0.f}, true, s);
            if ((any1 || fused) && e == cudaSuccess)
                e = launch_shat(*c, w, fs, n, false, c->opts.band_skip != 0, s, false);
        }
        if (fused && e == cudaSuccess) {
            // the dust rows: every group in one launch again, its epilogue
            // folding each group's block with G (aux still holds the young and
            // old values: the groups below rewrite it)
            {
                ProfScope ps(*c, 2, s, prof);
                e = launch_phot_tc_groups(*c, w, fs, n, &parts, s, reinterpret_cast<const float *>(w.shat));
            }
            if (e == cudaSuccess) {
                ProfScope ps(*c, 3, s, prof);
                agedep_dust_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
                    w.partial, parts, n, w.aux, w.gidx, n_gal, g0, c->grow_dust_old, param_bar);
                e = cudaGetLastError();
            }
        }
        // with the one-launch forward, the adjoint rows of every group from one
        // tensor-core launch over the dust-free adjoint spectrum
        const bool vjp1 = fused && agedep_vjp_tc_ok(*c);
        if (vjp1 && e == cudaSuccess) {
            ProfScope ps(*c, 3, s, prof);
            e = launch_vjp_groups_tc(*c, w, fs, params, n_gal, g0, n, s);
        }
        if (!vjp1 && any1 && e == cudaSuccess) {
            ProfScope ps(*c, 3, s, prof);
            e = launch_age1_adjoint(*c, w, &fs, params, n_gal, g0, n, tc, s);
        }
        for (size_t k = 0; !vjp1 && k < c->dust_groups.size() && e == cudaSuccess; ++k) {
            const DustGroup &gr = c->dust_groups[k];
            if (age1_direct(*c, gr)) continue;
            ProfScope ps(*c, 3, s, prof);
            e = launch_group_aux(*c, w, params, n_gal, g0, n, gr, s);
            if (e == cudaSuccess) e = launch_shat(*c, w, fs, n, tc, c->opts.band_skip != 0, s);
            if (e == cudaSuccess) e = tc ? launch_vjp_tc(*c, w, fs, n, s) : launch_vjp_simt(*c, w, n, s, 0, -1, &fs);
            if (e == cudaSuccess) e = launch_merge_rows(*c, w, n, gr, false, s);
        }
        if (e == cudaSuccess) {
            ProfScope ps(*c, 3, s, prof);
            Workspace wm = w;
            wm.w32 = w.what2;
            e = launch_weights_vjp(*c, wm, params, n_gal, g0, n, true, tc, param_bar, s);
        }
        if (e != cudaSuccess) return fail_cuda(e);
    }
    return DSPS_OK;
}

}  // namespace dsps
