// spectrum.cu -- rest-frame spectra on a window of the wavelength grid and the
// equivalent width of an emission line (Sec. 2.2, Eq. eqw), with its adjoint.
//
// Forward, per chunk of galaxies:
//   1. weights kernel (FP32, per unit mass, age-major k)          weights.cu
//   2. S[g, n] = sum_k omega[g, k] L[k, n] for the window's columns: a
//      register-tiled FP32 GEMM (spec_window_kernel) into the chunk's Shat rows
//   3. ew_kernel, one warp per galaxy: L_n = F_n S_n (Eq. attenuation), the
//      least-squares quadratic continuum beta = sum_m psi_m L_m over the
//      continuum points, L0_j = beta . (1, x_j, x_j^2) at the line points and
//      W = sum_j t_j (L_j - L0_j) / L0_j.
// Adjoint (ew_bar = dLoss/dW):
//   dW/dL_j = t_j / L0_j at a line point; with gamma = sum_j -t_j L_j / L0_j^2
//   (1, x_j, x_j^2), dW/dL_m = gamma . psi_m at a continuum point;
//   Shat_n = ew_bar dW/dL_n F_n replaces S_n in place, and the Av and delta
//   gradients are sums of ew_bar dW/dL_n L_n dlnF_n/d(Av, delta).  Then the
//   adjoint contraction against the metallicity-differenced block over the
//   window's columns only (vjp.cu) and the weights adjoint (weights.cu).
// W is a ratio of spectra: the mass cancels and its gradient is exactly 0.
//
// Age-dependent dust (Sec. 3.4.1): each group of age bins that shares a curve
// (Ctx::dust_groups) has its own window spectrum S_g (weights of the group's
// ages) and attenuation F_g.  Spectra add 10^logM F_g S_g over the groups in
// their fixed order; the line width runs on the summed attenuated window
// L = sum_g F_g S_g (atten_acc_kernel), and its adjoint takes lb = ew_bar
// dW/dL once, then per group Shat_g = lb F_g, the group's dust sums weighted
// by (1 - T_g, T_g) (ew_group_grad_kernel), the adjoint contraction and the
// group's columns of the merged adjoint rows, before one weights adjoint.
#include <cmath>

#include "dsps_internal.cuh"
#include "epilogue.cuh"
#include "simt_common.cuh"

namespace dsps {

void set_last_error(const char *msg);

namespace {

constexpr int BM = 128, BN = 64, BK = 16, THREADS = 256;
constexpr int AS_LD = BM + 4;

struct SwArgs {
    const float *W;          // [n][K_pad] FP32 weights per unit mass
    const float *L;          // [K_pad][N_pad]
    int K_pad, N_pad;
    int k_lo, k_hi;          // contracted k range (multiples of BK): a dust group's ages, or all
    int64_t n;
    int cs, ce;              // computed columns [cs, ce), cs a multiple of 4
    // FINAL = false: raw S to out[r * N_pad + col] for col in [cs, ce)
    // FINAL = true:  10^logM F S to out[r * ld + col - o0] for col in [o0, o1)
    float *out;
    int64_t ld;
    int o0, o1;
    int accumulate;          // FINAL: add to out (age-dependent dust groups after the first)
    const float *aux;
    ColConst cc;
    const float *params;     // row 10 = logM
    int64_t G_stride, g_begin;
};

template <bool FINAL>
__global__ void __launch_bounds__(THREADS, 2) spec_window_kernel(SwArgs a) {
    __shared__ __align__(16) float As[2][BK][AS_LD];
    __shared__ __align__(16) float Bs[2][BK][BN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int n0 = a.cs + blockIdx.y * BN;
    float c[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) c[i][j] = 0.f;
    float4 ra[2], rb;
    auto gload = [&](int k0) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int idx = tid + t * THREADS;
            const int row = idx >> 2, kq = (idx & 3) * 4;
            const int64_t gr = m0 + row;
            ra[t] = gr < a.n ? *reinterpret_cast<const float4 *>(a.W + gr * a.K_pad + k0 + kq)
                             : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int k = tid >> 4, nq = n0 + (tid & 15) * 4;
        rb = nq < a.ce ? *reinterpret_cast<const float4 *>(a.L + (int64_t)(k0 + k) * a.N_pad + nq)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int idx = tid + t * THREADS;
            const int row = idx >> 2, kq = (idx & 3) * 4;
            As[buf][kq + 0][row] = ra[t].x;
            As[buf][kq + 1][row] = ra[t].y;
            As[buf][kq + 2][row] = ra[t].z;
            As[buf][kq + 3][row] = ra[t].w;
        }
        *reinterpret_cast<float4 *>(&Bs[buf][tid >> 4][(tid & 15) * 4]) = rb;
    };
    // the weights vanish outside [k_lo, k_hi): an age-major dust group
    const int KT = (a.k_hi - a.k_lo) / BK;
    gload(a.k_lo);
    sstore(0);
    __syncthreads();
    for (int kt = 0; kt < KT; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < KT) gload(a.k_lo + (kt + 1) * BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; j += 2) simt::fma2(c[i][j], c[i][j + 1], av[i], bv[j], bv[j + 1]);
        }
        if (kt + 1 < KT) sstore(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (r >= a.n) continue;
        if constexpr (FINAL) {
            const RowConst rc = load_row_const(a.aux, r, a.n);
            const float mass = exp10f(a.params[10 * a.G_stride + a.g_begin + r]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int col = n0 + tx * 4 + j;
                if (col < a.o0 || col >= a.o1) continue;
                float v = __int_as_float(0x7fc00000);
                if (rc.valid) {
                    const float ell = fmaf((float)col, a.cc.dell, a.cc.ell0);
                    const float F = exp2f(rc.alpha * dust_curve(a.cc, rc, dust_pow(a.cc, rc, ell, col), col));
                    v = mass * F * c[i][j];
                }
                float *o = a.out + r * a.ld + (col - a.o0);
                *o = a.accumulate ? *o + v : v;
            }
        } else {
            const int col = n0 + tx * 4;
            if (col < a.ce)
                *reinterpret_cast<float4 *>(a.out + r * a.N_pad + col) = make_float4(c[i][0], c[i][1], c[i][2], c[i][3]);
        }
    }
}

struct EwArgs {
    float *S;                // [n][N_pad] window spectrum in, Shat out (GRAD)
    int N_pad, c0, n_pts, cs, ce;
    const float4 *tab;       // LineSet::d_tab
    const float *aux;
    ColConst cc;
    int64_t n, G_stride, g_begin;
    const float *ew_bar;     // [n] (GRAD)
    float *ew;               // [n] or nullptr
    float *param_bar;        // [ngrad][G_stride] (GRAD)
    int pre;                 // S holds the attenuated window (age-dependent dust): no dust here
    int grow_old;            // gradient row of Av_old (delta_old next), age-dependent dust
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Attenuation curve A/Av (u) and d(A/Av)/d delta (du) at grid column col.
__device__ __forceinline__ void window_curve(const ColConst &cc, const RowConst &rc, int col, float &u, float &du) {
    const float ell = fmaf((float)col, cc.dell, cc.ell0);
    const float v = dust_pow(cc, rc, ell, col);
    u = dust_curve(cc, rc, v, col);
    du = v * ell * 0.69314718055994531f;
    if (cc.bump) du = fmaf(rc.ed, __ldg(cc.bump + col), du);
}

// One warp per galaxy (chunk row r).
template <bool GRAD>
__global__ void __launch_bounds__(256) ew_kernel(EwArgs a) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= a.n) return;
    const RowConst rc = load_row_const(a.aux, r, a.n);
    float *srow = a.S + r * a.N_pad;
    // attenuation curve A/Av (u) and d(A/Av)/d delta (du) at window point j
    auto curve = [&](int j, float &u, float &du) { window_curve(a.cc, rc, a.c0 + j, u, du); };
    // attenuated luminosity at window point j, rounded as a product of its own
    // (never fused into a later FMA), so that the forward and the gradient
    // instantiations give the same W bit for bit; a pre-attenuated window is
    // read as it is
    auto lum = [&](int j, float &u, float &du) {
        if (a.pre) {
            u = du = 0.f;
            return srow[a.c0 + j];
        }
        curve(j, u, du);
        return __fmul_rn(exp2f(rc.alpha * u), srow[a.c0 + j]);
    };
    // 1. continuum fit: beta = sum_m psi_m L_m
    float b0 = 0.f, b1 = 0.f, b2 = 0.f;
    for (int j = lane; j < a.n_pts; j += 32) {
        const float4 p0 = __ldg(a.tab + 2 * j);
        if (p0.w == 0.f) continue;
        const float4 p1 = __ldg(a.tab + 2 * j + 1);
        float u, du;
        const float L = lum(j, u, du);
        b0 = fmaf(p1.x, L, b0);
        b1 = fmaf(p1.y, L, b1);
        b2 = fmaf(p1.z, L, b2);
    }
    b0 = warp_sum(b0);
    b1 = warp_sum(b1);
    b2 = warp_sum(b2);
    // 2. W = sum_j t_j (L_j - L0_j) / L0_j over the line points
    const float eb = GRAD ? a.ew_bar[r] : 0.f;
    float W = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    for (int j = lane; j < a.n_pts; j += 32) {
        const float4 p0 = __ldg(a.tab + 2 * j);
        if (p0.w != 0.f) continue;
        float u, du;
        const float L = lum(j, u, du);
        const float L0 = fmaf(p0.z, b2, fmaf(p0.y, b1, b0));
        W = fmaf(p0.x, (L - L0) / L0, W);
        if (GRAD) {
            const float gq = -eb * p0.x * L / (L0 * L0);
            g0 += gq;
            g1 = fmaf(gq, p0.y, g1);
            g2 = fmaf(gq, p0.z, g2);
        }
    }
    W = warp_sum(W);
    const float nan = __int_as_float(0x7fc00000);
    if (lane == 0 && a.ew) a.ew[r] = rc.valid ? W : nan;
    if constexpr (GRAD) {
        g0 = warp_sum(g0);
        g1 = warp_sum(g1);
        g2 = warp_sum(g2);
        // 3. Shat_n = ew_bar dW/dL_n F_n in place; dust gradients.  W is
        //    unchanged by scaling L, so sum_n dW/dL_n L_n = 0 and the sums
        //    sum_n dW/dL_n L_n (u_n - u_c), with the curve's value u_c at a
        //    reference point subtracted, equal the plain ones while keeping
        //    only the curve's variation across the window (a few per cent).
        float uc = 0.f, duc = 0.f;
        if (!a.pre) curve(a.n_pts / 2, uc, duc);
        float avb = 0.f, db = 0.f;
        for (int j = lane; j < a.n_pts; j += 32) {
            const float4 p0 = __ldg(a.tab + 2 * j);
            float u, du;
            const float L = lum(j, u, du);
            float lb;   // ew_bar dW/dL_j
            if (p0.w == 0.f) {
                const float L0 = fmaf(p0.z, b2, fmaf(p0.y, b1, b0));
                lb = eb * p0.x / L0;
            } else {
                const float4 p1 = __ldg(a.tab + 2 * j + 1);
                lb = fmaf(g2, p1.z, fmaf(g1, p1.y, g0 * p1.x));
            }
            const int col = a.c0 + j;
            if (a.pre) {   // lb itself, for the groups' pass
                srow[col] = lb;
                continue;
            }
            const float F = exp2f(rc.alpha * u);
            srow[col] = rc.valid ? lb * F : 0.f;
            avb = fmaf(lb * L, u - uc, avb);
            db = fmaf(lb * L, du - duc, db);
        }
        if (a.pre) {
            // the direct adjoint of a one-age group reads lb over [cs, ce)
            for (int col = a.cs + lane; col < a.ce; col += 32)
                if (col < a.c0 || col >= a.c0 + a.n_pts) srow[col] = 0.f;
            if (lane == 0) a.param_bar[10 * a.G_stride + a.g_begin + r] = rc.valid ? 0.f : nan;
            return;
        }
        // the contraction reads [cs, ce): zero its columns outside the window
        for (int col = a.cs + lane; col < a.ce; col += 32)
            if (col < a.c0 || col >= a.c0 + a.n_pts) srow[col] = 0.f;
        avb = warp_sum(avb);
        db = warp_sum(db);
        if (lane == 0) {
            const float kd = -0.4f * 2.302585092994046f;
            const float Av = a.aux[r * AUX_STRIDE + 4];
            const int64_t g = a.g_begin + r;
            a.param_bar[8 * a.G_stride + g] = rc.valid ? kd * avb : nan;
            a.param_bar[9 * a.G_stride + g] = rc.valid ? kd * Av * db : nan;
            a.param_bar[10 * a.G_stride + g] = rc.valid ? 0.f : nan;
        }
    }
}

// One dust group's attenuated window, added to the sum over the groups in
// their order: acc[r, c0 + j] (first group: =) += F_g S_g, rounded like the
// one-curve window (one warp per row).
__global__ void __launch_bounds__(256) atten_acc_kernel(EwArgs a, float *acc, bool first) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= a.n) return;
    const RowConst rc = load_row_const(a.aux, r, a.n);
    const float *srow = a.S + r * a.N_pad;
    float *arow = acc + r * a.N_pad;
    for (int j = lane; j < a.n_pts; j += 32) {
        float u, du;
        window_curve(a.cc, rc, a.c0 + j, u, du);
        const float L = __fmul_rn(exp2f(rc.alpha * u), srow[a.c0 + j]);
        arow[a.c0 + j] = first ? L : arow[a.c0 + j] + L;
    }
}

// One dust group's share of the line-width adjoint.  With lb_j = ew_bar
// dW/dL_j in acc, Shat_g = lb F_g replaces S_g in place (zero elsewhere in
// [cs, ce)); the group's sums sum_j lb_j L_gj (u_j, du_j) times d ln F /
// d(Av, delta) go to the row's accumulators gs[4] = {Av young, Av old,
// delta young, delta old} with the weights (1 - T, T); the last group writes
// the dust gradient rows (8, 9 and the old-star rows at the end).
__global__ void __launch_bounds__(256) ew_group_grad_kernel(EwArgs a, const float *acc, float *gsum, float T,
                                                            bool first, bool last) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= a.n) return;
    const RowConst rc = load_row_const(a.aux, r, a.n);
    float *srow = a.S + r * a.N_pad;
    const float *arow = acc + r * a.N_pad;
    float sav = 0.f, sdl = 0.f;
    for (int j = lane; j < a.n_pts; j += 32) {
        const int col = a.c0 + j;
        float u, du;
        window_curve(a.cc, rc, col, u, du);
        const float F = exp2f(rc.alpha * u);
        const float L = __fmul_rn(F, srow[col]);
        const float lb = arow[col];
        srow[col] = rc.valid ? lb * F : 0.f;
        sav = fmaf(lb * L, u, sav);
        sdl = fmaf(lb * L, du, sdl);
    }
    for (int col = a.cs + lane; col < a.ce; col += 32)
        if (col < a.c0 || col >= a.c0 + a.n_pts) srow[col] = 0.f;
    sav = warp_sum(sav);
    sdl = warp_sum(sdl);
    if (lane != 0) return;
    const float kd = -0.4f * 2.302585092994046f;
    const float Av = a.aux[r * AUX_STRIDE + 4];
    const float v[4] = {(1.f - T) * kd * sav, T * kd * sav, (1.f - T) * kd * Av * sdl, T * kd * Av * sdl};
    float *gs = gsum + r * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) gs[k] = first ? v[k] : gs[k] + v[k];
    if (!last) return;
    const float nan = __int_as_float(0x7fc00000);
    const int64_t g = a.g_begin + r;
    a.param_bar[8 * a.G_stride + g] = rc.valid ? gs[0] : nan;
    a.param_bar[9 * a.G_stride + g] = rc.valid ? gs[2] : nan;
    a.param_bar[(int64_t)a.grow_old * a.G_stride + g] = rc.valid ? gs[1] : nan;
    a.param_bar[(int64_t)(a.grow_old + 1) * a.G_stride + g] = rc.valid ? gs[3] : nan;
}

cudaError_t launch_spec_window(const Ctx &c, const Workspace &w, int64_t n, int cs, int ce, bool final_out,
                               float *out, int64_t ld, int o0, int o1, const float *params, int64_t G_stride,
                               int64_t g_begin, cudaStream_t s, const DustGroup *gr = nullptr,
                               bool accumulate = false) {
    SwArgs a{};
    a.W = w.w32;
    a.L = c.d_L32;
    a.K_pad = c.K_pad;
    group_k_range(c, gr, BK, a.k_lo, a.k_hi);
    a.N_pad = c.N_pad;
    a.n = n;
    a.cs = cs;
    a.ce = ce;
    a.out = out;
    a.ld = ld;
    a.o0 = o0;
    a.o1 = o1;
    a.aux = w.aux;
    a.cc = make_col_const(c);
    a.params = params;
    a.G_stride = G_stride;
    a.g_begin = g_begin;
    a.accumulate = accumulate ? 1 : 0;
    dim3 grid((unsigned)((n + BM - 1) / BM), (unsigned)((ce - cs + BN - 1) / BN));
    if (final_out) spec_window_kernel<true><<<grid, THREADS, 0, s>>>(a);
    else spec_window_kernel<false><<<grid, THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

int run_spectra_ws(Ctx *c, const Workspace &w, int64_t n_gal, const float *params, int n0, int n1, float *out,
                   cudaStream_t s) {
    const int cs = n0 & ~3;
    const bool ad = c->opts.dust_agedep != 0;
    const size_t n_groups = ad ? c->dust_groups.size() : 1;
    for (int64_t g0 = 0; g0 < n_gal; g0 += w.cap) {
        const int64_t n = n_gal - g0 < w.cap ? n_gal - g0 : w.cap;
        cudaError_t e = cudaSuccess;
        // one pass per dust group (one in all without age-dependent dust),
        // added into out in the groups' order
        for (size_t k = 0; k < n_groups && e == cudaSuccess; ++k) {
            e = launch_weights(*c, w, W_OMEGA_F32, params, n_gal, g0, n, nullptr, s, false,
                               ad ? &c->dust_groups[k] : nullptr);
            if (e == cudaSuccess)
                e = launch_spec_window(*c, w, n, cs, n1, true, out + g0 * (int64_t)(n1 - n0), n1 - n0, n0, n1,
                                       params, n_gal, g0, s, ad ? &c->dust_groups[k] : nullptr, k > 0);
        }
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            return DSPS_ERR_CUDA;
        }
    }
    return DSPS_OK;
}

int run_line_ew_ws(Ctx *c, const Workspace &w, int64_t n_gal, const float *params, const LineSet &ls,
                   const float *ew_bar, float *ew, float *param_bar, cudaStream_t s) {
    const bool grad = param_bar != nullptr;
    const bool ad = c->opts.dust_agedep != 0;
    for (int64_t g0 = 0; g0 < n_gal; g0 += w.cap) {
        const int64_t n = n_gal - g0 < w.cap ? n_gal - g0 : w.cap;
        float *S = reinterpret_cast<float *>(w.shat);
        EwArgs a{};
        a.S = S;
        a.N_pad = c->N_pad;
        a.c0 = ls.c0;
        a.n_pts = ls.n_pts;
        a.cs = ls.cs;
        a.ce = ls.ce;
        a.tab = ls.d_tab;
        a.aux = w.aux;
        a.cc = make_col_const(*c);
        a.n = n;
        a.G_stride = n_gal;
        a.g_begin = g0;
        a.ew_bar = grad ? ew_bar + g0 : nullptr;
        a.ew = ew ? ew + g0 : nullptr;
        a.param_bar = param_bar;
        a.grow_old = c->grow_dust_old;
        const unsigned blocks = (unsigned)((n * 32 + 255) / 256);
        cudaError_t e = cudaSuccess;
        // the window spectrum of the whole population, or of one dust group
        auto window = [&](const DustGroup *gr) {
            cudaError_t r = launch_weights(*c, w, W_OMEGA_F32, params, n_gal, g0, n, nullptr, s, false, gr);
            if (r == cudaSuccess)
                r = launch_spec_window(*c, w, n, ls.cs, ls.ce, false, S, c->N_pad, 0, 0, params, n_gal, g0, s, gr);
            return r;
        };
        auto width = [&](const EwArgs &x) {
            if (grad) ew_kernel<true><<<blocks, 256, 0, s>>>(x);
            else ew_kernel<false><<<blocks, 256, 0, s>>>(x);
            return cudaGetLastError();
        };
        if (!ad) {
            e = window(nullptr);
            if (e == cudaSuccess) e = width(a);
            if (grad && e == cudaSuccess) e = launch_vjp_simt(*c, w, n, s, ls.cs, ls.ce);
            if (grad && e == cudaSuccess)
                e = launch_weights_vjp(*c, w, params, n_gal, g0, n, false, false, param_bar, s);
        } else {
            const size_t G = c->dust_groups.size();
            for (size_t k = 0; k < G && e == cudaSuccess; ++k) {
                e = window(&c->dust_groups[k]);
                if (e == cudaSuccess) {
                    atten_acc_kernel<<<blocks, 256, 0, s>>>(a, w.ewacc, k == 0);
                    e = cudaGetLastError();
                }
            }
            EwArgs p = a;
            p.S = w.ewacc;
            p.pre = 1;
            if (e == cudaSuccess) e = width(p);
            // the merged adjoint rows: padding columns zeroed once; a one-age
            // group's n_z columns formed directly from lb and its curve, the
            // other groups' by the adjoint contraction over the window
            if (grad && e == cudaSuccess) e = launch_merge_rows(*c, w, n, DustGroup{0, 0, 0.f}, true, s);
            for (size_t k = 0; grad && k < G && e == cudaSuccess; ++k) {
                const DustGroup &gr = c->dust_groups[k];
                e = window(&gr);
                if (e == cudaSuccess) {
                    ew_group_grad_kernel<<<blocks, 256, 0, s>>>(a, w.ewacc, w.gacc, gr.T, k == 0, k + 1 == G);
                    e = cudaGetLastError();
                }
                if (age1_direct(*c, gr)) {
                    if (e == cudaSuccess)
                        e = launch_age1_adjoint(*c, w, nullptr, params, n_gal, g0, n, false, s, w.ewacc, ls.cs, ls.ce,
                                                &gr);
                } else {
                    if (e == cudaSuccess) e = launch_vjp_simt(*c, w, n, s, ls.cs, ls.ce);
                    if (e == cudaSuccess) e = launch_merge_rows(*c, w, n, gr, false, s);
                }
            }
            if (grad && e == cudaSuccess) {
                Workspace wm = w;
                wm.w32 = w.what2;
                e = launch_weights_vjp(*c, wm, params, n_gal, g0, n, false, false, param_bar, s);
            }
        }
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            return DSPS_ERR_CUDA;
        }
    }
    return DSPS_OK;
}

}  // namespace dsps
