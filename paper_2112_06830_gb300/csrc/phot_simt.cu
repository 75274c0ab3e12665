// phot_simt.cu -- FP32 SIMT form of the fused photometry kernel.
//
// S = omega . L (Eq. full_mdf) as a register-tiled FP32 GEMM: each CTA owns 128
// galaxies and one of `parts` interleaved subsets of the 256-wide wavelength
// tiles (tile nt belongs to part nt mod parts, as in the tensor-core form) and
// walks its tiles -- with sorted rows, only those inside the row tile's
// redshifted filter band (the others contribute exact zeros); after the K loop
// of a tile the 128x256 block of S goes through shared memory to the epilogue,
// where two threads per galaxy row apply dust, the redshifted filter lookup and
// the wavelength reduction (epilogue.cuh).  Per-(galaxy, filter) sums stay in
// registers across a CTA's tiles and are written per part (combined in a fixed
// order by the combine kernels), or, with one part, as magnitudes; no spectrum
// is written to global memory.  The CTAs of one row tile are adjacent in the
// grid, so they run together and read the tile's weights from DRAM about once
// (the rest from L2); the SSP operand is staged with cp.async.
#include "dsps_internal.cuh"
#include "epilogue.cuh"

namespace dsps {

namespace {

// Tile: BM = 128 galaxies x BN = 256 wavelength nodes x BK = 16 per K step;
// 256 threads, each an 8 x 16 register tile (rows ty*4 + {0..3, 64..67},
// columns tx*4 + {0..3} + 64 m); one CTA per SM (181 KB of shared memory).
constexpr int BM = 128, BN = 256, BK = 16, THREADS = 256;
constexpr int TN4 = BN / 64;          // float4 column groups per thread
constexpr int AS_LD = BM + 4;
constexpr int CS_LD = BN + 1;
constexpr int EPI_COLS = BN / 2;      // epilogue columns per thread (two threads per row)

struct SArgs {
    const float *W;        // [n][K_pad]
    const float *L;        // [K_pad][N_pad]
    int K_pad, N_pad, Q, m_last;
    int k_lo, k_hi;        // contracted k range (multiples of BK): a dust group's ages, or all
    int64_t n;
    const float *aux;
    const float *magoff;
    const float4 *tab;
    const float *offq;
    ColConst cc;
    float *mags;           // [n][Q] (row gidx[r] with sorted rows), one part only
    float *partial;        // otherwise [parts][n][NR * 4 * Q4]: per part the sums N (and A, D
                           // in gradient mode) per filter
    int parts;             // wavelength-tile subsets (CTAs per row tile)
    const int2 *trange;    // per 128-row tile redshift-shift range (sorted rows), or nullptr: every tile
    const int *gidx;       // sorted row -> chunk galaxy, or nullptr
    int m_nz_lo, m_nz_hi;  // filter table rows with non-zero transmission
    unsigned long long *steps;   // BM x BN x BK tile steps executed (profiling), or nullptr
};

__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// One K range of a tile: c += W[m0 + row, k] L[k, n0 + col] over k in [kb, ke)
// (multiples of BK), for the thread's 8 rows (ty*4 + {0..3}, 64 + ty*4 +
// {0..3}) and 4*TN4_ columns (tx*4 + {0..3} + 64 m).  W (row-major per galaxy)
// goes through registers, transposed into As; the SSP panel (row-major per k)
// straight into Bs with cp.async; two buffers.  With MASK the weights of k
// outside [kx0, kx1) are read as zero (a dust group's ages in a K step shared
// with the neighbouring group).  Starts and ends with the block synchronised.
template <int TN4_, bool MASK>
__device__ __forceinline__ void contract_range(const float *__restrict__ W, const float *__restrict__ L, int K_pad,
                                               int N_pad, int64_t n, int64_t m0, int n0, int kb, int ke, int kx0,
                                               int kx1, float (*As)[BK][AS_LD], float (*Bs)[BK][64 * TN4_],
                                               float (&c)[8][4 * TN4_]) {
    constexpr int BN_ = 64 * TN4_;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int KT = (ke - kb) / BK;
    constexpr int AQ = BK / 4, AL = BM * AQ / THREADS;   // float4 per weights row, per thread
    float4 ra[AL];
    auto gload = [&](int k0, int buf) {
#pragma unroll
        for (int t = 0; t < AL; ++t) {
            int idx = tid + t * THREADS;
            int row = idx / AQ, kq = (idx % AQ) * 4;
            int64_t gr = m0 + row;
            ra[t] = gr < n ? *reinterpret_cast<const float4 *>(W + gr * K_pad + k0 + kq)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (MASK) {
                const int k = k0 + kq;
                if (k < kx0 || k + 4 > kx1) {
                    if (k < kx0 || k >= kx1) ra[t].x = 0.f;
                    if (k + 1 < kx0 || k + 1 >= kx1) ra[t].y = 0.f;
                    if (k + 2 < kx0 || k + 2 >= kx1) ra[t].z = 0.f;
                    if (k + 3 < kx0 || k + 3 >= kx1) ra[t].w = 0.f;
                }
            }
        }
#pragma unroll
        for (int t = 0; t < BK * BN_ / 4 / THREADS; ++t) {
            int idx = tid + t * THREADS;
            int k = idx / (BN_ / 4), nq = (idx % (BN_ / 4)) * 4;
            cp_async16(&Bs[buf][k][nq], L + (int64_t)(k0 + k) * N_pad + n0 + nq);
        }
        cp_async_commit();
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int t = 0; t < AL; ++t) {
            int idx = tid + t * THREADS;
            int row = idx / AQ, kq = (idx % AQ) * 4;
            As[buf][kq + 0][row] = ra[t].x;
            As[buf][kq + 1][row] = ra[t].y;
            As[buf][kq + 2][row] = ra[t].z;
            As[buf][kq + 3][row] = ra[t].w;
        }
    };

    gload(kb, 0);
    sstore(0);
    cp_async_wait_all();
    __syncthreads();
    for (int kt = 0; kt < KT; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < KT) gload(kb + (kt + 1) * BK, buf ^ 1);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][64 + ty * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float bv[4 * TN4_];
#pragma unroll
            for (int m = 0; m < TN4_; ++m) {
                const float4 b = *reinterpret_cast<const float4 *>(&Bs[buf][k][64 * m + tx * 4]);
                bv[4 * m] = b.x;
                bv[4 * m + 1] = b.y;
                bv[4 * m + 2] = b.z;
                bv[4 * m + 3] = b.w;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4 * TN4_; ++j) c[i][j] = fmaf(av[i], bv[j], c[i][j]);
        }
        if (kt + 1 < KT) sstore(buf ^ 1);
        cp_async_wait_all();
        __syncthreads();
    }
}

template <int Q4, bool GRAD>
__global__ void __launch_bounds__(THREADS, 1) phot_simt_kernel(SArgs a) {
    // dynamic shared memory: the K-loop operands As [2][BK][AS_LD] and Bs
    // [2][BK][BN], and, aliasing them after the K loop, the tile of S, Cs
    // [BM][CS_LD] (barriers separate the two uses)
    extern __shared__ __align__(16) float smem_f[];
    float (*As)[BK][AS_LD] = reinterpret_cast<float (*)[BK][AS_LD]>(smem_f);
    float (*Bs)[BK][BN] = reinterpret_cast<float (*)[BK][BN]>(smem_f + 2 * BK * AS_LD);
    float *Cs = smem_f;

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int mt = blockIdx.x / a.parts, part = blockIdx.x - mt * a.parts;
    const int64_t m0 = (int64_t)mt * BM;
    const int er = tid >> 1, eh = tid & 1;

    constexpr int NR = GRAD ? 3 : 1;
    float acc[NR][4 * Q4];
#pragma unroll
    for (int r3 = 0; r3 < NR; ++r3)
#pragma unroll
        for (int q = 0; q < 4 * Q4; ++q) acc[r3][q] = 0.f;

    const int KT = (a.k_hi - a.k_lo) / BK;   // the weights vanish outside [k_lo, k_hi)
    // wavelength tiles whose interpolation rows can meet the filters' band for
    // some shift of this tile's rows (all tiles without ranges)
    int nbeg = 0, nend = a.N_pad;
    if (a.trange) {
        const int2 r = a.trange[mt];
        const int n_lo = a.m_nz_lo - r.y - 2, n_hi = a.m_nz_hi - r.x + 1;
        if (r.y < r.x || a.m_nz_hi < a.m_nz_lo || n_hi < 0) {
            nend = 0;
        } else {
            nbeg = max(n_lo, 0) / BN * BN;
            nend = min(a.N_pad, (n_hi / BN + 1) * BN);
        }
    }
    // this part's tiles: nt = nbeg/BN, ... with nt mod parts == part (a tile's
    // part does not depend on the band, so every galaxy's sums add the same
    // non-zero terms in the same order in any batch)
    const int t0 = nbeg / BN;
    const int nfirst = (t0 + ((part - t0 % a.parts) % a.parts + a.parts) % a.parts) * BN;
    const int nstep = a.parts * BN;
    if (a.steps && tid == 0 && nend > nfirst)   // counted in 128 x 128 x 16 steps
        atomicAdd(a.steps, (unsigned long long)((nend - nfirst + nstep - 1) / nstep) * KT * (BK / 16) * (BN / 128));
    for (int n0 = nfirst; n0 < nend; n0 += nstep) {
        float c[8][4 * TN4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4 * TN4; ++j) c[i][j] = 0.f;

        contract_range<TN4, false>(a.W, a.L, a.K_pad, a.N_pad, a.n, m0, n0, a.k_lo, a.k_hi, 0, 0, As, Bs, c);

#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int r = (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
#pragma unroll
            for (int j = 0; j < 4 * TN4; ++j) {
                int col = 64 * (j >> 2) + tx * 4 + (j & 3);
                Cs[r * CS_LD + col] = c[i][j];
            }
        }
        __syncthreads();

        const RowConst rc = load_row_const(a.aux, m0 + er, a.n);
        if (rc.valid) {
            Slide sl[3];
            const int nb = n0 + eh * EPI_COLS;
            for (int jj = 0; jj < EPI_COLS; ++jj) {
                if constexpr (GRAD)
                    epi_node_grad<Q4>(acc, sl, Cs[er * CS_LD + eh * EPI_COLS + jj], nb + jj, rc, a.cc, a.tab,
                                      a.m_last);
                else
                    epi_node<Q4>(acc[0], sl[0], Cs[er * CS_LD + eh * EPI_COLS + jj], nb + jj, rc, a.cc, a.tab,
                                 a.m_last);
            }
            if constexpr (GRAD)
                epi_close_grad<Q4>(acc, sl, nb + EPI_COLS, rc, a.tab, a.m_last);
            else
                epi_close<Q4>(acc[0], sl[0], nb + EPI_COLS, rc, a.tab, a.m_last);
        }
        __syncthreads();
    }

#pragma unroll
    for (int r3 = 0; r3 < NR; ++r3)
#pragma unroll
        for (int q = 0; q < 4 * Q4; ++q) acc[r3][q] += __shfl_xor_sync(0xffffffffu, acc[r3][q], 1);
    const int64_t row = m0 + er;
    if (eh == 0 && row < a.n) {
        if (GRAD || !a.mags) {
            float4 *dst = reinterpret_cast<float4 *>(a.partial + ((int64_t)part * a.n + row) * (NR * 4 * Q4));
#pragma unroll
            for (int r3 = 0; r3 < NR; ++r3)
#pragma unroll
                for (int qq = 0; qq < Q4; ++qq)
                    dst[r3 * Q4 + qq] = make_float4(acc[r3][4 * qq], acc[r3][4 * qq + 1], acc[r3][4 * qq + 2],
                                                    acc[r3][4 * qq + 3]);
        } else {
            write_mags<Q4>(acc[0], a.Q, a.magoff[row], a.offq, a.mags + (a.gidx ? (int64_t)a.gidx[row] : row) * a.Q);
        }
    }
}

// Age-dependent dust (Sec. 3.4.1, Eq. agedep_dust_csp) in one launch of the
// FP32 form.  With the weights of all ages from one pass (age-major k, so a
// dust group's ages are one k range), each 128-galaxy x 128-node tile
// contracts the groups one after another over their own k ranges -- a K step
// shared by two groups is contracted for each, the other group's weights read
// as zero -- and adds each group's block of S_g, attenuated by the group's curve
// of every row (Av_g = (1 - T_g) Av_young + T_g Av_old, delta_g likewise), into
// a running sum held in registers; the sum goes through the filter integral
// once (epilogue.cuh, without dust: it is already in the sum).  8 x 8
// accumulators and 8 x 8 running sums per thread.
constexpr int GBN = 128, GTN4 = GBN / 64, G_CS_LD = GBN + 1, G_EPI_COLS = GBN / 2;
constexpr int SG_MAX = AGEDEP_MAX_GROUPS;

struct SGroups {
    int n;
    int k0[SG_MAX], k1[SG_MAX];   // the group's k range [k0, k1)
    float T[SG_MAX];              // the group's weight of the old-star dust values
};

template <int Q4>
__global__ void __launch_bounds__(THREADS, 1) phot_simt_groups_kernel(SArgs a, const __grid_constant__ SGroups gs) {
    extern __shared__ __align__(16) float smem_f[];
    float (*As)[BK][AS_LD] = reinterpret_cast<float (*)[BK][AS_LD]>(smem_f);
    float (*Bs)[BK][GBN] = reinterpret_cast<float (*)[BK][GBN]>(smem_f + 2 * BK * AS_LD);
    float *Cs = smem_f;                  // the running sum after the groups (aliases As, Bs)
    __shared__ float4 dust[BM];          // per row: Av_young, delta_young, Av_old, delta_old

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int mt = blockIdx.x / a.parts, part = blockIdx.x - mt * a.parts;
    const int64_t m0 = (int64_t)mt * BM;
    const int er = tid >> 1, eh = tid & 1;
    if (tid < BM) {
        float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m0 + tid < a.n) {
            const float *ax = a.aux + (m0 + tid) * AUX_STRIDE;
            d = make_float4(ax[0], ax[1], ax[4], ax[5]);
        }
        dust[tid] = d;
    }
    __syncthreads();

    float acc[4 * Q4];
#pragma unroll
    for (int q = 0; q < 4 * Q4; ++q) acc[q] = 0.f;
    int nbeg = 0, nend = a.N_pad;
    if (a.trange) {
        const int2 r = a.trange[mt];
        const int n_lo = a.m_nz_lo - r.y - 2, n_hi = a.m_nz_hi - r.x + 1;
        if (r.y < r.x || a.m_nz_hi < a.m_nz_lo || n_hi < 0) {
            nend = 0;
        } else {
            nbeg = max(n_lo, 0) / GBN * GBN;
            nend = min(a.N_pad, (n_hi / GBN + 1) * GBN);
        }
    }
    const int t0 = nbeg / GBN;
    const int nfirst = (t0 + ((part - t0 % a.parts) % a.parts + a.parts) % a.parts) * GBN;
    const int nstep = a.parts * GBN;
    unsigned long long steps = 0;
    for (int n0 = nfirst; n0 < nend; n0 += nstep) {
        float run[8][4 * GTN4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4 * GTN4; ++j) run[i][j] = 0.f;
        for (int g = 0; g < gs.n; ++g) {
            const int kx0 = gs.k0[g], kx1 = gs.k1[g];
            const int kb = max(kx0 / BK * BK, a.k_lo), ke = min((kx1 + BK - 1) / BK * BK, a.k_hi);
            if (kb >= ke) continue;
            steps += (unsigned long long)((ke - kb) / BK) * (BK / 16);
            float c[8][4 * GTN4];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4 * GTN4; ++j) c[i][j] = 0.f;
            contract_range<GTN4, true>(a.W, a.L, a.K_pad, a.N_pad, a.n, m0, n0, kb, ke, kx0, kx1, As, Bs, c);
            const float T = gs.T[g];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 d = dust[i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4];
                const float Avg = group_dust_value(T, d.x, d.z), dlg = group_dust_value(T, d.y, d.w);
                RowConst rg{};
                rg.alpha = -0.4f * 3.32192809488736235f * Avg;
                rg.beta = a.cc.k0 ? dlg : dlg - 0.7f;
                rg.e = a.cc.bump ? (0.85f - 1.9f * dlg) * (1.f / 4.05f) : 0.f;
#pragma unroll
                for (int j = 0; j < 4 * GTN4; ++j) {
                    const int n = n0 + 64 * (j >> 2) + tx * 4 + (j & 3);
                    run[i][j] = fmaf(c[i][j], dust_factor(a.cc, rg, n), run[i][j]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
#pragma unroll
            for (int j = 0; j < 4 * GTN4; ++j) Cs[r * G_CS_LD + 64 * (j >> 2) + tx * 4 + (j & 3)] = run[i][j];
        }
        __syncthreads();
        const RowConst rc = load_row_const(a.aux, m0 + er, a.n);   // the row's shift and validity
        if (rc.valid) {
            Slide sl;
            const int nb = n0 + eh * G_EPI_COLS;
            for (int jj = 0; jj < G_EPI_COLS; ++jj)
                epi_node_plain<Q4>(acc, sl, Cs[er * G_CS_LD + eh * G_EPI_COLS + jj], nb + jj, rc, a.cc, a.tab,
                                   a.m_last);
            epi_close<Q4>(acc, sl, nb + G_EPI_COLS, rc, a.tab, a.m_last);
        }
        __syncthreads();
    }
    if (a.steps && tid == 0 && steps) atomicAdd(a.steps, steps);
#pragma unroll
    for (int q = 0; q < 4 * Q4; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], 1);
    const int64_t row = m0 + er;
    if (eh == 0 && row < a.n) {
        float4 *dst = reinterpret_cast<float4 *>(a.partial + ((int64_t)part * a.n + row) * (4 * Q4));
#pragma unroll
        for (int qq = 0; qq < Q4; ++qq)
            dst[qq] = make_float4(acc[4 * qq], acc[4 * qq + 1], acc[4 * qq + 2], acc[4 * qq + 3]);
    }
}

constexpr size_t SIMT_G_SMEM =
    sizeof(float) * (BM * G_CS_LD > 2 * BK * (AS_LD + GBN) ? BM * G_CS_LD : 2 * BK * (AS_LD + GBN));

template <int Q4>
cudaError_t launch_groups_q4(const SArgs &a, const SGroups &gs, int64_t n, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(phot_simt_groups_kernel<Q4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SIMT_G_SMEM);
    if (e != cudaSuccess) return e;
    phot_simt_groups_kernel<Q4><<<(unsigned)((n + BM - 1) / BM * a.parts), THREADS, SIMT_G_SMEM, s>>>(a, gs);
    return cudaGetLastError();
}

constexpr size_t SIMT_SMEM = sizeof(float) * (BM * CS_LD > 2 * BK * (AS_LD + BN) ? BM * CS_LD : 2 * BK * (AS_LD + BN));

template <int Q4, bool GRAD>
cudaError_t launch_q4(const SArgs &a, int64_t n, cudaStream_t s) {
    const size_t smem = SIMT_SMEM;
    cudaFuncSetAttribute(phot_simt_kernel<Q4, GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((unsigned)((n + BM - 1) / BM * a.parts));
    phot_simt_kernel<Q4, GRAD><<<grid, THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

ColConst make_col_const(const Ctx &c) {
    ColConst cc;
    cc.ell0 = (float)((c.lnlam0 - std::log(LAM_V)) / std::log(2.0));
    cc.dell = (float)(c.dlnlam / std::log(2.0));
    cc.kap0 = (float)(0.5 * std::expm1(c.dlnlam));
    cc.kapmid = (float)std::sinh(c.dlnlam);
    cc.kapN = (float)(-0.5 * std::expm1(-c.dlnlam));
    cc.N = c.n_lam;
    cc.bump = c.opts.dust_bump ? c.d_bump : nullptr;
    cc.k0 = c.opts.dust_law == DSPS_DUST_SALIM ? c.d_k0 : nullptr;
    return cc;
}

cudaError_t launch_phot_simt(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, float *mags,
                             cudaStream_t s, bool grad, bool sorted, const DustGroup *group, int *parts) {
    // magnitudes need one part; sums go out per part (TC_PARTS with sorted rows)
    const int np = (!grad && mags) || !sorted ? 1 : TC_PARTS;
    if (parts) *parts = np;
    if (n <= 0) return cudaSuccess;
    if (np > 1 && !w.partial) return cudaErrorInvalidValue;
    SArgs a{};
    a.parts = np;
    a.W = w.w32;
    a.L = c.d_L32;
    a.K_pad = c.K_pad;
    group_k_range(c, group, BK, a.k_lo, a.k_hi);
    a.N_pad = c.N_pad;
    a.Q = fs.Q;
    a.m_last = fs.m_rows - 1;
    a.n = n;
    a.aux = w.aux;
    a.magoff = w.magoff;
    a.tab = reinterpret_cast<const float4 *>(fs.d_tab);
    a.offq = fs.d_offq;
    a.cc = make_col_const(c);
    a.mags = mags;
    a.partial = w.partial;
    a.trange = sorted && c.opts.band_skip ? w.trange : nullptr;
    a.gidx = sorted ? w.gidx : nullptr;
    a.m_nz_lo = fs.m_nz_lo;
    a.m_nz_hi = fs.m_nz_hi;
    a.steps = w.stats ? w.stats + 1 : nullptr;
    if (grad) {
        switch (fs.Q4) {
        case 1: return launch_q4<1, true>(a, n, s);
        case 2: return launch_q4<2, true>(a, n, s);
        case 3: return launch_q4<3, true>(a, n, s);
        default: return launch_q4<4, true>(a, n, s);
        }
    }
    switch (fs.Q4) {
    case 1: return launch_q4<1, false>(a, n, s);
    case 2: return launch_q4<2, false>(a, n, s);
    case 3: return launch_q4<3, false>(a, n, s);
    default: return launch_q4<4, false>(a, n, s);
    }
}

cudaError_t launch_phot_simt_groups(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, int *parts,
                                    cudaStream_t s) {
    *parts = TC_PARTS;
    if (n <= 0) return cudaSuccess;
    if (!w.partial || (int)c.dust_groups.size() > SG_MAX) return cudaErrorInvalidValue;
    SArgs a{};
    a.parts = TC_PARTS;
    a.W = w.w32;
    a.L = c.d_L32;
    a.K_pad = c.K_pad;
    a.k_lo = 0;
    a.k_hi = c.K_pad;
    a.N_pad = c.N_pad;
    a.Q = fs.Q;
    a.m_last = fs.m_rows - 1;
    a.n = n;
    a.aux = w.aux;
    a.magoff = w.magoff;
    a.tab = reinterpret_cast<const float4 *>(fs.d_tab);
    a.offq = fs.d_offq;
    a.cc = make_col_const(c);
    a.partial = w.partial;
    a.trange = c.opts.band_skip ? w.trange : nullptr;
    a.gidx = w.gidx;
    a.m_nz_lo = fs.m_nz_lo;
    a.m_nz_hi = fs.m_nz_hi;
    a.steps = w.stats ? w.stats + 1 : nullptr;
    SGroups gs{};
    const int per_age = c.n_z * c.n_u;
    gs.n = (int)c.dust_groups.size();
    for (int g = 0; g < gs.n; ++g) {
        gs.k0[g] = c.dust_groups[g].i0 * per_age;
        gs.k1[g] = c.dust_groups[g].i1 * per_age;
        gs.T[g] = c.dust_groups[g].T;
    }
    switch (fs.Q4) {
    case 1: return launch_groups_q4<1>(a, gs, n, s);
    case 2: return launch_groups_q4<2>(a, gs, n, s);
    case 3: return launch_groups_q4<3>(a, gs, n, s);
    default: return launch_groups_q4<4>(a, gs, n, s);
    }
}

}  // namespace dsps
