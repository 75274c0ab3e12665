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
#include "simt_common.cuh"

namespace dsps {

namespace {

using namespace simt;

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

        // the gradient mode's three sums per filter leave no registers for paired operands
        contract_range<TN4, false, !GRAD>(a.W, a.L, a.K_pad, a.N_pad, a.n, m0, n0, a.k_lo, a.k_hi, 0, 0, As, Bs, c);

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

}  // namespace dsps
