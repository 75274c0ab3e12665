// agedep_simt.cu -- age-dependent dust (Sec. 3.4.1, Eq. agedep_dust_csp), FP32
// form: the forward of every dust group in one launch on the tile of
// simt_common.cuh.
#include "dsps_internal.cuh"
#include "epilogue.cuh"
#include "simt_common.cuh"

namespace dsps {

namespace {

using namespace simt;

// Age-dependent dust (Sec. 3.4.1, Eq. agedep_dust_csp) in one launch of the
// FP32 form.  With the weights of all ages from one pass (age-major k, so a
// dust group's ages are one k range), each 128-galaxy x 256-node tile
// contracts the groups one after another over their own k ranges -- a K step
// shared by two groups is contracted for each, the other group's weights read
// as zero -- and adds each group's block of S_g, attenuated by the group's curve
// of every row (Av_g = (1 - T_g) Av_young + T_g Av_old, delta_g likewise), into
// a running sum; the sum goes through the filter integral once (epilogue.cuh,
// without dust: it is already in the sum).  The tile and the 8 x 16
// accumulators per thread are those of phot_simt_kernel; the running sum lives
// in shared memory, each thread's 128 values as 32 float4 strided by the block
// (element e of thread t at float4 e * 256 + t: conflict-free), and the
// attenuation steps the power law across each thread's four consecutive
// columns with one ex2 per element (relative error below 2^-22).
constexpr int G_RUN_F4 = 8 * TN4;   // float4 of one thread's running sum
constexpr int SG_MAX = AGEDEP_MAX_GROUPS;

struct SGroups {
    int n;
    int k0[SG_MAX], k1[SG_MAX];   // the group's k range [k0, k1)
    float T[SG_MAX];              // the group's weight of the old-star dust values
};

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int Q4>
__global__ void __launch_bounds__(THREADS, 1) phot_simt_groups_kernel(SArgs a, const __grid_constant__ SGroups gs) {
    // dynamic shared memory: the running sum / the tile of S for the
    // epilogue, Cs [BM][CS_LD] (aliases), then the K-loop operands As, Bs
    extern __shared__ __align__(16) float smem_f[];
    float *Cs = smem_f;
    float4 *run4 = reinterpret_cast<float4 *>(smem_f);
    float *ops = smem_f + BM * CS_LD;
    float (*As)[BK][AS_LD] = reinterpret_cast<float (*)[BK][AS_LD]>(ops);
    float (*Bs)[BK][BN] = reinterpret_cast<float (*)[BK][BN]>(ops + 2 * BK * AS_LD);
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
            nbeg = max(n_lo, 0) / BN * BN;
            nend = min(a.N_pad, (n_hi / BN + 1) * BN);
        }
    }
    const int t0 = nbeg / BN;
    const int nfirst = (t0 + ((part - t0 % a.parts) % a.parts + a.parts) % a.parts) * BN;
    const int nstep = a.parts * BN;
    unsigned long long steps = 0;
    for (int n0 = nfirst; n0 < nend; n0 += nstep) {
#pragma unroll
        for (int e = 0; e < G_RUN_F4; ++e) run4[e * THREADS + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int g = 0; g < gs.n; ++g) {
            const int kx0 = gs.k0[g], kx1 = gs.k1[g];
            const int kb = max(kx0 / BK * BK, a.k_lo), ke = min((kx1 + BK - 1) / BK * BK, a.k_hi);
            if (kb >= ke) continue;
            steps += (unsigned long long)((ke - kb) / BK) * (BK / 16) * (BN / 128);
            float c[8][4 * TN4];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4 * TN4; ++j) c[i][j] = 0.f;
            contract_range<TN4, true>(a.W, a.L, a.K_pad, a.N_pad, a.n, m0, n0, kb, ke, kx0, kx1, As, Bs, c);
            const float T = gs.T[g];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 d = dust[i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4];
                const float Avg = group_dust_value(T, d.x, d.z), dlg = group_dust_value(T, d.y, d.w);
                const float alpha = -0.4f * 3.32192809488736235f * Avg;
                const float beta = a.cc.k0 ? dlg : dlg - 0.7f;
                const float eb = a.cc.bump ? (0.85f - 1.9f * dlg) * (1.f / 4.05f) : 0.f;
                const float ustep = exp2f(beta * a.cc.dell);
#pragma unroll
                for (int m = 0; m < TN4; ++m) {
                    const int nq = n0 + 64 * m + tx * 4;   // the thread's four consecutive columns
                    float u = exp2f(beta * fmaf((float)nq, a.cc.dell, a.cc.ell0));
                    float f[4];
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) {
                        const float cp = a.cc.k0 ? u * __ldg(a.cc.k0 + nq + cc) : u;
                        const float cn = a.cc.bump ? fmaf(eb, __ldg(a.cc.bump + nq + cc), cp) : cp;
                        f[cc] = ex2_approx(alpha * cn);
                        u *= ustep;
                    }
                    float4 &r = run4[(i * TN4 + m) * THREADS + tid];
                    float4 v = r;
                    v.x = fmaf(c[i][4 * m + 0], f[0], v.x);
                    v.y = fmaf(c[i][4 * m + 1], f[1], v.y);
                    v.z = fmaf(c[i][4 * m + 2], f[2], v.z);
                    v.w = fmaf(c[i][4 * m + 3], f[3], v.w);
                    r = v;
                }
            }
        }
        // the running sum into the row-major tile of S (Cs aliases it)
        float c[8][4 * TN4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int m = 0; m < TN4; ++m) {
                const float4 v = run4[(i * TN4 + m) * THREADS + tid];
                c[i][4 * m] = v.x;
                c[i][4 * m + 1] = v.y;
                c[i][4 * m + 2] = v.z;
                c[i][4 * m + 3] = v.w;
            }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
#pragma unroll
            for (int j = 0; j < 4 * TN4; ++j) Cs[r * CS_LD + 64 * (j >> 2) + tx * 4 + (j & 3)] = c[i][j];
        }
        __syncthreads();
        const RowConst rc = load_row_const(a.aux, m0 + er, a.n);   // the row's shift and validity
        if (rc.valid) {
            Slide sl;
            const int nb = n0 + eh * EPI_COLS;
            const float *crow = Cs + er * CS_LD + eh * EPI_COLS;
            for (int jj = 0; jj < EPI_COLS; jj += 2)
                epi_node_plain2<Q4>(acc, sl, crow[jj], crow[jj + 1], nb + jj, rc, a.cc, a.tab, a.m_last);
            epi_close<Q4>(acc, sl, nb + EPI_COLS, rc, a.tab, a.m_last);
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

constexpr size_t SIMT_G_SMEM = sizeof(float) * ((size_t)BM * CS_LD + 2 * BK * (AS_LD + BN));
static_assert(BM * CS_LD >= 4 * G_RUN_F4 * THREADS, "the running sum fits under the S tile");

template <int Q4>
cudaError_t launch_groups_q4(const SArgs &a, const SGroups &gs, int64_t n, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(phot_simt_groups_kernel<Q4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SIMT_G_SMEM);
    if (e != cudaSuccess) return e;
    phot_simt_groups_kernel<Q4><<<(unsigned)((n + BM - 1) / BM * a.parts), THREADS, SIMT_G_SMEM, s>>>(a, gs);
    return cudaGetLastError();
}

}  // namespace

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
