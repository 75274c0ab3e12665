// simt_common.cuh -- the FP32 SIMT contraction tile shared by the
// photometry kernels of the FP32 form (phot_simt.cu) and its one-launch
// age-dependent dust kernel (agedep_simt.cu).
#pragma once

#include "dsps_internal.cuh"
#include "epilogue.cuh"

namespace dsps {
namespace simt {

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

// Two FP32 FMAs in one instruction (PTX fma.rn.f32x2, sm_100 family): c0 +=
// a b0, c1 += a b1, each rounded once like fmaf, so the sums are bit-identical
// to the scalar form; half the issue slots, which the operand loads then use.
__device__ __forceinline__ void fma2(float &c0, float &c1, float a, float b0, float b1) {
    asm("{\n.reg .b64 d, x, y;\nmov.b64 x, {%2, %2};\nmov.b64 y, {%3, %4};\nmov.b64 d, {%0, %1};\n"
        "fma.rn.f32x2 d, x, y, d;\nmov.b64 {%0, %1}, d;\n}"
        : "+f"(c0), "+f"(c1)
        : "f"(a), "f"(b0), "f"(b1));
}

// One K range of a tile: c += W[m0 + row, k] L[k, n0 + col] over k in [kb, ke)
// (multiples of BK), for the thread's 8 rows (ty*4 + {0..3}, 64 + ty*4 +
// {0..3}) and 4*TN4_ columns (tx*4 + {0..3} + 64 m).  W (row-major per galaxy)
// goes through registers, transposed into As; the SSP panel (row-major per k)
// straight into Bs with cp.async; two buffers.  With MASK the weights of k
// outside [kx0, kx1) are read as zero (a dust group's ages in a K step shared
// with the neighbouring group).  Starts and ends with the block synchronised.
// PAIRED: the products as paired FMAs (fma2), else scalar (the same sums; for
// kernels whose other live registers leave no room for the operand pairs).
template <int TN4_, bool MASK, bool PAIRED = true>
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
            for (int i = 0; i < 8; ++i) {
                if constexpr (PAIRED) {
#pragma unroll
                    for (int j = 0; j < 4 * TN4_; j += 2) fma2(c[i][j], c[i][j + 1], av[i], bv[j], bv[j + 1]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4 * TN4_; ++j) c[i][j] = fmaf(av[i], bv[j], c[i][j]);
                }
            }
        }
        if (kt + 1 < KT) sstore(buf ^ 1);
        cp_async_wait_all();
        __syncthreads();
    }
}

}  // namespace simt
}  // namespace dsps
