// agedep_vjp_tc.cu -- age-dependent dust (Sec. 3.4.1, Eq. agedep_dust_csp):
// the adjoint rows of the weights for every dust group in one tcgen05 launch.
//
// With a curve per group, dLoss/domega at an age bin i of group g and
// metallicity bin j is
//   What[r, ij] = sum_n G[r, n] F_g[r, n] Ld[ij, n],
// G the dust-free adjoint spectrum (launch_shat without dust: dLoss/dS at node
// n), F_g the group's attenuation of row r and Ld the metallicity-differenced
// SSP block (prep.cu; the weights adjoint's summation by parts).  In the
// age-block order (ka = 32 i + j) a group's ages are one column range, so a
// work unit is (128-row tile, up to eight consecutive ages of one group): an
// MMA of N = 32 x (ages) columns per 16-node step, reduced over the tile's
// band of nodes (epilogue.cuh: vjp_band).  The B operand is the age-block copy
// of the split differenced block (Ctx::d_Ldab_*, TMA, 64-byte swizzle); the A
// operand, Shat_g = G F_g split into bf16 hi + lo, is written into shared
// memory by sixteen warps in the layout the TMA would give it (each 16-byte
// chunk c of row r at chunk c ^ ((r >> 1) & 3) of the row's 64 bytes), each
// thread a quarter of a row's 32 nodes: G read from global memory (the next
// slice's while the current one is written), F_g from the row's group curve
// (power law stepped from node to node, one ex2 per node).  Products
// hi.hi + hi.lo + lo.hi accumulate in TMEM (two 256-column accumulators); the
// epilogue writes each age's n_z columns to the merged adjoint rows in the
// metallicity-major order (kz = j A_pad + i; two neighbouring ages of a bin as
// one 8-byte store), which carry the row scale of the tensor adjoint (the B
// rows are those of d_L_* permuted).
//
// Warp roles: 0 TMA producer (4-stage ring), 1 TMEM allocator and
// single-thread MMA issuer, 2..17 A writers, 18..21 epilogue (one TMEM lane
// quadrant each).  Every mbarrier wait is bounded; on expiry the kernel records
// DERR_TIMEOUT, lets its copies and MMAs land, frees TMEM and returns.
#include <cudaTypedefs.h>

#include "dsps_internal.cuh"
#include "epilogue.cuh"
#include "tc_common.cuh"
#include "f32x2.cuh"

namespace dsps {

namespace {

using namespace tc;

constexpr int BM = 128, BK = KBLOCK, BNMAX = 256;
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;            // one bf16 part of the A tile (64 bytes per row)
constexpr int B_BYTES = BNMAX * BK * 2;         // one bf16 part of the widest B tile
constexpr int B_OFF = 2 * A_BYTES;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int NUM_GEN_WARPS = 16, NUM_EPI_WARPS = 4;
constexpr int TPR = NUM_GEN_WARPS * 32 / BM;   // A writer threads per row
constexpr int NPT = BK / TPR;                   // nodes of a K slice per A writer thread
static_assert(NPT % 8 == 0, "whole 16-byte chunks per thread");
constexpr int GEN_WARP0 = 2, EPI_WARP0 = GEN_WARP0 + NUM_GEN_WARPS;
constexpr int THREADS = 32 * (EPI_WARP0 + NUM_EPI_WARPS);
constexpr uint32_t TMEM_COLS = 2 * BNMAX;
constexpr size_t BAR_BYTES = 1024;
constexpr size_t SMEM_BYTES = 1024 + (size_t)STAGES * STAGE_BYTES + BAR_BYTES;
constexpr int MAX_TYPES = 256;
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA");
static_assert((4 * STAGES + 4 + 2 * UNIT_RING) * 8 + 8 + UNIT_RING * 4 <= BAR_BYTES, "barrier area");
static_assert(EPI_WARP0 % 4 == 2, "epilogue warps cover the four TMEM lane quadrants in turn");

struct VGArgs {
    const float *G;             // [n][N_pad] dLoss/dS without dust (sorted rows), the tiles' band columns
    const float *params;        // [npar][G_stride]
    const int *gidx;            // sorted row -> chunk galaxy
    const int2 *trange;
    VjpBand band;
    ColConst cc;
    int64_t n, G_stride, g_begin;
    int N_pad, KZ_pad, A_pad, n_z, row_old, dust_law, bump;
    int n_types, n_units;
    // unit type t: group gt (its T), ages [i0, i0 + na) (na <= 8), B box size bsel (32 << bsel rows)
    short t_i0[MAX_TYPES], t_na[MAX_TYPES], t_bsel[MAX_TYPES];
    float t_T[MAX_TYPES];
    int *sched;                 // unit counter, zero at launch
    float *what;                // out: [n][KZ_pad] the merged adjoint rows
    unsigned *err;
};

// Writes NPT consecutive values (nodes NPT h .. NPT h + NPT - 1 of the 32-node
// K slice) of row r as bf16 hi and lo into the A tiles, in the 64-byte
// swizzled K-major layout: row r holds 64 bytes, its 16-byte chunk c at
// position c ^ ((r >> 1) & 3).
__device__ __forceinline__ void write_a_row_part(unsigned char *a_hi, unsigned char *a_lo, int r, int h,
                                                 const float (&x)[NPT]) {
    uint32_t hw[NPT / 2], lw[NPT / 2];
#pragma unroll
    for (int q = 0; q < NPT / 2; ++q) {
        const __nv_bfloat162 hv = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
        const float2 rv = sub2(make_float2(x[2 * q], x[2 * q + 1]), __bfloat1622float2(hv));
        const __nv_bfloat162 lv = __floats2bfloat162_rn(rv.x, rv.y);
        hw[q] = *reinterpret_cast<const uint32_t *>(&hv);
        lw[q] = *reinterpret_cast<const uint32_t *>(&lv);
    }
    const int sw = (r >> 1) & 3;
#pragma unroll
    for (int cc = 0; cc < NPT / 8; ++cc) {
        const int chunk = ((NPT / 8) * h + cc) ^ sw;
        const size_t off = (size_t)r * 64 + (size_t)chunk * 16;
        *reinterpret_cast<uint4 *>(a_hi + off) = make_uint4(hw[4 * cc], hw[4 * cc + 1], hw[4 * cc + 2], hw[4 * cc + 3]);
        *reinterpret_cast<uint4 *>(a_lo + off) = make_uint4(lw[4 * cc], lw[4 * cc + 1], lw[4 * cc + 2], lw[4 * cc + 3]);
    }
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int LAW>   // bit 0: k0 tilted by delta (DSPS_DUST_SALIM); bit 1: the UV bump
__global__ void __launch_bounds__(THREADS, 1)
vjp_groups_tc_kernel(const __grid_constant__ CUtensorMap tmB_hi0, const __grid_constant__ CUtensorMap tmB_hi1,
                     const __grid_constant__ CUtensorMap tmB_hi2, const __grid_constant__ CUtensorMap tmB_hi3,
                     const __grid_constant__ CUtensorMap tmB_lo0, const __grid_constant__ CUtensorMap tmB_lo1,
                     const __grid_constant__ CUtensorMap tmB_lo2, const __grid_constant__ CUtensorMap tmB_lo3,
                     const __grid_constant__ VGArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + (size_t)STAGES * STAGE_BYTES);
    const uint32_t full0 = smem_u32(bars);                      // B loaded (TMA transaction bytes)
    const uint32_t afull0 = smem_u32(bars + STAGES);            // A written (one arrival per writer warp)
    const uint32_t empty0 = smem_u32(bars + 2 * STAGES);        // stage consumed (MMA commit)
    const uint32_t accf0 = smem_u32(bars + 3 * STAGES);         // accumulator ready
    const uint32_t acce0 = smem_u32(bars + 3 * STAGES + 2);     // accumulator read
    const uint32_t drain = smem_u32(bars + 3 * STAGES + 4);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 3 * STAGES + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    UnitRing ring;
    ring.full0 = smem_u32(bars + 3 * STAGES + 6);
    ring.empty0 = smem_u32(bars + 3 * STAGES + 6 + UNIT_RING);
    ring.slot = reinterpret_cast<volatile int *>(bars + 3 * STAGES + 6 + 2 * UNIT_RING);
    const uint32_t sbase = smem_u32(sm);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(afull0 + 8 * s, NUM_GEN_WARPS);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(accf0 + 8 * i, 1);
            mbar_init(acce0 + 8 * i, NUM_EPI_WARPS);
        }
        mbar_init(drain, 1);
        for (int i = 0; i < UNIT_RING; ++i) {
            mbar_init(ring.full0 + 8 * i, 1);
            mbar_init(ring.empty0 + 8 * i, 1 + NUM_GEN_WARPS + NUM_EPI_WARPS);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int armed[STAGES];
            for (int s = 0; s < STAGES; ++s) armed[s] = -1;
            bool ok = true;
            while (ok) {
                int u;
                if (!ring_claim(ring, a.sched, a.n_units, u, abort_flag, a.err) || u < 0) break;
                const int mt = u / a.n_types, t = u - mt * a.n_types;
                const int bsel = a.t_bsel[t], c0 = a.t_i0[t] * BK;
                const CUtensorMap *mh = bsel == 0 ? &tmB_hi0 : bsel == 1 ? &tmB_hi1 : bsel == 2 ? &tmB_hi2 : &tmB_hi3;
                const CUtensorMap *ml = bsel == 0 ? &tmB_lo0 : bsel == 1 ? &tmB_lo1 : bsel == 2 ? &tmB_lo2 : &tmB_lo3;
                const uint32_t bbytes = (uint32_t)(2 * (32 << bsel) * BK * 2);
                int kb0, kb1;
                vjp_band(a.band, a.trange, mt, a.N_pad, kb0, kb1);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u, abort_flag, a.err)) { ok = false; break; }
                    const uint32_t fb = full0 + 8 * stage;
                    const uint32_t st = sbase + stage * STAGE_BYTES;
                    mbar_expect_tx(fb, bbytes);
                    tma_load_2d(st + B_OFF, mh, fb, kb * BK, c0);
                    tma_load_2d(st + B_OFF + B_BYTES, ml, fb, kb * BK, c0);
                    armed[stage] = (int)phase;
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
            }
            for (int s = 0; s < STAGES; ++s)
                if (armed[s] >= 0) {
                    const long long t0 = clock64();
                    while (!mbar_try_wait(full0 + 8 * s, (uint32_t)armed[s]) && clock64() - t0 < WAIT_LIMIT) {
                    }
                }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int stage = 0, as = 0;
            uint32_t phase = 0, aphase = 0;
            bool ok = true;
            while (ok) {
                int u;
                if (!ring_next(ring, u, abort_flag, a.err) || u < 0) break;
                const int mt = u / a.n_types, t = u - mt * a.n_types;
                const uint32_t idesc = make_idesc(BM, (uint32_t)(a.t_na[t] * BK));
                int kb0, kb1;
                vjp_band(a.band, a.trange, mt, a.N_pad, kb0, kb1);
                if (!mbar_wait(acce0 + 8 * as, aphase ^ 1u, abort_flag, a.err)) break;
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(as * BNMAX);
                for (int kb = kb0; ok && kb < kb1; ++kb) {
                    if (!mbar_wait(full0 + 8 * stage, phase, abort_flag, a.err) ||
                        !mbar_wait(afull0 + 8 * stage, phase, abort_flag, a.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = sbase + stage * STAGE_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint64_t ah = sdesc_sw64(st + kk * 32);
                        const uint64_t al = sdesc_sw64(st + A_BYTES + kk * 32);
                        const uint64_t bh = sdesc_sw64(st + B_OFF + kk * 32);
                        const uint64_t bl = sdesc_sw64(st + B_OFF + B_BYTES + kk * 32);
                        mma_bf16_desc(d, ah, bh, idesc, (kb != kb0 || kk != 0) ? 1u : 0u);
                        mma_bf16_desc(d, ah, bl, idesc, 1u);
                        mma_bf16_desc(d, al, bh, idesc, 1u);
                    }
                    mma_commit(empty0 + 8 * stage);
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                mma_commit(accf0 + 8 * as);
                if (++as == 2) { as = 0; aphase ^= 1u; }
            }
            mma_commit(drain);
            const long long t0 = clock64();
            while (!mbar_try_wait(drain, 0) && clock64() - t0 < WAIT_LIMIT) {
            }
        }
    } else if (warp < EPI_WARP0) {
        // ---------------------------------------------------------------- A writers
        // thread t: row t / TPR of the tile, nodes NPT (t % TPR) .. + NPT - 1 of each K slice
        const int t = threadIdx.x - 32 * GEN_WARP0;
        const int r = t / TPR, h = t % TPR;
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        // the row's young and old dust values, kept while the units stay in one row tile
        int mt_cached = -1, kb0 = 0, kb1 = 0;
        float avy = 0.f, dly = 0.f, avo = 0.f, dlo = 0.f;
        while (ok) {
            int u = -1, have = 1;
            if (lane == 0) have = ring_next(ring, u, abort_flag, a.err) ? 1 : 0;
            have = __shfl_sync(0xffffffffu, have, 0);
            u = __shfl_sync(0xffffffffu, u, 0);
            if (!have || u < 0) break;
            const int mt = u / a.n_types, ty = u - mt * a.n_types;
            const int64_t rowg = (int64_t)mt * BM + r;
            if (mt != mt_cached) {
                vjp_band(a.band, a.trange, mt, a.N_pad, kb0, kb1);
                if (rowg < a.n) {
                    const int64_t g = a.g_begin + a.gidx[rowg];
                    avy = a.params[8 * a.G_stride + g];
                    dly = a.params[9 * a.G_stride + g];
                    avo = a.params[(int64_t)a.row_old * a.G_stride + g];
                    dlo = a.params[(int64_t)(a.row_old + 1) * a.G_stride + g];
                }
                mt_cached = mt;
            }
            // the row's curve for the unit's group (Sec. 3.4.1)
            float alpha = 0.f, beta = 0.f, eb = 0.f;
            if (rowg < a.n) {
                const float T = a.t_T[ty];
                float ax[AUX_STRIDE] = {};
                store_dust_aux(ax, group_dust_value(T, avy, avo), group_dust_value(T, dly, dlo), a.dust_law, a.bump);
                alpha = ax[0];
                beta = ax[1];
                eb = ax[6];
                // an invalid row (G = 0) gets a finite unit curve: its A row is exactly 0
                if (!(isfinite(alpha) && isfinite(beta) && isfinite(eb))) alpha = beta = eb = 0.f;
            }
            const float ustep = ex2_approx(beta * a.cc.dell);
            // G of the next two K slices is loaded while the current one is written
            constexpr int NQ = NPT / 4;
            float4 gv[NQ], gn[NQ], gn2[NQ];
            auto load_g = [&](int kb, float4 (&dst)[NQ]) {
                if (rowg < a.n) {
                    const float4 *src = reinterpret_cast<const float4 *>(a.G + rowg * a.N_pad + kb * BK + NPT * h);
#pragma unroll
                    for (int q = 0; q < NQ; ++q) dst[q] = src[q];
                } else {
#pragma unroll
                    for (int q = 0; q < NQ; ++q) dst[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            };
            load_g(kb0, gv);
            if (kb0 + 1 < kb1) load_g(kb0 + 1, gn);
            for (int kb = kb0; kb < kb1; ++kb) {
                if (kb + 2 < kb1) load_g(kb + 2, gn2);
                int got = 1;
                if (lane == 0) got = mbar_wait(empty0 + 8 * stage, phase ^ 1u, abort_flag, a.err) ? 1 : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) { ok = false; break; }
                const int n0 = kb * BK + NPT * h;
                float x[NPT];
                float uc = ex2_approx(beta * fmaf((float)n0, a.cc.dell, a.cc.ell0));
                // two nodes per paired FP32 operation (the power law itself is a
                // running product, node by node)
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float2 g2[2] = {make_float2(gv[q].x, gv[q].y), make_float2(gv[q].z, gv[q].w)};
#pragma unroll
                    for (int e = 0; e < 4; e += 2) {
                        const int nn = n0 + 4 * q + e;
                        float2 cn;
                        cn.x = uc;
                        uc *= ustep;
                        cn.y = uc;
                        uc *= ustep;
                        if constexpr ((LAW & 1) != 0) cn = mul2(cn, make_float2(__ldg(a.cc.k0 + nn), __ldg(a.cc.k0 + nn + 1)));
                        if constexpr ((LAW & 2) != 0)
                            cn = fma2v(splat2(eb), make_float2(__ldg(a.cc.bump + nn), __ldg(a.cc.bump + nn + 1)), cn);
                        const float2 ac = mul2(splat2(alpha), cn);
                        const float2 xv = mul2(g2[e >> 1], make_float2(ex2_approx(ac.x), ex2_approx(ac.y)));
                        x[4 * q + e] = xv.x;
                        x[4 * q + e + 1] = xv.y;
                    }
                }
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    gv[q] = gn[q];
                    gn[q] = gn2[q];
                }
                unsigned char *st = sm + (size_t)stage * STAGE_BYTES;
                write_a_row_part(st, st + A_BYTES, r, h, x);
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(afull0 + 8 * stage);
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int qd = warp & 3;
        const int row = qd * 32 + lane;
        const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
        int as = 0;
        uint32_t aphase = 0;
        while (true) {
            int u = -1, have = 1;
            if (lane == 0) have = ring_next(ring, u, abort_flag, a.err) ? 1 : 0;
            have = __shfl_sync(0xffffffffu, have, 0);
            u = __shfl_sync(0xffffffffu, u, 0);
            if (!have || u < 0) break;
            const int mt = u / a.n_types, ty = u - mt * a.n_types;
            const int i0 = a.t_i0[ty], na = a.t_na[ty];
            int got = 1;
            if (lane == 0) got = mbar_wait(accf0 + 8 * as, aphase, abort_flag, a.err) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) break;
            tc_fence_after();
            const int64_t rowg = (int64_t)mt * BM + row;
            // two neighbouring ages of one metallicity bin are adjacent in the
            // merged rows (kz = j A_pad + i): stored as one 8-byte pair where
            // the first age is even (A_pad is a multiple of 4)
            for (int c = 0; c < na;) {
                const bool pair = c + 1 < na && ((i0 + c) & 1) == 0;
                uint32_t v[32], w[32];
                tmem_ld32(tmem_base + lane_base + (uint32_t)(as * BNMAX + c * BK), v);
                if (pair) tmem_ld32(tmem_base + lane_base + (uint32_t)(as * BNMAX + (c + 1) * BK), w);
                const int cn = c + (pair ? 2 : 1);
                if (cn == na) {
                    // this warp's reads of the accumulator are done
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(acce0 + 8 * as);
                }
                if (rowg < a.n) {
                    float *dst = a.what + rowg * a.KZ_pad + (i0 + c);
                    if (pair) {
#pragma unroll
                        for (int j = 0; j < BK; ++j)
                            if (j < a.n_z)
                                *reinterpret_cast<float2 *>(dst + (int64_t)j * a.A_pad) =
                                    make_float2(__uint_as_float(v[j]), __uint_as_float(w[j]));
                    } else {
#pragma unroll
                        for (int j = 0; j < BK; ++j)
                            if (j < a.n_z) dst[(int64_t)j * a.A_pad] = __uint_as_float(v[j]);
                    }
                }
                c = cn;
            }
            if (++as == 2) { as = 0; aphase ^= 1u; }
        }
    }

    __syncwarp();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
    }
}

template <int LAW>
cudaError_t launch_law(const CUtensorMap (&bh)[4], const CUtensorMap (&bl)[4], const VGArgs &a, int grid,
                       cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(vjp_groups_tc_kernel<LAW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    vjp_groups_tc_kernel<LAW><<<grid, THREADS, SMEM_BYTES, s>>>(bh[0], bh[1], bh[2], bh[3], bl[0], bl[1], bl[2], bl[3],
                                                                a);
    return cudaGetLastError();
}

}  // namespace

bool agedep_vjp_tc_ok(const Ctx &c) {
    if (!c.d_Ldab_hi || !c.opts.dust_agedep || c.n_u != 1) return false;
    int types = 0;
    for (const DustGroup &g : c.dust_groups) types += (g.i1 - g.i0 + 7) / 8;
    return types <= MAX_TYPES;
}

cudaError_t launch_vjp_groups_tc(const Ctx &c, const Workspace &w, const FilterSet &fs, const float *params,
                                 int64_t G_stride, int64_t g_begin, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (!agedep_vjp_tc_ok(c)) return cudaErrorInvalidValue;
    CUtensorMap bh[4], bl[4];
    for (int b = 0; b < 4; ++b)
        if (!make_tmap(&bh[b], c.d_Ldab_hi, (uint64_t)c.N_pad, (uint64_t)c.KA_pad, 32u << b) ||
            !make_tmap(&bl[b], c.d_Ldab_lo, (uint64_t)c.N_pad, (uint64_t)c.KA_pad, 32u << b))
            return cudaErrorInvalidValue;
    VGArgs a{};
    a.G = reinterpret_cast<const float *>(w.shat);
    a.params = params;
    a.gidx = w.gidx;
    a.trange = w.trange;
    a.band = make_vjp_band(c, fs, c.opts.band_skip != 0);
    a.cc = make_col_const(c);
    a.n = n;
    a.G_stride = G_stride;
    a.g_begin = g_begin;
    a.N_pad = c.N_pad;
    a.KZ_pad = c.KZ_pad;
    a.A_pad = c.A_pad;
    a.n_z = c.n_z;
    a.row_old = c.row_dust_old;
    a.dust_law = c.opts.dust_law;
    a.bump = c.opts.dust_bump;
    // unit types: each group's ages in runs of up to eight (N = 32 per age)
    int nt = 0;
    for (const DustGroup &g : c.dust_groups)
        for (int i = g.i0; i < g.i1; i += 8) {
            const int na = g.i1 - i < 8 ? g.i1 - i : 8;
            a.t_i0[nt] = (short)i;
            a.t_na[nt] = (short)na;
            a.t_bsel[nt] = (short)(na <= 1 ? 0 : na <= 2 ? 1 : na <= 4 ? 2 : 3);
            a.t_T[nt] = g.T;
            ++nt;
        }
    a.n_types = nt;
    const int64_t n_mtiles = (n + BM - 1) / BM;
    if (n_mtiles * nt > INT32_MAX) return cudaErrorInvalidValue;
    a.n_units = (int)(n_mtiles * nt);
    a.sched = w.sched;
    a.what = w.what2;
    a.err = c.d_err;
    const int grid = a.n_units < c.num_sms ? a.n_units : c.num_sms;
    cudaError_t e = cudaMemsetAsync(w.sched, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    switch ((c.opts.dust_law == DSPS_DUST_SALIM ? 1 : 0) + (c.opts.dust_bump ? 2 : 0)) {
    case 0: return launch_law<0>(bh, bl, a, grid, s);
    case 1: return launch_law<1>(bh, bl, a, grid, s);
    case 2: return launch_law<2>(bh, bl, a, grid, s);
    default: return launch_law<3>(bh, bl, a, grid, s);
    }
}

}  // namespace dsps
