// agedep_tc.cu -- age-dependent dust (Sec. 3.4.1, Eq. agedep_dust_csp): the
// split-bf16 forward of every dust group in one tcgen05 launch.
//
// With a curve per age bin the spectrum of a galaxy is
//   L(lam) = sum_g F_g(lam) S_g(lam),   S_g = sum_{i in g} sum_j omega_ij L_ij,
// F_g = 10^(-0.4 Av_g c_g(lam)) the attenuation of group g (the age bins that
// share one curve: Av_g = (1 - T_g) Av_young + T_g Av_old, delta_g likewise).
// The weights of all ages come in the age-block order (weights kernel, mode
// W_OMEGA_BF16X2_AB): column ka = i * 32 + j, so that each age bin is one
// 32-wide K block and a group is a contiguous run of blocks.  Per work unit (a
// 128-galaxy tile and one of TC_PARTS interleaved subsets of its 128-wide
// wavelength tiles) and per wavelength tile, the groups are contracted one after
// another -- only the age blocks the tile's mask holds (ages where some galaxy
// of the tile has a non-zero weight); a group without such a block is skipped by
// every role -- into one of two TMEM accumulators (128 columns each).  The
// epilogue warps read the group's block of S_g, multiply it by F_g of each row
// and add it into a running sum held in registers (each thread one row and 64
// columns); after
// the last group the running sum goes once through the redshifted filter
// integral (epilogue.cuh, without dust: it is already in the sum).  So each
// element pays one light attenuation step per group and one filter reduction,
// where one launch per group paid the whole epilogue per group.
//
// Warp roles as in phot_tc.cu: warp 0 TMA producer (4-stage ring of {W_hi,
// W_lo, L_hi, L_lo} 32-wide K slices, 64-byte swizzle), warp 1 TMEM allocator
// and single-thread MMA issuer (per K slice six 128x128x16 tcgen05.mma
// kind::f16: hi.hi, hi.lo, lo.hi, two K steps), warps 2..9 epilogue (two warps
// per TMEM lane quadrant, 64 columns each, the running sum of those 64 columns
// in registers).  Every mbarrier wait is bounded; on
// expiry the kernel records DERR_TIMEOUT, lets its copies and MMAs land, frees
// TMEM and returns.
#include <cudaTypedefs.h>

#include "dsps_internal.cuh"
#include "epilogue.cuh"
#include "tc_common.cuh"
#include "f32x2.cuh"

namespace dsps {

namespace {

using namespace tc;

constexpr int BM = 128, BN = 128, BK = KBLOCK;
constexpr int STAGES = 4;
constexpr int NACC = 2;                      // TMEM accumulators (MMA runs NACC - 1 groups ahead)
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int NUM_EPI_WARPS = 8;
constexpr int THREADS = 32 * (2 + NUM_EPI_WARPS);
constexpr uint32_t TMEM_COLS = NACC * BN;    // accumulator i at column i * BN
constexpr int SPLIT = NUM_EPI_WARPS / 4;     // epilogue threads per row (one per column group)
constexpr int EPI_COLS = BN / SPLIT;         // columns of a row per epilogue thread
constexpr int QMAX = 16;
constexpr int MAX_GROUPS = AGEDEP_MAX_GROUPS;
constexpr size_t BAR_BYTES = 1024;
constexpr size_t COMB_BYTES = (size_t)(SPLIT > 1 ? SPLIT - 1 : 1) * BM * QMAX * 4;
constexpr size_t ACC_BYTES = (size_t)NUM_EPI_WARPS * 32 * QMAX * 4;   // each epilogue thread's filter sums
constexpr size_t SMEM_BYTES = 1024 + (size_t)STAGES * STAGE_BYTES + BAR_BYTES + COMB_BYTES + ACC_BYTES;
constexpr uint32_t IDESC = make_idesc(BM, BN);
static_assert(TMEM_COLS <= 512 && (TMEM_COLS & (TMEM_COLS - 1)) == 0, "TMEM allocation: a power of two up to 512");
static_assert((2 * STAGES + 2 * NACC + 4 + 2 * UNIT_RING) * 8 + UNIT_RING * 4 <= BAR_BYTES, "barrier area");
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA");
static_assert(NUM_EPI_WARPS % 4 == 0 && EPI_COLS % 32 == 0, "each epilogue thread: one row, whole 32-column blocks");

struct GArgs {
    const float *aux;              // Av_young, delta_young, s, valid, Av_old, delta_old (weights mode AB)
    const int2 *trange;            // per-tile redshift-shift ranges
    const unsigned *kmask;         // per-tile masks of the age blocks (4 words)
    const float4 *tab;
    ColConst cc;
    int m_last, n_mtiles, n_ntiles, parts, n_units;
    int band_skip, m_nz_lo, m_nz_hi, dust_law, bump;
    int n_groups;
    short g_i0[MAX_GROUPS], g_i1[MAX_GROUPS];   // age bins [i0, i1) of each group
    float g_T[MAX_GROUPS];                      // weight of the old-star dust values
    int64_t n;
    int *sched;                    // unit counter, zero at launch
    unsigned long long *kblk;      // 128 x 128 x 32 block products executed (profiling), or nullptr
    float *partial;                // [parts][n][4*Q4]
    // gradient pass (GRAD): the dust-free adjoint spectrum and the dust sums
    const float *G;                // [n][N_pad] dLoss/dS without dust, each row tile's band columns
    int N_pad;
    VjpBand band;                  // the columns of G written
    float *dpart;                  // out: [parts][n][4] the sums of grad_group_chunk, weighted per group
    unsigned *err;
};

// Wavelength tiles [nt0, nt1) of tile mt (as phot_tc.cu, with 128-wide tiles)
// and its mask of age blocks; an empty tile does no work.
__device__ __forceinline__ void tile_ranges(const GArgs &a, int mt, int &nt0, int &nt1, uint4 &km) {
    nt0 = 0;
    nt1 = a.n_ntiles;
    const unsigned *m = a.kmask + (size_t)mt * 4;
    km = make_uint4(__ldg(m), __ldg(m + 1), __ldg(m + 2), __ldg(m + 3));
    const int2 r = a.trange[mt];
    if (r.y < r.x || a.m_nz_hi < a.m_nz_lo || (km.x | km.y | km.z | km.w) == 0u) {
        nt1 = nt0;
        return;
    }
    if (!a.band_skip) return;
    const int n_lo = a.m_nz_lo - r.y - 2;
    const int n_hi = a.m_nz_hi - r.x + 1;
    if (n_hi < 0) { nt1 = nt0; return; }
    nt0 = n_lo <= 0 ? 0 : n_lo / BN;
    nt1 = min(a.n_ntiles, n_hi / BN + 1);
    if (nt1 < nt0) nt1 = nt0;
}

__device__ __forceinline__ unsigned mask_word(const uint4 &km, int w) {
    return w == 0 ? km.x : w == 1 ? km.y : w == 2 ? km.z : km.w;
}

// The tile's age blocks of group g in increasing order (a.n_groups..: none).
struct GroupBlocks {
    uint4 km;
    int b, hi;
    __device__ __forceinline__ GroupBlocks(const uint4 &k, int i0, int i1) : km(k), b(i0 - 1), hi(i1) {}
    // next set block in (b, hi), or hi
    __device__ __forceinline__ int next() {
        for (++b; b < hi; ++b) {
            const unsigned w = mask_word(km, b >> 5) >> (b & 31);
            if (w & 1u) return b;
            if (w == 0u) b = (b | 31);   // rest of this word empty
        }
        return hi;
    }
};

__device__ __forceinline__ bool group_present(const uint4 &km, int i0, int i1) {
    for (int w = i0 >> 5; w <= (i1 - 1) >> 5; ++w) {
        unsigned m = mask_word(km, w);
        const int lo = max(i0 - 32 * w, 0), hi = min(i1 - 32 * w, 32);
        m &= (hi >= 32 ? ~0u : ((1u << hi) - 1u)) & (~0u << lo);
        if (m) return true;
    }
    return false;
}

__device__ __forceinline__ int first_tile(int nt0, int part, int parts) {
    return nt0 + ((part - nt0 % parts) % parts + parts) % parts;
}

// 2^x in one MUFU instruction (PTX ex2.approx, relative error below 2^-22;
// flushes results below the normal range to 0).
__device__ __forceinline__ float ex2_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Adds 16 columns of a group's S_g (nodes n0 ..), times the group's
// attenuation F_g = 2^(alpha c_g) (Eq. attenuation, alpha = -0.4 log2(10) Av_g;
// c_g = [k0/4.05] u + e_g D0 with u = (lam/lam_V)^beta_g = 2^(beta_g ell)),
// into the running sum.  u is exact at the first node and stepped by the
// factor ustep = 2^(beta_g dell) between nodes (15 products at most: ~2e-6
// relative), one ex2 per node; the law and the bump are fixed at compile time
// so that the loop has no branch.  A row that is out of range or invalid
// accumulates whatever its accumulator holds: its sum is never integrated.
template <bool SALIM, bool BUMP>
__device__ __forceinline__ void add_group_chunk(float *run, const uint32_t (&r)[16], int n0, float alpha, float beta,
                                                float ustep, float e, const ColConst &cc) {
    float u = ex2_fast(beta * fmaf((float)n0, cc.dell, cc.ell0));
    // two nodes per paired FP32 operation (u itself is a running product)
#pragma unroll
    for (int j = 0; j < 16; j += 2) {
        float2 cn;
        cn.x = u;
        u *= ustep;
        cn.y = u;
        u *= ustep;
        if constexpr (SALIM) cn = mul2(cn, make_float2(__ldg(cc.k0 + n0 + j), __ldg(cc.k0 + n0 + j + 1)));
        if constexpr (BUMP) cn = fma2v(splat2(e), make_float2(__ldg(cc.bump + n0 + j), __ldg(cc.bump + n0 + j + 1)), cn);
        const float2 ac = mul2(splat2(alpha), cn);
        const float2 rr = fma2v(make_float2(__uint_as_float(r[j]), __uint_as_float(r[j + 1])),
                                make_float2(ex2_fast(ac.x), ex2_fast(ac.y)), make_float2(run[j], run[j + 1]));
        run[j] = rr.x;
        run[j + 1] = rr.y;
    }
}

// Gradient pass: with x_n = S_g,n F_g,n G_n (G the dust-free adjoint spectrum,
// dLoss/dS at node n), adds sum_n x_n c_g,n to sA and sum_n x_n dc_g,n/ddelta
// to sD over 16 nodes; dF/dAv = -0.4 ln10 c F and dF/ddelta = -0.4 ln10 Av
// dc/ddelta F (Eq. attenuation), with dc/ddelta = [k0/4.05] u ln(lam/lam_V) +
// e' D0 (e' = de/ddelta).  lell0 + n ldell = ln(lam_n / lam_V).
template <bool SALIM, bool BUMP>
__device__ __forceinline__ void grad_group_chunk(float &sA, float &sD, const float *gk, const uint32_t (&r)[16],
                                                 int n0, float alpha, float beta, float ustep, float e, float ed,
                                                 const ColConst &cc, float lell0, float ldell) {
    float u = ex2_fast(beta * fmaf((float)n0, cc.dell, cc.ell0));
    float lj = fmaf((float)n0, ldell, lell0);   // ln(lam_n / lam_V), stepped
    // two nodes per paired FP32 operation; u, lj and the two sums run node by node
#pragma unroll
    for (int j = 0; j < 16; j += 2) {
        float2 cp, l2;
        cp.x = u;
        u *= ustep;
        cp.y = u;
        u *= ustep;
        l2.x = lj;
        lj += ldell;
        l2.y = lj;
        lj += ldell;
        if constexpr (SALIM) cp = mul2(cp, make_float2(__ldg(cc.k0 + n0 + j), __ldg(cc.k0 + n0 + j + 1)));
        const float2 bj = BUMP ? make_float2(__ldg(cc.bump + n0 + j), __ldg(cc.bump + n0 + j + 1)) : splat2(0.f);
        const float2 cn = BUMP ? fma2v(splat2(e), bj, cp) : cp;
        const float2 ac = mul2(splat2(alpha), cn);
        const float2 x = mul2(mul2(make_float2(__uint_as_float(r[j]), __uint_as_float(r[j + 1])),
                                   make_float2(ex2_fast(ac.x), ex2_fast(ac.y))),
                              make_float2(gk[j], gk[j + 1]));
        float2 dc = mul2(cp, l2);
        if constexpr (BUMP) dc = fma2v(splat2(ed), bj, dc);
        sA = fmaf(x.x, cn.x, sA);
        sD = fmaf(x.x, dc.x, sD);
        sA = fmaf(x.y, cn.y, sA);
        sD = fmaf(x.y, dc.y, sD);
    }
}

template <int Q4, int LAW, bool GRAD>
__global__ void __launch_bounds__(THREADS, 1)
phot_tc_groups_kernel(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
                      const __grid_constant__ CUtensorMap tmB_hi, const __grid_constant__ CUtensorMap tmB_lo,
                      const __grid_constant__ GArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + (size_t)STAGES * STAGE_BYTES);
    const uint32_t full0 = smem_u32(bars);
    const uint32_t empty0 = smem_u32(bars + STAGES);
    const uint32_t accf0 = smem_u32(bars + 2 * STAGES);
    const uint32_t acce0 = smem_u32(bars + 2 * STAGES + NACC);
    const uint32_t ebar = smem_u32(bars + 2 * STAGES + 2 * NACC);
    const uint32_t drain = smem_u32(bars + 2 * STAGES + 2 * NACC + 1);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 2 * NACC + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    UnitRing ring;
    ring.full0 = smem_u32(bars + 2 * STAGES + 2 * NACC + 4);
    ring.empty0 = smem_u32(bars + 2 * STAGES + 2 * NACC + 4 + UNIT_RING);
    ring.slot = reinterpret_cast<volatile int *>(bars + 2 * STAGES + 2 * NACC + 4 + 2 * UNIT_RING);
    float *comb = reinterpret_cast<float *>(sm + (size_t)STAGES * STAGE_BYTES + BAR_BYTES);
    // the filter sums of each epilogue thread live in shared memory between
    // wavelength tiles (the group loop keeps 64 running-sum registers)
    float *accbuf = comb + COMB_BYTES / 4;
    const uint32_t sbase = smem_u32(sm);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int i = 0; i < NACC; ++i) {
            mbar_init(accf0 + 8 * i, 1);
            mbar_init(acce0 + 8 * i, NUM_EPI_WARPS);
        }
        mbar_init(ebar, NUM_EPI_WARPS);
        mbar_init(drain, 1);
        for (int i = 0; i < UNIT_RING; ++i) {
            mbar_init(ring.full0 + 8 * i, 1);
            mbar_init(ring.empty0 + 8 * i, 1 + NUM_EPI_WARPS);
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
                const int mt = u / a.parts, part = u - mt * a.parts;
                int nt0, nt1;
                uint4 km;
                tile_ranges(a, mt, nt0, nt1, km);
                for (int nt = first_tile(nt0, part, a.parts); ok && nt < nt1; nt += a.parts)
                    for (int g = 0; ok && g < a.n_groups; ++g) {
                        GroupBlocks it(km, a.g_i0[g], a.g_i1[g]);
                        for (int kb = it.next(); kb < it.hi; kb = it.next()) {
                            if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u, abort_flag, a.err)) { ok = false; break; }
                            const uint32_t fb = full0 + 8 * stage;
                            const uint32_t st = sbase + stage * STAGE_BYTES;
                            mbar_expect_tx(fb, STAGE_BYTES);
                            tma_load_2d(st, &tmA_hi, fb, kb * BK, mt * BM);
                            tma_load_2d(st + A_BYTES, &tmA_lo, fb, kb * BK, mt * BM);
                            tma_load_2d(st + 2 * A_BYTES, &tmB_hi, fb, kb * BK, nt * BN);
                            tma_load_2d(st + 2 * A_BYTES + B_BYTES, &tmB_lo, fb, kb * BK, nt * BN);
                            armed[stage] = (int)phase;
                            if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                        }
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
            unsigned long long nblk = 0;
            while (ok) {
                int u;
                if (!ring_next(ring, u, abort_flag, a.err) || u < 0) break;
                const int mt = u / a.parts, part = u - mt * a.parts;
                int nt0, nt1;
                uint4 km;
                tile_ranges(a, mt, nt0, nt1, km);
                for (int nt = first_tile(nt0, part, a.parts); ok && nt < nt1; nt += a.parts)
                    for (int g = 0; ok && g < a.n_groups; ++g) {
                        if (!group_present(km, a.g_i0[g], a.g_i1[g])) continue;
                        if (!mbar_wait(acce0 + 8 * as, aphase ^ 1u, abort_flag, a.err)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t d = tmem_base + (uint32_t)(as * BN);
                        GroupBlocks it(km, a.g_i0[g], a.g_i1[g]);
                        bool first = true;
                        for (int kb = it.next(); kb < it.hi; kb = it.next()) {
                            ++nblk;
                            if (!mbar_wait(full0 + 8 * stage, phase, abort_flag, a.err)) { ok = false; break; }
                            tc_fence_after();
                            const uint32_t st = sbase + stage * STAGE_BYTES;
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk) {
                                const uint64_t ah = sdesc_sw64(st + kk * 32);
                                const uint64_t al = sdesc_sw64(st + A_BYTES + kk * 32);
                                const uint64_t bh = sdesc_sw64(st + 2 * A_BYTES + kk * 32);
                                const uint64_t bl = sdesc_sw64(st + 2 * A_BYTES + B_BYTES + kk * 32);
                                mma_bf16_desc(d, ah, bh, IDESC, (!first || kk != 0) ? 1u : 0u);
                                mma_bf16_desc(d, ah, bl, IDESC, 1u);
                                mma_bf16_desc(d, al, bh, IDESC, 1u);
                            }
                            mma_commit(empty0 + 8 * stage);
                            if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                            first = false;
                        }
                        if (!ok) break;
                        mma_commit(accf0 + 8 * as);
                        if (++as == NACC) { as = 0; aphase ^= 1u; }
                    }
            }
            if (a.kblk) atomicAdd(a.kblk, nblk);
            mma_commit(drain);
            const long long t0 = clock64();
            while (!mbar_try_wait(drain, 0) && clock64() - t0 < WAIT_LIMIT) {
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int qd = warp & 3;
        const int cg = (warp - 2) >> 2;   // column group
        const int row = qd * 32 + lane;
        const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
        int as = 0;
        uint32_t aphase = 0, ephase = 0;
        bool ok = true;
        while (ok) {
            int u = -1, have = 1;
            if (lane == 0) have = ring_next(ring, u, abort_flag, a.err) ? 1 : 0;
            have = __shfl_sync(0xffffffffu, have, 0);
            u = __shfl_sync(0xffffffffu, u, 0);
            if (!have || u < 0) break;
            const int mt = u / a.parts, part = u - mt * a.parts;
            int nt0, nt1;
            uint4 km;
            tile_ranges(a, mt, nt0, nt1, km);
            const int64_t rowg = (int64_t)mt * BM + row;
            // the row's dust values (the redshift interpolation is read again
            // for each wavelength tile's filter integral)
            const bool valid = load_row_const(a.aux, rowg, a.n).valid;
            float avy = 0.f, dly = 0.f, avo = 0.f, dlo = 0.f;
            if (rowg < a.n) {
                const float *ax = a.aux + rowg * AUX_STRIDE;
                avy = ax[0];
                dly = ax[1];
                avo = ax[4];
                dlo = ax[5];
            }
            float *accs = accbuf + (threadIdx.x - 64) * QMAX;
#pragma unroll
            for (int q = 0; q < 4 * Q4; ++q) accs[q] = 0.f;
            // the dust law (LAW bit 0: k0 tilted by delta; bit 1: the bump), fixed at compile time
            constexpr bool SALIM = (LAW & 1) != 0, BUMP = (LAW & 2) != 0;
            constexpr int NCHUNK = EPI_COLS / 16;
            // gradient pass: sum_g (1 - T_g) s_g, T_g s_g, (1 - T_g) Av_g t_g,
            // T_g Av_g t_g over this thread's columns, and G's columns
            float dsum[4] = {0.f, 0.f, 0.f, 0.f};
            int gc0 = 0, gc1 = 0;
            if constexpr (GRAD) {
                int kb0, kb1;
                vjp_band(a.band, a.trange, mt, a.N_pad, kb0, kb1);
                gc0 = 32 * kb0;
                gc1 = 32 * kb1;
            }
            const float lell0 = a.cc.ell0 * 0.69314718055994531f, ldell = a.cc.dell * 0.69314718055994531f;
            for (int nt = first_tile(nt0, part, a.parts); ok && nt < nt1; nt += a.parts) {
                const int nb = nt * BN + cg * EPI_COLS;
                // forward: the running sum; gradient pass: G at the columns
                float run[EPI_COLS / 32][32];
#pragma unroll
                for (int c = 0; c < EPI_COLS / 32; ++c) {
                    // (nb and the band edges are multiples of 32: a 32-column block is in or out)
                    const int col0 = nb + c * 32;
                    const bool in = GRAD && valid && rowg < a.n && col0 >= gc0 && col0 < gc1;
                    const float4 *src = reinterpret_cast<const float4 *>(a.G + (in ? rowg * a.N_pad + col0 : 0));
#pragma unroll
                    for (int j4 = 0; j4 < 8; ++j4) {
                        const float4 v = in ? src[j4] : make_float4(0.f, 0.f, 0.f, 0.f);
                        run[c][4 * j4] = v.x;
                        run[c][4 * j4 + 1] = v.y;
                        run[c][4 * j4 + 2] = v.z;
                        run[c][4 * j4 + 3] = v.w;
                    }
                }
                bool any = false;
                for (int g = 0; ok && g < a.n_groups; ++g) {
                    if (!group_present(km, a.g_i0[g], a.g_i1[g])) continue;
                    int got = 1;
                    if (lane == 0) got = mbar_wait(accf0 + 8 * as, aphase, abort_flag, a.err) ? 1 : 0;
                    got = __shfl_sync(0xffffffffu, got, 0);
                    if (!got) { ok = false; break; }
                    tc_fence_after();
                    // the group's curve (Sec. 3.4.1), as the weights kernel forms it
                    const float T = a.g_T[g];
                    const float Avg = group_dust_value(T, avy, avo), dlg = group_dust_value(T, dly, dlo);
                    const float alpha = -0.4f * 3.32192809488736235f * Avg;
                    const float beta = SALIM ? dlg : dlg - 0.7f;
                    const float eg = BUMP ? (0.85f - 1.9f * dlg) * (1.f / 4.05f) : 0.f;
                    const float ustep = ex2_fast(beta * a.cc.dell);
                    const uint32_t tacc = tmem_base + lane_base + (uint32_t)(as * BN + cg * EPI_COLS);
                    float sA = 0.f, sD = 0.f;
                    // chunk c + 1 is read from TMEM while chunk c is added
                    uint32_t rb[2][16];
                    tmem_ld16_async(tacc, rb[0]);
                    tmem_wait_ld16(rb[0]);
#pragma unroll
                    for (int c = 0; c < NCHUNK; ++c) {
                        if (c == NCHUNK - 1) {
                            // this warp's reads of the accumulator are done
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(acce0 + 8 * as);
                        }
                        if (c + 1 < NCHUNK) tmem_ld16_async(tacc + (c + 1) * 16, rb[(c + 1) & 1]);
                        if constexpr (GRAD)
                            grad_group_chunk<SALIM, BUMP>(sA, sD, &run[c >> 1][(c & 1) * 16], rb[c & 1], nb + c * 16,
                                                          alpha, beta, ustep, eg, BUMP ? -1.9f / 4.05f : 0.f, a.cc,
                                                          lell0, ldell);
                        else
                            add_group_chunk<SALIM, BUMP>(&run[c >> 1][(c & 1) * 16], rb[c & 1], nb + c * 16, alpha,
                                                         beta, ustep, eg, a.cc);
                        if (c + 1 < NCHUNK) tmem_wait_ld16(rb[(c + 1) & 1]);
                    }
                    if constexpr (GRAD) {
                        dsum[0] = fmaf(1.f - T, sA, dsum[0]);
                        dsum[1] = fmaf(T, sA, dsum[1]);
                        dsum[2] = fmaf((1.f - T) * Avg, sD, dsum[2]);
                        dsum[3] = fmaf(T * Avg, sD, dsum[3]);
                    }
                    any = true;
                    if (++as == NACC) { as = 0; aphase ^= 1u; }
                }
                if (!ok) break;
                if (GRAD || !any || !valid) continue;
                // the attenuated spectrum of the tile: one filter integral
                const RowConst rc = load_row_const(a.aux, rowg, a.n);
                float acc[4 * Q4];
#pragma unroll
                for (int q = 0; q < 4 * Q4; ++q) acc[q] = accs[q];
                Slide sl;
#pragma unroll
                for (int c = 0; c < EPI_COLS / 32; ++c)
#pragma unroll
                    for (int j = 0; j < 32; j += 2)
                        epi_node_plain2<Q4>(acc, sl, run[c][j], run[c][j + 1], nb + c * 32 + j, rc, a.cc, a.tab,
                                            a.m_last);
                epi_close<Q4>(acc, sl, nb + EPI_COLS, rc, a.tab, a.m_last);
#pragma unroll
                for (int q = 0; q < 4 * Q4; ++q) accs[q] = acc[q];
            }
            if (!ok) break;
            float acc[4 * Q4];
#pragma unroll
            for (int q = 0; q < 4 * Q4; ++q) acc[q] = GRAD ? (q < 4 ? dsum[q] : 0.f) : accs[q];
            // combine the column groups of each row in a fixed order (bounded barrier)
            if (cg > 0) {
                float *cr = comb + ((cg - 1) * BM + row) * QMAX;
#pragma unroll
                for (int q = 0; q < 4 * Q4; ++q) cr[q] = acc[q];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(ebar);
            int got = 1;
            if (lane == 0) got = mbar_wait(ebar, ephase, abort_flag, a.err) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            ephase ^= 1u;
            if (!got) break;
            if (cg == 0 && rowg < a.n) {
#pragma unroll
                for (int k = 1; k < SPLIT; ++k) {
                    const float *cr = comb + ((k - 1) * BM + row) * QMAX;
#pragma unroll
                    for (int q = 0; q < 4 * Q4; ++q) acc[q] += cr[q];
                }
                if constexpr (GRAD) {
                    *reinterpret_cast<float4 *>(a.dpart + ((int64_t)part * a.n + rowg) * 4) =
                        make_float4(acc[0], acc[1], acc[2], acc[3]);
                } else {
                    float4 *dst = reinterpret_cast<float4 *>(a.partial + ((int64_t)part * a.n + rowg) * (4 * Q4));
#pragma unroll
                    for (int qq = 0; qq < Q4; ++qq)
                        dst[qq] = make_float4(acc[4 * qq], acc[4 * qq + 1], acc[4 * qq + 2], acc[4 * qq + 3]);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(ebar);
            got = 1;
            if (lane == 0) got = mbar_wait(ebar, ephase, abort_flag, a.err) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            ephase ^= 1u;
            if (!got) break;
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

template <int Q4, int LAW, bool GRAD>
cudaError_t launch_qlg(const CUtensorMap &ah, const CUtensorMap &al, const CUtensorMap &bh, const CUtensorMap &bl,
                       const GArgs &a, int grid, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(phot_tc_groups_kernel<Q4, LAW, GRAD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    phot_tc_groups_kernel<Q4, LAW, GRAD><<<grid, THREADS, SMEM_BYTES, s>>>(ah, al, bh, bl, a);
    return cudaGetLastError();
}

template <int Q4, int LAW>
cudaError_t launch_ql(const CUtensorMap &ah, const CUtensorMap &al, const CUtensorMap &bh, const CUtensorMap &bl,
                      const GArgs &a, int grid, cudaStream_t s) {
    return a.G ? launch_qlg<Q4, LAW, true>(ah, al, bh, bl, a, grid, s)
               : launch_qlg<Q4, LAW, false>(ah, al, bh, bl, a, grid, s);
}

template <int Q4>
cudaError_t launch_q4(const CUtensorMap &ah, const CUtensorMap &al, const CUtensorMap &bh, const CUtensorMap &bl,
                      const GArgs &a, int grid, cudaStream_t s) {
    switch ((a.dust_law == DSPS_DUST_SALIM ? 1 : 0) + (a.bump ? 2 : 0)) {
    case 0: return launch_ql<Q4, 0>(ah, al, bh, bl, a, grid, s);
    case 1: return launch_ql<Q4, 1>(ah, al, bh, bl, a, grid, s);
    case 2: return launch_ql<Q4, 2>(ah, al, bh, bl, a, grid, s);
    default: return launch_ql<Q4, 3>(ah, al, bh, bl, a, grid, s);
    }
}

}  // namespace

bool agedep_fused_ok(const Ctx &c) {
    return c.KA_pad > 0 && c.opts.dust_agedep && c.n_u == 1 && (int)c.dust_groups.size() <= MAX_GROUPS &&
           c.kmask_words == 4;
}

cudaError_t launch_phot_tc_groups(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, int *parts,
                                  cudaStream_t s, const float *G) {
    *parts = TC_PARTS;
    if (n <= 0) return cudaSuccess;
    if (fs.Q > QMAX || !agedep_fused_ok(c)) return cudaErrorInvalidValue;
    CUtensorMap ah, al, bh, bl;
    if (!make_tmap(&ah, w.whi, (uint64_t)c.KA_pad, (uint64_t)n, BM) ||
        !make_tmap(&al, w.wlo, (uint64_t)c.KA_pad, (uint64_t)n, BM) ||
        !make_tmap(&bh, c.d_Lab_hi, (uint64_t)c.KA_pad, (uint64_t)c.N_pad, BN) ||
        !make_tmap(&bl, c.d_Lab_lo, (uint64_t)c.KA_pad, (uint64_t)c.N_pad, BN))
        return cudaErrorInvalidValue;
    GArgs a{};
    a.aux = w.aux;
    a.trange = w.trange;
    a.kmask = w.kmask;
    a.tab = reinterpret_cast<const float4 *>(fs.d_tab);
    a.cc = make_col_const(c);
    a.m_last = fs.m_rows - 1;
    a.n_mtiles = (int)((n + BM - 1) / BM);
    a.n_ntiles = c.N_pad / BN;
    a.parts = TC_PARTS;
    a.n_units = a.n_mtiles * TC_PARTS;
    a.band_skip = c.opts.band_skip ? 1 : 0;
    a.m_nz_lo = fs.m_nz_lo;
    a.m_nz_hi = fs.m_nz_hi;
    a.dust_law = c.opts.dust_law;
    a.bump = c.opts.dust_bump ? 1 : 0;
    a.n_groups = (int)c.dust_groups.size();
    for (int g = 0; g < a.n_groups; ++g) {
        a.g_i0[g] = (short)c.dust_groups[g].i0;
        a.g_i1[g] = (short)c.dust_groups[g].i1;
        a.g_T[g] = c.dust_groups[g].T;
    }
    a.n = n;
    a.sched = w.sched;
    a.kblk = w.stats ? w.stats + 2 : nullptr;
    a.partial = w.partial;
    a.G = G;
    a.N_pad = c.N_pad;
    a.band = make_vjp_band(c, fs, c.opts.band_skip != 0);
    a.dpart = w.partial;
    a.err = c.d_err;
    const int grid = a.n_units < c.num_sms ? a.n_units : c.num_sms;
    cudaError_t e = cudaMemsetAsync(w.sched, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    switch (fs.Q4) {
    case 1: return launch_q4<1>(ah, al, bh, bl, a, grid, s);
    case 2: return launch_q4<2>(ah, al, bh, bl, a, grid, s);
    case 3: return launch_q4<3>(ah, al, bh, bl, a, grid, s);
    default: return launch_q4<4>(ah, al, bh, bl, a, grid, s);
    }
}

}  // namespace dsps
