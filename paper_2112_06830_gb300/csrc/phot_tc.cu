// phot_tc.cu -- tcgen05 (5th-generation tensor core) form of the fused
// photometry kernel for sm_103a.
//
// Contraction S[g, n] = sum_k omega[g, k] L[k, n] (Eq. full_mdf), M = galaxies,
// N = wavelength nodes, K = n_age * n_z, in the split-bf16 form
//   S = W_hi L_hi + W_hi L_lo + W_lo L_hi     (bf16 operands, FP32 accumulate)
// where W = omega * 2^E_k and L = L_ssp * 2^-E_k are split into bf16 hi + lo.
//
// Persistent CTAs (one per SM) take work units -- a 128-galaxy tile and one of
// TC_PARTS interleaved subsets of its wavelength tiles -- from a global counter
// (tc::UnitRing), so that units of unequal cost balance across SMs; each tile sweeps the
// 256-wide wavelength tiles inside its redshifted filter band, and contracts
// only the K blocks (metallicity-major K) where some row's weights are non-zero
// (tile_ranges, KbIter).  Warp roles:
//   warp 0      TMA producer: 4-stage ring of {W_hi, W_lo, L_hi, L_lo} K-slices
//               (32 bf16 = 64 B rows, 64-byte swizzle), one mbarrier per stage.
//   warp 1      TMEM allocator and single-thread MMA issuer: per K-slice six
//               128x256x16 tcgen05.mma kind::f16 into one of two TMEM
//               accumulators (2 x 256 columns), tcgen05.commit to free the
//               stage and, per tile, to hand the accumulator to the epilogue.
//   warps 2..9  epilogue: tcgen05.ld 32x32b (one galaxy row per thread), dust,
//               redshifted filter lookup and wavelength reduction in registers
//               (epilogue.cuh); two warps per TMEM lane quadrant split the 256
//               columns.  No spectrum leaves the SM.
// Every wait on an mbarrier is bounded; on expiry the kernel records
// DERR_TIMEOUT, lets its in-flight copies and MMAs land, frees TMEM and returns.
#include <cudaTypedefs.h>

#include <cmath>

#include "dsps_internal.cuh"
#include "epilogue.cuh"
#include "tc_common.cuh"

namespace dsps {

namespace {

using namespace tc;

constexpr int BM = 128, BN = 256, BK = 32;
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int NUM_EPI_WARPS = 8;
constexpr int THREADS = 32 * (2 + NUM_EPI_WARPS);
constexpr uint32_t TMEM_COLS = 2 * BN;
constexpr int QMAX = 16;
constexpr size_t BAR_BYTES = 1024;
constexpr size_t COMB_BYTES = (size_t)BM * 3 * QMAX * 4;   // up to 3 sums per filter (gradient mode)
constexpr size_t SMEM_BYTES = 1024 + (size_t)STAGES * STAGE_BYTES + BAR_BYTES + COMB_BYTES;

struct TArgs {
    const float *aux;
    const int2 *trange;             // per-tile redshift-shift ranges from the weights kernel
    const unsigned *kmask;          // per-tile kz-block masks from the weights kernel, or nullptr
    int kmw;                        // mask words per tile
    const int2 *urange;             // per-tile log U section ranges from the weights kernel
    int sec_blocks, n_sec;          // K blocks per section, sections (log U bins)
    const float4 *tab;
    ColConst cc;
    int m_last, n_mtiles, n_ntiles, kblocks, parts, n_units;
    int band_skip, m_nz_lo, m_nz_hi;
    int64_t n;
    int *sched;                     // unit counter, zero at launch
    float *partial;                 // [parts][n][4*Q4]
    unsigned long long *kblk;       // 128 x 256 x 32 block products executed (profiling)
    unsigned *err;
};

// K blocks of a tile: the blocks set in a mask of one section's blocks (up to
// 128, held in registers) in each section (log U bin) of the tile's range,
// which spans the K blocks [lo, hi) (whole sections).
struct TileMask {
    uint4 w;
    int lo, hi;
};

// Wavelength tiles [nt0, nt1) that galaxy tile mt needs and its K-block mask
// (all blocks without skipping), from the tile's exact ranges over its valid
// rows.  A wavelength tile whose interpolation rows (grid indices n + i0 - 1
// .. n + i0 + 2) fall outside the band [m_nz_lo, m_nz_hi] of non-zero
// transmission for every i0 of the tile, and a K block where every row's
// weights are zero, contribute exact zeros and are skipped.  A tile with no
// non-zero weight does no work.
__device__ __forceinline__ void tile_ranges(const TArgs &a, int mt, int &nt0, int &nt1, TileMask &km) {
    nt0 = 0;
    nt1 = a.n_ntiles;
    km.w = make_uint4(~0u, ~0u, ~0u, ~0u);
    km.lo = 0;
    km.hi = a.n_sec * a.sec_blocks;
    if (!a.band_skip) return;
    const int2 r = a.trange[mt];
    if (a.kmask) {
        const unsigned *m = a.kmask + (size_t)mt * a.kmw;
        km.w = make_uint4(__ldg(m), a.kmw > 1 ? __ldg(m + 1) : 0u, a.kmw > 2 ? __ldg(m + 2) : 0u,
                          a.kmw > 3 ? __ldg(m + 3) : 0u);
    }
    const int2 ur = a.urange[mt];
    km.lo = ur.x * a.sec_blocks;
    km.hi = (ur.y + 1) * a.sec_blocks;
    if (r.y < r.x || a.m_nz_hi < a.m_nz_lo || (km.w.x | km.w.y | km.w.z | km.w.w) == 0u || ur.y < ur.x) {
        nt1 = nt0;
        return;
    }
    const int n_lo = a.m_nz_lo - r.y - 2;
    const int n_hi = a.m_nz_hi - r.x + 1;
    if (n_hi < 0) { nt1 = nt0; return; }
    nt0 = n_lo <= 0 ? 0 : n_lo / BN;
    nt1 = min(a.n_ntiles, n_hi / BN + 1);
    if (nt1 < nt0) nt1 = nt0;
}

// The tile's K blocks in increasing order: block base + b for the sections
// base = lo, lo + sec_blocks, .. < hi and the bits b < sec_blocks of the mask.
// The producer and the MMA issuer step it once per K block, so a step keeps
// the current mask word and clears its lowest bit (a few instructions).
struct KbIter {
    uint4 w;
    int base, hi, sb, wi, kblocks;
    unsigned cur;
    __device__ __forceinline__ KbIter(const TArgs &a, const TileMask &km)
        : w(km.w), base(km.lo), hi(km.hi), sb(a.sec_blocks), wi(0), kblocks(a.kblocks), cur(km.w.x) {}
    __device__ __forceinline__ unsigned word(int i) const {
        return i == 0 ? w.x : i == 1 ? w.y : i == 2 ? w.z : w.w;
    }
    // next block, a.kblocks after the last
    __device__ __forceinline__ int next() {
        while (base < hi) {
            if (cur) {
                const int b = (wi << 5) + __ffs(cur) - 1;
                cur &= cur - 1;
                if (b < sb) return base + b;
                cur = 0;   // the rest of this section's mask lies beyond its blocks
                wi = 3;
            } else if (wi < 3 && ((wi + 1) << 5) < sb) {
                cur = word(++wi);
            } else {
                base += sb;
                wi = 0;
                cur = w.x;
            }
        }
        return kblocks;
    }
};

// Wavelength tile nt belongs to part nt mod parts, whatever the tile's range:
// every galaxy's partial sums then add the same non-zero terms in the same
// order in any batch (skipped tiles would only have added exact zeros).
__device__ __forceinline__ int first_tile(int nt0, int part, int parts) {
    return nt0 + ((part - nt0 % parts) % parts + parts) % parts;
}

template <int Q4, bool GRAD>
__global__ void __launch_bounds__(THREADS, 1)
phot_tc_kernel(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
               const __grid_constant__ CUtensorMap tmB_hi, const __grid_constant__ CUtensorMap tmB_lo,
               const TArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + (size_t)STAGES * STAGE_BYTES);
    const uint32_t full0 = smem_u32(bars);
    const uint32_t empty0 = smem_u32(bars + STAGES);
    const uint32_t accf0 = smem_u32(bars + 2 * STAGES);
    const uint32_t acce0 = smem_u32(bars + 2 * STAGES + 2);
    const uint32_t ebar = smem_u32(bars + 2 * STAGES + 4);
    const uint32_t drain = smem_u32(bars + 2 * STAGES + 5);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 6);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    UnitRing ring;
    ring.full0 = smem_u32(bars + 2 * STAGES + 8);
    ring.empty0 = smem_u32(bars + 2 * STAGES + 8 + UNIT_RING);
    ring.slot = reinterpret_cast<volatile int *>(bars + 2 * STAGES + 8 + 2 * UNIT_RING);
    float *comb = reinterpret_cast<float *>(sm + (size_t)STAGES * STAGE_BYTES + BAR_BYTES);
    const uint32_t sbase = smem_u32(sm);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int i = 0; i < 2; ++i) {
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
                if (!ring_claim(ring, a.sched, a.n_units, u, abort_flag, a.err)) break;
                if (u < 0) break;
                const int mt = u / a.parts, part = u - mt * a.parts;
                int nt0, nt1;
                TileMask km;
                tile_ranges(a, mt, nt0, nt1, km);
                for (int nt = first_tile(nt0, part, a.parts); ok && nt < nt1; nt += a.parts) {
                    KbIter it(a, km);
                    for (int kb = it.next(); kb < a.kblocks; kb = it.next()) {
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
            // Let every armed copy land before the CTA can exit.
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
            unsigned long long nblk = 0;
            bool ok = true;
            while (ok) {
                int u;
                if (!ring_next(ring, u, abort_flag, a.err) || u < 0) break;
                const int mt = u / a.parts, part = u - mt * a.parts;
                int nt0, nt1;
                TileMask km;
                tile_ranges(a, mt, nt0, nt1, km);
                for (int nt = first_tile(nt0, part, a.parts); ok && nt < nt1; nt += a.parts) {
                    if (!mbar_wait(acce0 + 8 * as, aphase ^ 1u, abort_flag, a.err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t d = tmem_base + (uint32_t)(as * BN);
                    KbIter it(a, km);
                    bool first = true;
                    for (int kb = it.next(); kb < a.kblocks; kb = it.next()) {
                        if (!mbar_wait(full0 + 8 * stage, phase, abort_flag, a.err)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t st = sbase + stage * STAGE_BYTES;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            const uint64_t ah = sdesc_sw64(st + kk * 32);
                            const uint64_t al = sdesc_sw64(st + A_BYTES + kk * 32);
                            const uint64_t bh = sdesc_sw64(st + 2 * A_BYTES + kk * 32);
                            const uint64_t bl = sdesc_sw64(st + 2 * A_BYTES + B_BYTES + kk * 32);
                            mma_bf16(d, ah, bh, (!first || kk != 0) ? 1u : 0u);
                            mma_bf16(d, ah, bl, 1u);
                            mma_bf16(d, al, bh, 1u);
                        }
                        mma_commit(empty0 + 8 * stage);
                        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                        ++nblk;
                        first = false;
                    }
                    if (!ok) break;
                    mma_commit(accf0 + 8 * as);
                    if (++as == 2) { as = 0; aphase ^= 1u; }
                }
            }
            // Every MMA issued so far completes before this commit arrives.
            mma_commit(drain);
            const long long t0 = clock64();
            while (!mbar_try_wait(drain, 0) && clock64() - t0 < WAIT_LIMIT) {
            }
            if (a.kblk) atomicAdd(a.kblk, nblk);
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int ew = warp - 2;
        const int qd = warp & 3;
        const int half = ew >> 2;
        const int row = qd * 32 + lane;
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
            TileMask km;
            tile_ranges(a, mt, nt0, nt1, km);
            const int64_t rowg = (int64_t)mt * BM + row;
            const RowConst rc = load_row_const(a.aux, rowg, a.n);
            constexpr int NR = GRAD ? 3 : 1;   // sums per filter: N (and A, D for the gradient)
            float acc[NR][4 * Q4];
#pragma unroll
            for (int r3 = 0; r3 < NR; ++r3)
#pragma unroll
                for (int q = 0; q < 4 * Q4; ++q) acc[r3][q] = 0.f;
            for (int nt = first_tile(nt0, part, a.parts); nt < nt1; nt += a.parts) {
                int got = 1;
                if (lane == 0) got = mbar_wait(accf0 + 8 * as, aphase, abort_flag, a.err) ? 1 : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) { ok = false; break; }
                tc_fence_after();
                const uint32_t tb = tmem_base + ((uint32_t)(qd * 32) << 16) + (uint32_t)(as * BN + half * 128);
                const int nb = nt * BN + half * 128;
                Slide sl[3];
#pragma unroll 1
                for (int c = 0; c < 4; ++c) {
                    uint32_t r[32];
                    tmem_ld32(tb + c * 32, r);
                    if (c == 3) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(acce0 + 8 * as);
                    }
                    if (rc.valid) {
                        if constexpr (GRAD) {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                epi_node_grad<Q4>(acc, sl, __uint_as_float(r[j]), nb + c * 32 + j, rc, a.cc, a.tab,
                                                  a.m_last);
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; j += 2)
                                epi_node2<Q4>(acc[0], sl[0], __uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                              nb + c * 32 + j, rc, a.cc, a.tab, a.m_last);
                        }
                    }
                }
                if (rc.valid) {
                    if constexpr (GRAD)
                        epi_close_grad<Q4>(acc, sl, nb + 128, rc, a.tab, a.m_last);
                    else
                        epi_close<Q4>(acc[0], sl[0], nb + 128, rc, a.tab, a.m_last);
                }
                if (++as == 2) { as = 0; aphase ^= 1u; }
            }
            if (!ok) break;
            // Combine the two column halves of each row (bounded barrier).
            float *cr = comb + row * (3 * QMAX);
            if (half == 1)
#pragma unroll
                for (int r3 = 0; r3 < NR; ++r3)
#pragma unroll
                    for (int q = 0; q < 4 * Q4; ++q) cr[r3 * 4 * Q4 + q] = acc[r3][q];
            __syncwarp();
            if (lane == 0) mbar_arrive(ebar);
            int got = 1;
            if (lane == 0) got = mbar_wait(ebar, ephase, abort_flag, a.err) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            ephase ^= 1u;
            if (!got) break;
            if (half == 0 && rowg < a.n) {
                float4 *dst = reinterpret_cast<float4 *>(a.partial + ((int64_t)part * a.n + rowg) * (NR * 4 * Q4));
#pragma unroll
                for (int r3 = 0; r3 < NR; ++r3)
#pragma unroll
                    for (int qq = 0; qq < Q4; ++qq) {
                        const float *cq = cr + r3 * 4 * Q4 + 4 * qq;
                        dst[r3 * Q4 + qq] = make_float4(acc[r3][4 * qq + 0] + cq[0], acc[r3][4 * qq + 1] + cq[1],
                                                        acc[r3][4 * qq + 2] + cq[2], acc[r3][4 * qq + 3] + cq[3]);
                    }
            }
            // Second bounded barrier: half 0 has read comb before half 1 rewrites it.
            __syncwarp();
            if (lane == 0) mbar_arrive(ebar);
            got = 1;
            if (lane == 0) got = mbar_wait(ebar, ephase, abort_flag, a.err) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            ephase ^= 1u;
            if (!got) break;
        }
    }

    __syncwarp();   // lanes 1..31 of the producer / MMA warps wait for their lane 0
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
    }
}

template <int Q4, bool GRAD>
cudaError_t launch_q4(const CUtensorMap &ah, const CUtensorMap &al, const CUtensorMap &bh, const CUtensorMap &bl,
                      const TArgs &a, int grid, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(phot_tc_kernel<Q4, GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    phot_tc_kernel<Q4, GRAD><<<grid, THREADS, SMEM_BYTES, s>>>(ah, al, bh, bl, a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_phot_tc(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, int *parts,
                           cudaStream_t s, bool grad) {
    *parts = TC_PARTS;
    if (n <= 0) return cudaSuccess;
    if (fs.Q > QMAX) return cudaErrorInvalidValue;
    CUtensorMap ah, al, bh, bl;
    if (!make_tmap(&ah, w.whi, (uint64_t)c.KZ_pad, (uint64_t)n, BM) ||
        !make_tmap(&al, w.wlo, (uint64_t)c.KZ_pad, (uint64_t)n, BM) ||
        !make_tmap(&bh, c.d_Lt_hi, (uint64_t)c.KZ_pad, (uint64_t)c.N_pad, BN) ||
        !make_tmap(&bl, c.d_Lt_lo, (uint64_t)c.KZ_pad, (uint64_t)c.N_pad, BN))
        return cudaErrorInvalidValue;
    TArgs a{};
    a.aux = w.aux;
    a.trange = w.trange;
    a.kmask = c.kmask_words <= 4 ? w.kmask : nullptr;   // larger grids contract every K block
    a.kmw = c.kmask_words;
    a.urange = w.urange;
    a.sec_blocks = c.SEC / BK;
    a.n_sec = c.n_u;
    a.tab = reinterpret_cast<const float4 *>(fs.d_tab);
    a.cc = make_col_const(c);
    a.m_last = fs.m_rows - 1;
    a.n_mtiles = (int)((n + BM - 1) / BM);
    a.n_ntiles = c.N_pad / BN;
    a.kblocks = c.KZ_pad / BK;
    a.parts = TC_PARTS;
    a.n_units = a.n_mtiles * TC_PARTS;
    a.band_skip = c.opts.band_skip ? 1 : 0;
    a.m_nz_lo = fs.m_nz_lo;
    a.m_nz_hi = fs.m_nz_hi;
    a.n = n;
    a.sched = w.sched;
    a.partial = w.partial;
    a.kblk = w.stats;
    a.err = c.d_err;
    int grid = a.n_units < c.num_sms ? a.n_units : c.num_sms;
    cudaError_t e = cudaMemsetAsync(w.sched, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (grad) {
        switch (fs.Q4) {
        case 1: return launch_q4<1, true>(ah, al, bh, bl, a, grid, s);
        case 2: return launch_q4<2, true>(ah, al, bh, bl, a, grid, s);
        case 3: return launch_q4<3, true>(ah, al, bh, bl, a, grid, s);
        default: return launch_q4<4, true>(ah, al, bh, bl, a, grid, s);
        }
    }
    switch (fs.Q4) {
    case 1: return launch_q4<1, false>(ah, al, bh, bl, a, grid, s);
    case 2: return launch_q4<2, false>(ah, al, bh, bl, a, grid, s);
    case 3: return launch_q4<3, false>(ah, al, bh, bl, a, grid, s);
    default: return launch_q4<4, false>(ah, al, bh, bl, a, grid, s);
    }
}

}  // namespace dsps
