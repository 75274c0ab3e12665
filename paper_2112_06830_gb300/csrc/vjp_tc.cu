// vjp_tc.cu -- tcgen05 form of the adjoint contraction
//   What[g, kz] = sum_n Shat[g, n] Ld[kz, n]      (dLoss/domega, see vjp.cu)
// with Shat and the row-scaled SSP block both split into bf16 hi + lo
// (hi*hi + hi*lo + lo*hi, FP32 accumulate in TMEM), written as FP32.
//
// Work unit = (128-galaxy tile, 256-wide block of SSP indices k), claimed from
// a global counter (tc::UnitRing); the reduction runs only over the wavelength
// blocks where the tile's Shat can be non-zero (the redshifted filter band,
// epilogue.cuh: vjp_band).  With the nebular axis, a unit whose columns meet
// neither the tile's log U sections nor the reference section is skipped by
// every role (no galaxy of the tile reads those columns).  Warp roles
// as in phot_tc.cu: TMA producer, single-thread MMA issuer with a double
// TMEM accumulator, eight epilogue warps that read rows with tcgen05.ld and
// write them as 32 x 32 blocks through shared memory and TMA stores (a row per
// thread would scatter every warp store over 32 rows).  Every mbarrier wait is
// bounded.
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
constexpr size_t BAR_BYTES = 1024;
constexpr size_t STAGE_OUT_BYTES = 32 * 32 * 4;   // per epilogue warp: one 32 x 32 FP32 block
constexpr size_t SMEM_BYTES = 1024 + (size_t)STAGES * STAGE_BYTES + BAR_BYTES + NUM_EPI_WARPS * STAGE_OUT_BYTES;

struct VArgs {
    const int2 *trange;
    const int2 *urange;   // per-tile log U section ranges (a superset of each row's), or nullptr
    int sec, u_ref;       // section length (columns), reference section
    VjpBand band;
    int n_mtiles, n_ktiles, n_units, N_pad, K_pad;   // K_pad: the context's KZ_pad (output row length)
    int64_t n;
    int *sched;       // unit counter, zero at launch
    unsigned *err;
};

// Whether unit (mt, kt) writes columns that the tile's weights adjoint reads:
// the log U sections of the tile's range, and the reference section, which
// every galaxy reads (Sec. 3.3: the P_u sum to one).
__device__ __forceinline__ bool unit_live(const VArgs &a, int mt, int kt) {
    if (!a.urange) return true;
    const int2 ur = a.urange[mt];
    const int c0 = kt * BN, c1 = c0 + BN;
    const bool in_range = ur.y >= ur.x && c0 < (ur.y + 1) * a.sec && c1 > ur.x * a.sec;
    const bool in_ref = c0 < (a.u_ref + 1) * a.sec && c1 > a.u_ref * a.sec;
    return in_range || in_ref;
}

__global__ void __launch_bounds__(THREADS, 1)
vjp_tc_kernel(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
              const __grid_constant__ CUtensorMap tmB_hi, const __grid_constant__ CUtensorMap tmB_lo,
              const __grid_constant__ CUtensorMap tmOut, const VArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + (size_t)STAGES * STAGE_BYTES);
    const uint32_t full0 = smem_u32(bars);
    const uint32_t empty0 = smem_u32(bars + STAGES);
    const uint32_t accf0 = smem_u32(bars + 2 * STAGES);
    const uint32_t acce0 = smem_u32(bars + 2 * STAGES + 2);
    const uint32_t drain = smem_u32(bars + 2 * STAGES + 4);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 5);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    UnitRing ring;
    ring.full0 = smem_u32(bars + 2 * STAGES + 8);
    ring.empty0 = smem_u32(bars + 2 * STAGES + 8 + UNIT_RING);
    ring.slot = reinterpret_cast<volatile int *>(bars + 2 * STAGES + 8 + 2 * UNIT_RING);
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
                const int mt = u / a.n_ktiles, kt = u - mt * a.n_ktiles;
                if (!unit_live(a, mt, kt)) continue;
                int kb0, kb1;
                vjp_band(a.band, a.trange, mt, a.N_pad, kb0, kb1);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u, abort_flag, a.err)) { ok = false; break; }
                    const uint32_t fb = full0 + 8 * stage;
                    const uint32_t st = sbase + stage * STAGE_BYTES;
                    mbar_expect_tx(fb, STAGE_BYTES);
                    tma_load_2d(st, &tmA_hi, fb, kb * BK, mt * BM);
                    tma_load_2d(st + A_BYTES, &tmA_lo, fb, kb * BK, mt * BM);
                    tma_load_2d(st + 2 * A_BYTES, &tmB_hi, fb, kb * BK, kt * BN);
                    tma_load_2d(st + 2 * A_BYTES + B_BYTES, &tmB_lo, fb, kb * BK, kt * BN);
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
                const int mt = u / a.n_ktiles, kt = u - mt * a.n_ktiles;
                if (!unit_live(a, mt, kt)) continue;
                int kb0, kb1;
                vjp_band(a.band, a.trange, mt, a.N_pad, kb0, kb1);
                if (!mbar_wait(acce0 + 8 * as, aphase ^ 1u, abort_flag, a.err)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(as * BN);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(full0 + 8 * stage, phase, abort_flag, a.err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t st = sbase + stage * STAGE_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint64_t ah = sdesc_sw64(st + kk * 32);
                        const uint64_t al = sdesc_sw64(st + A_BYTES + kk * 32);
                        const uint64_t bh = sdesc_sw64(st + 2 * A_BYTES + kk * 32);
                        const uint64_t bl = sdesc_sw64(st + 2 * A_BYTES + B_BYTES + kk * 32);
                        mma_bf16(d, ah, bh, (kb != kb0 || kk != 0) ? 1u : 0u);
                        mma_bf16(d, ah, bl, 1u);
                        mma_bf16(d, al, bh, 1u);
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
    } else {
        // ---------------------------------------------------------------- epilogue
        const int ew = warp - 2;
        const int qd = warp & 3;
        const int half = ew >> 2;
        // Each warp writes its 32 rows x 32 columns per step through a 4 KB
        // shared-memory block (128-byte swizzle) and one TMA store.
        unsigned char *outs = sm + (size_t)STAGES * STAGE_BYTES + BAR_BYTES + (size_t)ew * STAGE_OUT_BYTES;
        const uint32_t outs_u32 = smem_u32(outs);
        int as = 0;
        uint32_t aphase = 0;
        while (true) {
            int u = -1, have = 1;
            if (lane == 0) have = ring_next(ring, u, abort_flag, a.err) ? 1 : 0;
            have = __shfl_sync(0xffffffffu, have, 0);
            u = __shfl_sync(0xffffffffu, u, 0);
            if (!have || u < 0) break;
            const int mt = u / a.n_ktiles, kt = u - mt * a.n_ktiles;
            if (!unit_live(a, mt, kt)) continue;
            int got = 1;
            if (lane == 0) got = mbar_wait(accf0 + 8 * as, aphase, abort_flag, a.err) ? 1 : 0;
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) break;
            tc_fence_after();
            const uint32_t tb = tmem_base + ((uint32_t)(qd * 32) << 16) + (uint32_t)(as * BN + half * 128);
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                uint32_t r[32];
                tmem_ld32(tb + c * 32, r);
                if (c == 3) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(acce0 + 8 * as);
                }
                const int col0 = kt * BN + half * 128 + c * 32;
                if (col0 < a.K_pad && (int64_t)mt * BM + qd * 32 < a.n) {   // a box past the last row writes nothing
                    if (lane == 0) bulk_wait_read();   // the previous store has read the block
                    __syncwarp();
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        *reinterpret_cast<float4 *>(outs + lane * 128 + ((j ^ (lane & 7)) << 4)) =
                            make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                        __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_2d(&tmOut, outs_u32, col0, mt * BM + qd * 32);
                        bulk_commit();
                    }
                }
            }
            if (++as == 2) { as = 0; aphase ^= 1u; }
        }
        if (lane == 0) bulk_wait_all();
    }

    __syncwarp();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

cudaError_t launch_vjp_tc(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const auto *hi = reinterpret_cast<const __nv_bfloat16 *>(w.shat);
    const __nv_bfloat16 *lo = hi + (size_t)w.cap * c.N_pad;
    CUtensorMap ah, al, bh, bl, ot;
    if (!make_tmap(&ah, hi, (uint64_t)c.N_pad, (uint64_t)n, BM) ||
        !make_tmap(&al, lo, (uint64_t)c.N_pad, (uint64_t)n, BM) ||
        !make_tmap(&bh, c.d_L_hi, (uint64_t)c.N_pad, (uint64_t)c.KZ_pad, BN) ||
        !make_tmap(&bl, c.d_L_lo, (uint64_t)c.N_pad, (uint64_t)c.KZ_pad, BN) ||
        !make_tmap_f32_store(&ot, w.w32, (uint64_t)c.KZ_pad, (uint64_t)n))
        return cudaErrorInvalidValue;
    VArgs a{};
    a.trange = w.trange;
    // the rows are sorted and, with skipping on, the sort presets the tiles'
    // log U ranges before the weights run
    a.urange = c.n_u > 1 && c.opts.band_skip ? w.urange : nullptr;
    a.sec = c.SEC;
    a.u_ref = c.u_ref;
    a.band = make_vjp_band(c, fs, c.opts.band_skip != 0);
    a.n_mtiles = (int)((n + BM - 1) / BM);
    a.n_ktiles = (c.KZ_pad + BN - 1) / BN;
    a.n_units = a.n_mtiles * a.n_ktiles;
    a.N_pad = c.N_pad;
    a.K_pad = c.KZ_pad;
    a.n = n;
    a.sched = w.sched;
    a.err = c.d_err;
    const int grid = a.n_units < c.num_sms ? a.n_units : c.num_sms;
    cudaError_t e = cudaFuncSetAttribute(vjp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.sched, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    vjp_tc_kernel<<<grid, THREADS, SMEM_BYTES, s>>>(ah, al, bh, bl, ot, a);
    return cudaGetLastError();
}

}  // namespace dsps
