// dsps_internal.cuh -- context layout and device helpers shared by the CUDA
// translation units of libdsps (sm_103a only).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/dsps.h"

namespace dsps {

// Tracing: an NVTX range named after the ABI function around each call (the
// header-only NVTX 3; it costs a branch unless a profiler or an NVTX tool is
// attached, which then sees every library call on the host timeline).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define DSPS_TRACE(name) ::dsps::NvtxRange dsps_trace_range_(name)

constexpr int NPAR = DSPS_NPAR;
constexpr int NGRAD = DSPS_NGRAD;
constexpr int NPAR_MAX = DSPS_NPAR_NEB;   // parameter rows with a nebular axis
constexpr int MAX_NU = DSPS_MAX_NU;
constexpr int K_ALIGN = 64;      // K (= n_age * n_z) padding: multiple of the 32-wide TMA box
constexpr int N_ALIGN = 256;     // wavelength padding: multiple of the 256-wide MMA tile
constexpr int MAX_NT = 1024;     // SFR time nodes
constexpr int MAX_NAGE = 512;
constexpr int AUX_STRIDE = 8;    // floats of per-galaxy epilogue constants
constexpr int ZSORT_BUCKETS = 4096;  // sort buckets (multiple of 1024) = ZSORT_ZBINS x ZSORT_MUBINS
constexpr int ZSORT_ZBINS = 32;      // coarse redshift-shift bins of the sort key
constexpr int ZSORT_MUBINS = ZSORT_BUCKETS / ZSORT_ZBINS;  // mean-metallicity bins inside each
constexpr int TC_PARTS = 4;      // work units per 128-galaxy tile in the tensor-core kernel
constexpr int QSTRIDE_MAX = 16;  // floats per row of the partial filter sums

// Device error word bits.
constexpr unsigned DERR_PARAM = 1u;    // out-of-range galaxy parameters
constexpr unsigned DERR_TIMEOUT = 2u;  // a kernel gave up on a bounded wait

constexpr double AB0 = 1.13492e-13;     // Sec. 2.2, Eq. (restmag)
constexpr double LAM_V = 5500.0;        // Sec. 3.4, Eq. (salim)
constexpr double SIG_Q = 0.3;           // quench transition width [Gyr]

// Order of the K = n_age * n_z * n_u axis (n_u = 1 without a nebular axis).
// The SSP block, dsps_weights and the FP32 paths use the age-major
// k = (i * n_z + j) * n_u + u.  The tensor-core operands (split weights,
// d_Lt_*) and the adjoint's differenced block use the metallicity-major
// kz = u * SEC + j * A_pad + i: A_pad = n_age rounded up to 4 (every
// metallicity row starts on a 16-byte boundary; ages n_age .. A_pad-1 are zero
// columns), one section of SEC = n_z * A_pad rounded up to 32 per log U value,
// rows of KZ_pad = n_u * SEC rounded up to K_ALIGN.  The triweight kernels have
// compact support, so a galaxy's non-zero weights fill one contiguous run of
// each section, for a contiguous range of sections; a tile of galaxies with
// similar metallicity needs only the K blocks of that run.
struct KzLayout {
    int a_pad, sec, n_age, n_z, n_u;
};
__host__ __device__ inline int kz_to_k(int kz, const KzLayout &l) {   // -1: padding
    const int u = kz / l.sec, r = kz - u * l.sec;
    const int j = r / l.a_pad, i = r - j * l.a_pad;
    return (u < l.n_u && j < l.n_z && i < l.n_age) ? (i * l.n_z + j) * l.n_u + u : -1;
}
__host__ __device__ inline int k_to_kz(int k, const KzLayout &l) {
    const int u = k % l.n_u, ij = k / l.n_u;
    const int i = ij / l.n_z, j = ij - i * l.n_z;
    return u * l.sec + j * l.a_pad + i;
}

// Per 128-row tile of sorted galaxies, reduced with atomics by the weights
// kernel over the tile's valid rows:
//   Workspace::trange  {smallest, largest} floor(s) (s = aux[.+2], the
//                      redshift shift); an empty tile keeps {INT_MAX, INT_MIN}
//   Workspace::kmask   Ctx::kmask_words words: bit b set if some row's split
//                      weights are non-zero in kz block [32 b, 32 b + 32) of
//                      some section (blocks counted inside a section)
//   Workspace::urange  {lowest, highest} section (log U bin) where some row
//                      has non-zero weight; an empty tile keeps {n_u, -1}
constexpr int TRANGE_EMPTY_LO = 0x7fffffff;
constexpr int TRANGE_EMPTY_HI = (int)0x80000000;
constexpr int KBLOCK = 32;   // kz block of the tensor-core contraction (one TMA box)

// Per-galaxy epilogue constants (aux[g*AUX_STRIDE + .]):
//   0 alpha = -0.4 log2(10) Av      (F = 2^(alpha u))
//   1 beta  = delta - 0.7, or delta with the starburst curve (u = [k0/4.05] 2^(beta log2(lam/5500)))
//   2 s     = ln(1+z) / dlnlam      (observer-frame shift in grid steps)
//   3 valid (1 or 0)
//   4 Av, 5 delta  (gradient path)
//   6 e  = (0.85 - 1.9 delta) / 4.05, 7 de/ddelta = -1.9 / 4.05  (UV bump; 0 without)
// magoff[g] = -2.5 logM + Dmod(z) - 2.5 log10(1+z)

// Entries 0, 1, 4-7 of aux from the curve's Av and delta (Sec. 3.4): the one
// definition the weights kernel and the age-dependent dust passes share.
__device__ __forceinline__ void store_dust_aux(float *ax, float Av, float dl, int dust_law, int bump) {
    ax[0] = -0.4f * 3.32192809488736235f * Av;
    ax[1] = dust_law == DSPS_DUST_SALIM ? dl : dl - 0.7f;
    ax[4] = Av;
    ax[5] = dl;
    ax[6] = bump ? (0.85f - 1.9f * dl) * (1.f / 4.05f) : 0.f;
    ax[7] = bump ? -1.9f / 4.05f : 0.f;
}

// Sec. 3.4.1: a dust value of an age group, (1 - T) young + T old.
__device__ __forceinline__ float group_dust_value(float T, float young, float old) {
    return fmaf(T, old - young, young);
}

struct FilterSet {
    int Q = 0, Q4 = 0;         // filters; float4 groups per table row
    int m_rows = 0;            // table rows; row m_rows-1 is all zero
    int m_nz_lo = 0, m_nz_hi = -1;  // first / last table row where some filter is non-zero
    float *d_tab = nullptr;    // [m_rows][4*Q4] T_q(lam0 exp(m dlnlam))
    float *d_offq = nullptr;   // [Q] 2.5 log10(AB0 D_q)
    int rest = 0;              // 1: rest-frame absolute magnitudes (Eq. restmag: no shift, no distance terms)
    // band coverage (coverage.cu): per filter q, points cov_off[q] .. cov_off[q+1] - 1
    // of the filter's own table as (ln lam, A, B), A / B the response int T dlam / lam
    // left / right of the point over D_q (FP64), and the point where A reaches 1/2
    double *d_cov = nullptr;
    int cov_off[DSPS_MAX_FILTERS + 1] = {};
    int cov_mid[DSPS_MAX_FILTERS] = {};
};

// A registered emission line (spectrum.cu): the window of grid columns
// [c0, c0 + n_pts) holding its continuum and line points, and per point j
// two float4: {t_j, x_j, x_j^2, 1 for a continuum point} and {psi_j, 0} with
// t_j the trapezoid weight of a line point (0 for continuum points), x_j =
// (lam_j - lam_line) / (half_width + cont_width), and psi_j = M^-1 (1, x_j,
// x_j^2) the fit operator of a continuum point (0 for line points).
struct LineSet {
    int c0 = 0, n_pts = 0;
    int cs = 0, ce = 0;        // [c0, c0 + n_pts) widened to multiples of 16 columns
    float4 *d_tab = nullptr;   // [n_pts][2]
};

// Age-dependent dust (agedep.cu): the age bins split into groups of one
// attenuation curve each -- the young bins with T = 0, every bin of the
// transition, the old bins with T = 1 -- contracted one group at a time.
struct DustGroup {
    int i0, i1;     // age bins [i0, i1)
    float T;        // weight of the old-star values
};

struct Serve;  // request loop (serve.cu)

// Colour-cut histogram of the magnitudes (dsps.h: dsps_hist_spec), as used by
// the kernels; counts == nullptr disables it.
struct HistArgs {
    int band_a = 0, band_b = 0, band_r = 0, n_bins = 0;
    float cut = 0.f, lo = 0.f, hi = 0.f, scale = 0.f;   // scale = n_bins / (hi - lo) in FP32
    unsigned long long *counts = nullptr;
};

// Per-galaxy scalars of the cosmology (weights.cu: galaxy_prep_kernel).
struct GalPrep {
    int m_obs;       // interval of the SFR time grid holding t_obs(z); -1 if z is out of range
    float f_obs;     // position of t_obs inside that interval, [0, 1)
    float magoff;    // -2.5 logM + Dmod(z) - 2.5 log10(1+z) (NaN if z is out of range)
    float pad;
};

// Per-launch work space of the photometry path (rows = galaxies of one chunk
// or batch).  The context owns one (Ctx::ws); the request loop carves one per
// in-flight batch out of its device arena; the allocation-free entry point
// points one at its static array.
struct Workspace {
    int64_t cap = 0;                            // rows
    float *w32 = nullptr;                       // [cap][K_pad] FP32 weights / [cap][KZ_pad] adjoint output
    __nv_bfloat16 *whi = nullptr, *wlo = nullptr;  // [cap][KZ_pad] split weights (metallicity-major)
    float *aux = nullptr;                       // [cap][AUX_STRIDE]
    float *magoff = nullptr;                    // [cap]
    GalPrep *prep = nullptr;                    // [cap] (chunk order)
    int *perm = nullptr, *gidx = nullptr;       // [cap]
    int *hist = nullptr;                        // [ZSORT_BUCKETS]
    float *partial = nullptr;                   // [TC_PARTS][cap][3 * QSTRIDE_MAX]
    int2 *trange = nullptr;                     // [cap/128 + 1] per sorted 128-row tile (see above)
    int2 *urange = nullptr;                     // [cap/128 + 1] per tile (see above)
    unsigned *kmask = nullptr;                  // [cap/128 + 1][kmask_words]
    int *sched = nullptr;                       // [1] work-unit counter of the tensor-core kernels
    float *cq = nullptr;                        // [cap][QSTRIDE_MAX]
    float *gacc = nullptr;                      // [cap][5 * QSTRIDE_MAX] sums over dust groups (age-dependent dust)
    float *what2 = nullptr;                     // [cap][KZ_pad] adjoint rows merged over dust groups (likewise)
    void *shat = nullptr;                       // [cap][N_pad] x 4 bytes (adjoint only)
    float *ewacc = nullptr;                     // [cap][N_pad] summed attenuated window of the line widths
                                                // (age-dependent dust; made on first use)
    unsigned long long *stats = nullptr;        // [2] executed-work counters (profiling), or nullptr
    int rest = 0;                               // this call's filter set is rest-frame (FilterSet::rest)
    // age-dependent dust, split-bf16: the chunk's age fractions [cap][n_age]
    // (NaN for an invalid galaxy), written by the first multi-age group's
    // weights (fcache_mode 1) and read by the one-age groups' (fcache_mode 2)
    float *fcache = nullptr;
    int fcache_mode = 0;
};

struct Ctx {
    int device = 0;
    dsps_opts opts{};
    int n_age = 0, n_z = 0, n_lam = 0, K = 0, K_pad = 0, N_pad = 0, n_t = 0;
    int A_pad = 0, KZ_pad = 0;              // metallicity-major K: n_age padded to 4, row length
    int n_u = 1, SEC = 0, u_ref = 0;        // nebular axis: log U values, section length, reference section
    // Parameter rows 0..11, [u_mean, u_sigma], [Av_old, delta_old], [SFR table];
    // gradient rows 0..10 and the same optional blocks in the same order.
    int npar = NPAR, ngrad = NGRAD;         // parameter and gradient rows
    int row_dust_old = -1;                  // age-dependent dust: parameter row of Av_old (delta_old next)
    int grow_dust_old = -1;                 //   and its gradient row
    int row_sfr = -1, grow_sfr = -1;        // tabulated SFH: rows of the node SFRs and of their gradient
    std::vector<DustGroup> dust_groups;     // age-dependent dust: the groups of age bins
    // Age-dependent dust, fused split-bf16 forward (agedep_tc.cu): K in age
    // blocks, column ka = i * KBLOCK + j (age i, metallicity j < n_z <= 32,
    // the rest zero), rows of KA_pad = n_age * KBLOCK rounded up to K_ALIGN;
    // built when the grid has no nebular axis and n_z <= KBLOCK (else 0).
    int KA_pad = 0;
    __nv_bfloat16 *d_Lab_hi = nullptr;      // [N_pad][KA_pad] row-scaled SSP hi, age-block order
    __nv_bfloat16 *d_Lab_lo = nullptr;      // [N_pad][KA_pad] lo
    __nv_bfloat16 *d_Ldab_hi = nullptr;     // [KA_pad][N_pad] the differenced split rows, age-block order
    __nv_bfloat16 *d_Ldab_lo = nullptr;
    float *d_wmul_ab = nullptr;             // [KA_pad] 2^E_k at column ka (0 at padding)
    int kmask_words = 0;                    // ceil(SEC / KBLOCK / 32)
    double t0 = 0, t1 = 0;
    double lnlam0 = 0, dlnlam = 0;
    int num_sms = 0;
    // Sort key of the tensor-core path: the MDF mean at the middle log age,
    // sort_mua p5 + sort_mub p7, binned from sort_mu_lo at sort_mu_scale bins per dex.
    float sort_mu_lo = 0.f, sort_mu_scale = 0.f, sort_mua = 1.f, sort_mub = 0.f;
    float sort_u_lo = 0.f, sort_u_scale = 0.f;   // nebular axis: 8 bins of the mean log U

    // Resident SSP copies.
    float *d_L32 = nullptr;                 // [K_pad][N_pad] fp32 (SIMT path)
    __nv_bfloat16 *d_Lt_hi = nullptr;       // [N_pad][KZ_pad] row-scaled hi, metallicity-major K (tensor path)
    __nv_bfloat16 *d_Lt_lo = nullptr;       // [N_pad][KZ_pad] row-scaled lo
    float *d_wmul = nullptr;                // [KZ_pad] 2^E_k of the scaled rows, metallicity-major K

    // Grids and tables.
    float *d_logage = nullptr;              // [n_age] log10(age/yr)
    float *d_mua = nullptr, *d_mub = nullptr;   // [n_age] MDF mean of bin i: mua_i p5 + mub_i p7
    float *d_bump = nullptr;                // [N_pad] unit Drude profile at lam_n (Eq. uvbump), 0 past n_lam
    float *d_k0 = nullptr;                  // [N_pad] k0(lam_n) / 4.05 (Eq. kzero), 0 past n_lam
    double *d_edges = nullptr;              // [n_age+1] age-bin edges [Gyr]
    float *d_einh = nullptr;                // [n_age+1] edge / time step
    float *d_bwidth = nullptr;              // [n_age] bin widths [Gyr]
    float *d_zedge = nullptr;               // [n_z+1] lgZ bin edges (+-1e30 outer)
    float *d_uedge = nullptr;               // [n_u+1] log U bin edges (+-1e30 outer)
    double *d_tlut = nullptr;               // [n_lut] t_obs(z) [Gyr]
    float *d_glut = nullptr;                // [n_lut] Dmod(z) - 5 log10 z
    int n_lut = 0;
    double dz_lut = 0;

    // Work space of the direct calls (one chunk of galaxies; Shat made lazily).
    int64_t chunk = 0;                      // galaxies per chunk (multiple of 128)
    unsigned char *d_ws_block = nullptr;    // device block holding ws (without Shat)
    Workspace ws;
    unsigned long long *d_stats = nullptr;  // [3] tensor-core blocks, FP32 tile steps, 128-wide tensor-core blocks (profiling)
    float *d_Ld32 = nullptr;                // [KZ_pad][N_pad] differenced block (FP32 adjoint; prep.cu)
    float *d_wmul_d = nullptr;              // [KZ_pad] 2^E'_kz of the differenced rows
    __nv_bfloat16 *d_L_hi = nullptr;        // [KZ_pad][N_pad] differenced block, row-scaled hi (tensor adjoint)
    __nv_bfloat16 *d_L_lo = nullptr;        // [KZ_pad][N_pad] row-scaled lo
    unsigned *d_err = nullptr;              // sticky error word
    unsigned char *d_hio = nullptr;         // dsps_photometry_host: device inputs + outputs of one chunk
    size_t hio_bytes = 0;

    KzLayout kzl() const { return KzLayout{A_pad, SEC, n_age, n_z, n_u}; }

    std::vector<FilterSet> sets;
    std::vector<LineSet> lines;
    std::vector<double> h_lam;              // [n_lam] the caller's rest wavelengths [A]
    std::mutex mu;
    Serve *serve = nullptr;

    // Kernel timing (dsps_profile_*): event pairs recorded around launches.
    struct ProfRec {
        int kind;
        cudaEvent_t a, b;
    };
    bool prof = false;
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> ev_pool;
};

// Records an event pair around the launches made during its lifetime when the
// context's profiling is on (caller holds ctx.mu).
struct ProfScope {
    Ctx &c;
    int kind;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEvent_t take() {
        cudaEvent_t e = nullptr;
        if (!c.ev_pool.empty()) {
            e = c.ev_pool.back();
            c.ev_pool.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
        }
        return e;
    }
    ProfScope(Ctx &c_, int kind_, cudaStream_t s_, bool on = true) : c(c_), kind(kind_), s(s_) {
        if (!on || !c.prof) return;
        a = take();
        b = take();
        if (a && b) cudaEventRecord(a, s);
    }
    ~ProfScope() {
        if (a && b) {
            cudaEventRecord(b, s);
            c.prof_recs.push_back({kind, a, b});
        }
    }
};

// ----------------------------------------------------------------------------
// Kernel launch wrappers (defined in the .cu files)
// ----------------------------------------------------------------------------
// W_OMEGA_BF16X2_AGE1: the split weights of one age bin (an age-dependent dust
// group of the transition), written only in the kz blocks holding that age.
// W_OMEGA_BF16X2_AB: the split weights of all ages in the age-block order of
// the fused age-dependent dust forward (Ctx::KA_pad), the tiles' K-block mask
// holding one bit per age with a non-zero weight, and aux holding the young and
// old dust values (agedep_tc.cu: Av_young, delta_young, s, valid, Av_old,
// delta_old at entries 0, 1, 2, 3, 4, 5).
enum WeightsMode { W_MSUN = 0, W_OMEGA_F32 = 1, W_OMEGA_BF16X2 = 2, W_OMEGA_BF16X2_AGE1 = 3, W_OMEGA_BF16X2_AB = 4 };

// Bytes of a work space for `rows` galaxies (what = 1: forward only, 2: with adjoint).
size_t workspace_bytes(const Ctx &c, int64_t rows, bool adjoint);
// Carves a work space for `rows` galaxies out of [base, base + workspace_bytes).
Workspace workspace_carve(const Ctx &c, void *base, int64_t rows, bool adjoint);

// group: with age-dependent dust, the weights of the group's ages only and its
// dust constants in aux (nullptr: all ages, one curve).
// aux_yo: aux holds the young and old dust values instead of one curve's
// constants (a one-launch age-dependent dust contraction).
cudaError_t launch_weights(const Ctx &c, const Workspace &w, int mode, const float *params, int64_t G_stride,
                           int64_t g_begin, int64_t n, float *w_msun, cudaStream_t s, bool sorted = false,
                           const DustGroup *group = nullptr, bool aux_yo = false);

// Counting sort of the chunk's galaxies into w.perm by (coarse redshift shift,
// mean metallicity); also resets w.trange and w.kmask.
cudaError_t launch_zsort(const Ctx &c, const Workspace &w, const float *params, int64_t G_stride, int64_t g_begin,
                         int64_t n, cudaStream_t s);
// Sums the tensor-core kernel's per-part filter sums and writes magnitudes
// (mags may be nullptr), or bins them into hist->counts.
cudaError_t launch_combine(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, int parts, float *mags,
                           cudaStream_t s, const HistArgs *hist = nullptr);
// Colour-cut histogram of device magnitudes [n][Q] (histogram.cu).
cudaError_t launch_histogram(const float *mags, int64_t n, int Q, const HistArgs &h, cudaStream_t s);
int make_hist_args(const dsps_hist_spec *spec, int n_filt, unsigned long long *counts, HistArgs *out);

// Magnitudes (mags != nullptr, forward) are written directly with one part.
// Otherwise the sums N (grad: N, A, D; see epilogue.cuh) per filter go to
// w.partial in *parts parts (TC_PARTS interleaved wavelength-tile subsets with
// sorted rows, one part without), for launch_combine / launch_combine_grad /
// the dust groups' sums.
// sorted: rows in the order of launch_zsort (magnitudes written through
// w.gidx), each 128-row tile contracting only the wavelength tiles of its band.
// group: weights of one dust group's ages only (age-dependent dust), so the
// contraction runs over the group's k range alone.
cudaError_t launch_phot_simt(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, float *mags,
                             cudaStream_t s, bool grad = false, bool sorted = false,
                             const DustGroup *group = nullptr, int *parts = nullptr);

// The k range [k_lo, k_hi) of the FP32 (age-major, k = (i n_z + j) n_u + u)
// weights of a dust group's ages, widened to multiples of bk (all of
// [0, K_pad) without a group).
inline void group_k_range(const Ctx &c, const DustGroup *gr, int bk, int &k_lo, int &k_hi) {
    k_lo = 0;
    k_hi = c.K_pad;
    if (!gr) return;
    const int per_age = c.n_z * c.n_u;
    k_lo = gr->i0 * per_age / bk * bk;
    const int hi = (gr->i1 * per_age + bk - 1) / bk * bk;
    k_hi = hi < c.K_pad ? hi : c.K_pad;
}

// Most dust groups a one-launch age-dependent contraction takes.
constexpr int AGEDEP_MAX_GROUPS = 128;

// Age-dependent dust, split-bf16: the merged adjoint rows of the weights (w.what2,
// in the tensor adjoint's row scale) for every dust group in one launch, from
// the dust-free adjoint spectrum in w.shat (agedep_vjp_tc.cu).
bool agedep_vjp_tc_ok(const Ctx &c);
cudaError_t launch_vjp_groups_tc(const Ctx &c, const Workspace &w, const FilterSet &fs, const float *params,
                                 int64_t G_stride, int64_t g_begin, int64_t n, cudaStream_t s);

// Age-dependent dust, FP32 form, every group in one launch (agedep_simt.cu):
// per-part filter sums of the sorted rows from the weights of all ages
// (launch_weights with aux_yo); *parts gets the number of parts.
cudaError_t launch_phot_simt_groups(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, int *parts,
                                    cudaStream_t s);

// Writes per-part filter sums to ctx.d_partial (sorted rows); returns the
// number of parts through *parts.
cudaError_t launch_phot_tc(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, int *parts,
                           cudaStream_t s, bool grad = false);

cudaError_t prepare_ssp_device(Ctx &c, const float *h_lssp);

// Age-dependent dust, fused split-bf16 forward (agedep_tc.cu): whether the
// context has the age-block operands, and the contraction of every dust group
// of each tile in one launch (each group's spectrum attenuated by its curve and
// summed in TMEM, one filter integral), writing per-part filter sums for
// launch_combine.  Needs the chunk sorted (launch_zsort) and its weights in the
// W_OMEGA_BF16X2_AB form.
bool agedep_fused_ok(const Ctx &c);
// With G (the dust-free adjoint spectrum of the sorted rows, launch_shat
// without dust): the gradient pass, writing per part and row the four dust
// sums (Av and delta, young and old; the -0.4 ln10 factor left out) to
// w.partial as [parts][n][4].
cudaError_t launch_phot_tc_groups(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, int *parts,
                                  cudaStream_t s, const float *G = nullptr);

// Adjoint (vjp.cu, vjp_tc.cu, weights.cu).
cudaError_t launch_combine_grad(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, int parts,
                                bool sorted, const float *mag_bar, float *mags, float *param_bar, int64_t G_stride,
                                int64_t g_begin, cudaStream_t s);
// dust = false: FP32 Shat without the dust factor (age-dependent dust's
// one-age groups apply their own curves).
cudaError_t launch_shat(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, bool bf16, bool band,
                        cudaStream_t s, bool dust = true);
// col0/col1: the Shat columns that take part (multiples of 16; 0, N_pad for all);
// fs: with sorted rows and band skipping, each 128-row tile's band only.
cudaError_t launch_vjp_simt(const Ctx &c, const Workspace &w, int64_t n, cudaStream_t s, int col0 = 0,
                            int col1 = -1, const FilterSet *fs = nullptr);
cudaError_t launch_vjp_tc(const Ctx &c, const Workspace &w, const FilterSet &fs, int64_t n, cudaStream_t s);
cudaError_t launch_weights_vjp(const Ctx &c, const Workspace &w, const float *params, int64_t G_stride,
                               int64_t g_begin, int64_t n, bool sorted, bool scaled, float *param_bar,
                               cudaStream_t s);

// Whole photometry / adjoint of a population on one stream with one work space
// (dispatch.cu); mags/param_bar are the caller's device pointers.
int run_photometry_ws(Ctx *c, const Workspace &w, int64_t n_gal, const float *params, const FilterSet &fs,
                      int32_t precision, float *mags, cudaStream_t s, bool profile, const HistArgs *hist = nullptr);
// dsps_photometry_host: host params and mags, synchronous on s (dispatch.cu).
int run_photometry_host(Ctx *c, int64_t n_gal, const float *h_params, int32_t set_id, int32_t precision,
                        float *h_mags, cudaStream_t s);
// Allocates ctx.ws.shat (and, with ewacc, ctx.ws.ewacc) if it is not there
// yet (dispatch.cu).
int ensure_shat(Ctx *c, bool ewacc = false);

// Age-dependent dust (agedep.cu).  A one-age group whose n_z adjoint columns
// are formed directly (n_z <= 32) instead of by an adjoint contraction:
bool age1_direct(const Ctx &c, const DustGroup &gr);
// those columns, in w.what2, for every such group (or only *only): the FP32
// dot products of G (w.shat, the dust-free Shat, when G is null) times the
// group's attenuation with the group's rows of the differenced block, over
// each row tile's band of fs (sorted rows) or over columns [col0, col1)
// (multiples of 16; rows in chunk order when G is given); divided by wmul_d
// when scaled.
cudaError_t launch_age1_adjoint(const Ctx &c, const Workspace &w, const FilterSet *fs, const float *params,
                                int64_t G_stride, int64_t g_begin, int64_t n, bool scaled, cudaStream_t s,
                                const float *G = nullptr, int col0 = 0, int col1 = 0,
                                const DustGroup *only = nullptr);
// Keeps, in w.what2, the adjoint rows of w.w32 at the columns of the group's
// ages (first: also zeroes the padding columns).
cudaError_t launch_merge_rows(const Ctx &c, const Workspace &w, int64_t n, const DustGroup &gr, bool first,
                              cudaStream_t s);
// Spectra and line widths (spectrum.cu); w.shat must be allocated.
int run_spectra_ws(Ctx *c, const Workspace &w, int64_t n_gal, const float *params, int n0, int n1, float *out,
                   cudaStream_t s);
int run_line_ew_ws(Ctx *c, const Workspace &w, int64_t n_gal, const float *params, const LineSet &ls,
                   const float *ew_bar, float *ew, float *param_bar, cudaStream_t s);
// Age-dependent dust (agedep.cu): the same calls, one dust group at a time.
int run_photometry_agedep_ws(Ctx *c, const Workspace &w, int64_t n_gal, const float *params, const FilterSet &fs,
                             int32_t precision, float *mags, cudaStream_t s, bool profile, const HistArgs *hist);
int run_photometry_vjp_agedep_ws(Ctx *c, const Workspace &w, int64_t n_gal, const float *params,
                                 const FilterSet &fs, int32_t precision, const float *mag_bar, float *mags,
                                 float *param_bar, cudaStream_t s, bool profile);
int run_photometry_vjp_ws(Ctx *c, const Workspace &w, int64_t n_gal, const float *params, const FilterSet &fs,
                          int32_t precision, const float *mag_bar, float *mags, float *param_bar, cudaStream_t s,
                          bool profile);

// ----------------------------------------------------------------------------
// Device helpers
// ----------------------------------------------------------------------------
#ifdef __CUDACC__

// Appendix B, Eq. (terf) for z <= 0, written in x = z + 3: the same polynomial
// equals (35/69984) x^4 (54 - 21.6 x + 3 x^2 - x^3/7), which keeps its relative
// precision in FP32 down to the far lower tail (the printed monomial form
// cancels there).  Zero below z = -3.
__device__ __forceinline__ float terf_lower_f(float z) {
    const float x = z + 3.f;
    if (x <= 0.f) return 0.f;
    const float x2 = x * x;
    const float poly = fmaf(x, fmaf(x, fmaf(x, -1.f / 7.f, 3.f), -21.6f), 54.f);
    return (35.f / 69984.f) * x2 * x2 * poly;
}

// Triweight CDF, saturated to 0 / 1 outside [-3, 3]; upper half by symmetry.
__device__ __forceinline__ float terf_f(float z) {
    return z <= 0.f ? terf_lower_f(z) : 1.f - terf_lower_f(-z);
}

// Appendix B, Eq. (triweight): density in the standardised variable.
__device__ __forceinline__ float triweight_f(float z) {
    if (z <= -3.f || z >= 3.f) return 0.f;
    float t = fmaf(-z / 3.f, z / 3.f, 1.f);
    return (35.f / 96.f) * t * t * t;
}

__device__ __forceinline__ float gauss_cdf_f(float z) { return 0.5f * erfcf(-z * 0.70710678118654752f); }
__device__ __forceinline__ float gauss_pdf_f(float z) { return 0.39894228040143268f * expf(-0.5f * z * z); }

#endif  // __CUDACC__

}  // namespace dsps
