// prep.cu -- one-time preparation of the resident SSP block (Sec. 2.1: the SSP
// spectra are computed in advance, loaded once as a contiguous block and held
// fixed).  Builds, from the caller's FP32 L[k][n] (k = (i * n_z + j) * n_u + u,
// n_u = 1 without a nebular axis):
//   d_L32   [K_pad][N_pad] FP32, zero padded                (SIMT form)
//   d_Lt_*  [N_pad][KZ_pad] bf16 hi / lo of L[k][n] 2^-E_k   (tensor form, K-contiguous
//           rows, columns in the metallicity-major order kz = u * SEC + j * A_pad + i)
//   d_Ld32  [KZ_pad][N_pad] FP32 differenced block, rows in the same order:
//           with D_j L = L[i, j, u] - L[i, j-1, u] (L[i, 0, u] for j = 0), row
//           (u_ref, j, i) is D_j L[i, j, u_ref] and row (u != u_ref, j, i) is
//           D_j L[i, j, u] - D_j L[i, j, u_ref]             (FP32 adjoint)
//   d_L_*   [KZ_pad][N_pad] bf16 hi / lo of the differenced block scaled by
//           2^-E'_kz, with d_wmul_d = 2^E'_kz              (tensor adjoint)
// The adjoint contracts with the differenced block so that the differences of
// dLoss/domega between neighbouring metallicity bins -- all the metallicity
// gradients need (summation by parts) -- and, with a nebular axis, between each
// log U bin and the reference one -- all the log U gradients need, since the
// bin probabilities sum to 1 -- come out at full relative precision.
//   d_wmul  [KZ_pad] 2^E_k, the factor folded into the weights, so that
//           sum_k (omega_k 2^E_k)(L_kn 2^-E_k) = sum_k omega_k L_kn exactly
//           (indexed by kz, like d_Lt_*).
//   d_Lab_*  [N_pad][KA_pad] bf16 hi / lo of L[k][n] 2^-E_k in the age-block
//           order ka = i * 32 + j (age-dependent dust's fused forward), with
//           d_wmul_ab = 2^E_k at ka (only when Ctx::KA_pad > 0)
//   d_Ldab_* [KA_pad][N_pad] the rows of d_L_* in the age-block order (row ka =
//           32 i + j holds row kz = j A_pad + i; zero for j >= n_z or i >= n_age):
//           the age-dependent adjoint's operand, whose products then carry the
//           same 2^-E'_kz as the tensor adjoint's (only when KA_pad > 0, n_u = 1)
// E_k is the binary exponent of max_n L[k][n]: every scaled row peaks in
// [1, 2), far from the bf16 underflow threshold.
#include "dsps_internal.cuh"

namespace dsps {

namespace {

// wmul is written at the metallicity-major position of row k, rscale at k.
__global__ void row_exponent_kernel(const float *L, int K, int N, int K_pad, KzLayout kl, float *wmul,
                                    float *rscale) {
    const int k = blockIdx.x;
    if (k >= K_pad) return;
    float m = 0.f;
    if (k < K)
        for (int n = threadIdx.x; n < N; n += blockDim.x) m = fmaxf(m, L[(size_t)k * N + n]);
    __shared__ float red[32];
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float mm = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmaxf(mm, red[w]);
        int E = 0;
        if (mm > 0.f) E = ilogbf(mm);
        E = max(-120, min(120, E));
        if (k < K) wmul[k_to_kz(k, kl)] = ldexpf(1.f, E);
        rscale[k] = k < K ? ldexpf(1.f, -E) : 0.f;
    }
}

__global__ void build_l32_kernel(const float *L, int K, int N, int K_pad, int N_pad, float *L32) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)K_pad * N_pad;
    if (idx >= total) return;
    const int k = (int)(idx / N_pad), n = (int)(idx % N_pad);
    L32[idx] = (k < K && n < N) ? L[(size_t)k * N + n] : 0.f;
}

// Transposing split: tile of 32 (kz) x 32 (n) through shared memory; column
// kz of the output [N_pad][KZ_pad] takes SSP row k = kz_to_k(kz) (zero for
// padding columns).
__global__ void build_lt_kernel(const float *L, const float *rscale, int N, int KZ_pad, int N_pad, KzLayout kl,
                                __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
    __shared__ float t[32][33];
    const int k0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int kz = k0 + r, n = n0 + tx;
        const int k = kz_to_k(kz, kl);
        t[r][tx] = (k >= 0 && n < N) ? L[(size_t)k * N + n] * rscale[k] : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        int n = n0 + r, k = k0 + tx;
        if (n < N_pad && k < KZ_pad) {
            float v = t[tx][r];
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            hi[(size_t)n * KZ_pad + k] = h;
            lo[(size_t)n * KZ_pad + k] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

// The same split in the age-block order: column ka = i * KBLOCK + j of the
// output [N_pad][KA_pad] takes SSP row k = i * n_z + j (n_u = 1; zero for
// j >= n_z and the padding); wmul_ab[ka] = 1 / rscale[k] = 2^E_k.
__global__ void build_lab_kernel(const float *L, const float *rscale, int N, int n_age, int n_z, int KA_pad,
                                 int N_pad, __nv_bfloat16 *hi, __nv_bfloat16 *lo, float *wmul_ab) {
    __shared__ float t[32][33];
    const int ka0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int i = ka0 / KBLOCK;                    // one age per 32 columns
    for (int r = ty; r < 32; r += 8) {
        const int j = r, n = n0 + tx;
        const bool ok = i < n_age && j < n_z && n < N;
        const int k = i * n_z + j;
        t[r][tx] = ok ? L[(size_t)k * N + n] * rscale[k] : 0.f;
    }
    if (blockIdx.x == 0 && ty == 0) {
        const int j = tx;
        wmul_ab[ka0 + j] = (i < n_age && j < n_z && rscale[i * n_z + j] > 0.f) ? 1.f / rscale[i * n_z + j] : 0.f;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        int n = n0 + r, k = ka0 + tx;
        if (n < N_pad && k < KA_pad) {
            float v = t[tx][r];
            __nv_bfloat16 h = __float2bfloat16_rn(v);
            hi[(size_t)n * KA_pad + k] = h;
            lo[(size_t)n * KA_pad + k] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

// Differenced block (see the top of the file), FP32 [KZ_pad][N_pad],
// metallicity-major rows (padding zero).
__global__ void build_ldiff_kernel(const float *L, int N, KzLayout kl, int u_ref, int KZ_pad, int N_pad,
                                   float *Ld) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)KZ_pad * N_pad) return;
    const int kz = (int)(idx / N_pad), n = (int)(idx % N_pad);
    const int k = kz_to_k(kz, kl);
    float v = 0.f;
    if (k >= 0 && n < N) {
        const int u = k % kl.n_u, j = (k / kl.n_u) % kl.n_z;
        // D_j L at log U bin uu
        auto dj = [&](int uu) {
            const int kk = k - u + uu;
            float d = L[(size_t)kk * N + n];
            if (j > 0) d -= L[(size_t)(kk - kl.n_u) * N + n];
            return d;
        };
        v = dj(u);
        if (u != u_ref) v -= dj(u_ref);
    }
    Ld[idx] = v;
}

// Binary exponent of max_n |row k| of a [K_pad][N_pad] block.
__global__ void row_exponent_abs_kernel(const float *A, int K, int N_pad, float *wmul, float *rscale) {
    const int k = blockIdx.x;
    float m = 0.f;
    if (k < K)
        for (int n = threadIdx.x; n < N_pad; n += blockDim.x) m = fmaxf(m, fabsf(A[(size_t)k * N_pad + n]));
    __shared__ float red[32];
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float mm = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmaxf(mm, red[w]);
        int E = mm > 0.f ? ilogbf(mm) : 0;
        E = max(-120, min(120, E));
        wmul[k] = k < K ? ldexpf(1.f, E) : 0.f;
        rscale[k] = k < K ? ldexpf(1.f, -E) : 0.f;
    }
}

// Row-scaled bf16 split of a [K_pad][N_pad] FP32 block.
__global__ void build_split_kernel(const float *A, const float *rscale, int K_pad, int N_pad, __nv_bfloat16 *hi,
                                   __nv_bfloat16 *lo) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)K_pad * N_pad) return;
    const float v = A[idx] * rscale[idx / N_pad];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[idx] = h;
    lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// Row ka of the age-block differenced copy from row kz of d_L_* (bf16 pairs
// moved as 32-bit words; N_pad is even).
__global__ void build_ldab_kernel(const __nv_bfloat16 *hi, const __nv_bfloat16 *lo, int n_age, int n_z, int A_pad,
                                  int N_pad, __nv_bfloat16 *ohi, __nv_bfloat16 *olo) {
    const int ka = blockIdx.y, i = ka / KBLOCK, j = ka % KBLOCK;
    const bool ok = i < n_age && j < n_z;
    const size_t src = (size_t)(j * A_pad + i) * N_pad, dst = (size_t)ka * N_pad;
    for (int n2 = blockIdx.x * blockDim.x + threadIdx.x; 2 * n2 < N_pad; n2 += gridDim.x * blockDim.x) {
        const unsigned vh = ok ? reinterpret_cast<const unsigned *>(hi + src)[n2] : 0u;
        const unsigned vl = ok ? reinterpret_cast<const unsigned *>(lo + src)[n2] : 0u;
        reinterpret_cast<unsigned *>(ohi + dst)[n2] = vh;
        reinterpret_cast<unsigned *>(olo + dst)[n2] = vl;
    }
}

}  // namespace

cudaError_t prepare_ssp_device(Ctx &c, const float *h_lssp) {
    const size_t KN = (size_t)c.K * c.n_lam;
    float *d_raw = nullptr, *d_rscale = nullptr;
    cudaError_t e = cudaMalloc(&d_raw, KN * sizeof(float));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&d_rscale, (size_t)(c.K_pad > c.KZ_pad ? c.K_pad : c.KZ_pad) * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(d_raw, h_lssp, KN * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c.d_wmul, 0, (size_t)c.KZ_pad * sizeof(float));
    if (e == cudaSuccess) {
        const KzLayout kl = c.kzl();
        row_exponent_kernel<<<c.K_pad, 256>>>(d_raw, c.K, c.n_lam, c.K_pad, kl, c.d_wmul, d_rscale);
        const size_t tot = (size_t)c.K_pad * c.N_pad;
        build_l32_kernel<<<(unsigned)((tot + 255) / 256), 256>>>(d_raw, c.K, c.n_lam, c.K_pad, c.N_pad, c.d_L32);
        dim3 g(c.N_pad / 32, c.KZ_pad / 32), b(32, 8);
        build_lt_kernel<<<g, b>>>(d_raw, d_rscale, c.n_lam, c.KZ_pad, c.N_pad, kl, c.d_Lt_hi, c.d_Lt_lo);
        if (c.KA_pad) {
            dim3 ga(c.N_pad / 32, c.KA_pad / 32);
            build_lab_kernel<<<ga, b>>>(d_raw, d_rscale, c.n_lam, c.n_age, c.n_z, c.KA_pad, c.N_pad, c.d_Lab_hi,
                                        c.d_Lab_lo, c.d_wmul_ab);
        }
        const size_t totz = (size_t)c.KZ_pad * c.N_pad;
        const unsigned blkz = (unsigned)((totz + 255) / 256);
        build_ldiff_kernel<<<blkz, 256>>>(d_raw, c.n_lam, kl, c.u_ref, c.KZ_pad, c.N_pad, c.d_Ld32);
        row_exponent_abs_kernel<<<c.KZ_pad, 256>>>(c.d_Ld32, c.KZ_pad, c.N_pad, c.d_wmul_d, d_rscale);
        build_split_kernel<<<blkz, 256>>>(c.d_Ld32, d_rscale, c.KZ_pad, c.N_pad, c.d_L_hi, c.d_L_lo);
        if (c.d_Ldab_hi)
            build_ldab_kernel<<<dim3(4, c.KA_pad), 256>>>(c.d_L_hi, c.d_L_lo, c.n_age, c.n_z, c.A_pad, c.N_pad,
                                                         c.d_Ldab_hi, c.d_Ldab_lo);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    cudaFree(d_rscale);
    cudaFree(d_raw);
    return e;
}

}  // namespace dsps
