// dispatch.cu -- per-call driver of the fused path: for each chunk of at most
// ctx.chunk galaxies, the weights kernel writes the chunk's SSP weights (in the
// operand form of the chosen contraction) and per-galaxy epilogue constants,
// then the photometry kernel contracts, attenuates, redshifts and integrates
// them into magnitudes.  Both launches go to the caller's stream.
#include "dsps_internal.cuh"

namespace dsps {

void set_last_error(const char *msg);

int run_photometry(Ctx *c, int64_t n_gal, const float *params, int32_t set_id, int32_t precision, float *mags,
                   cudaStream_t s) {
    if (n_gal < 0 || (n_gal > 0 && (!params || !mags))) {
        set_last_error("dsps_photometry: bad argument");
        return DSPS_ERR_INVALID_ARG;
    }
    if (set_id < 0 || set_id >= (int)c->sets.size()) {
        set_last_error("dsps_photometry: unknown filter set");
        return DSPS_ERR_INVALID_ARG;
    }
    if (precision != DSPS_PREC_FP32 && precision != DSPS_PREC_BF16X3) {
        set_last_error("dsps_photometry: unknown precision");
        return DSPS_ERR_INVALID_ARG;
    }
    if (n_gal == 0) return DSPS_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return DSPS_ERR_CUDA;
    const FilterSet &fs = c->sets[set_id];
    for (int64_t g0 = 0; g0 < n_gal; g0 += c->chunk) {
        const int64_t n = n_gal - g0 < c->chunk ? n_gal - g0 : c->chunk;
        cudaError_t e = cudaSuccess;
        if (precision == DSPS_PREC_FP32) {
            {
                ProfScope ps(*c, 0, s);
                e = launch_weights(*c, W_OMEGA_F32, params, n_gal, g0, n, nullptr, s);
            }
            if (e == cudaSuccess) {
                ProfScope ps(*c, 1, s);
                e = launch_phot_simt(*c, fs, n, mags + g0 * fs.Q, s);
            }
        } else {
            int parts = 0;
            {
                ProfScope ps(*c, 0, s);
                e = launch_zsort(*c, params + (int64_t)11 * n_gal + g0, n, s);
                if (e == cudaSuccess) e = launch_weights(*c, W_OMEGA_BF16X2, params, n_gal, g0, n, nullptr, s,
                                                         nullptr, true);
            }
            if (e == cudaSuccess) {
                ProfScope ps(*c, 2, s);
                e = launch_phot_tc(*c, fs, n, &parts, s);
            }
            if (e == cudaSuccess) {
                ProfScope ps(*c, 0, s);
                e = launch_combine(*c, fs, n, parts, mags + g0 * fs.Q, s);
            }
        }
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            return DSPS_ERR_CUDA;
        }
    }
    return DSPS_OK;
}

int run_photometry_vjp(Ctx *c, int64_t n_gal, const float *params, int32_t set_id, int32_t precision,
                       const float *mag_bar, float *mags, float *param_bar, cudaStream_t s) {
    if (n_gal < 0 || (n_gal > 0 && (!params || !mag_bar || !param_bar))) {
        set_last_error("dsps_photometry_vjp: bad argument");
        return DSPS_ERR_INVALID_ARG;
    }
    if (set_id < 0 || set_id >= (int)c->sets.size()) {
        set_last_error("dsps_photometry_vjp: unknown filter set");
        return DSPS_ERR_INVALID_ARG;
    }
    if (precision != DSPS_PREC_FP32 && precision != DSPS_PREC_BF16X3) {
        set_last_error("dsps_photometry_vjp: unknown precision");
        return DSPS_ERR_INVALID_ARG;
    }
    if (n_gal == 0) return DSPS_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return DSPS_ERR_CUDA;
    if (!c->d_shat) {
        // Adjoint work space, made on the first gradient call (FP32, or bf16 hi + lo).
        cudaError_t e = cudaMalloc(&c->d_shat, (size_t)c->chunk * c->N_pad * 4);
        if (e != cudaSuccess) {
            c->d_shat = nullptr;
            set_last_error(cudaGetErrorString(e));
            return DSPS_ERR_CUDA;
        }
    }
    const FilterSet &fs = c->sets[set_id];
    const bool tc = precision == DSPS_PREC_BF16X3;
    for (int64_t g0 = 0; g0 < n_gal; g0 += c->chunk) {
        const int64_t n = n_gal - g0 < c->chunk ? n_gal - g0 : c->chunk;
        cudaError_t e = cudaSuccess;
        int parts = 1;
        {
            ProfScope ps(*c, 0, s);
            if (tc) e = launch_zsort(*c, params + (int64_t)11 * n_gal + g0, n, s);
            if (e == cudaSuccess)
                e = launch_weights(*c, tc ? W_OMEGA_BF16X2 : W_OMEGA_F32, params, n_gal, g0, n, nullptr, s, nullptr,
                                   tc);
        }
        if (e == cudaSuccess) {
            ProfScope ps(*c, tc ? 2 : 1, s);
            e = tc ? launch_phot_tc(*c, fs, n, &parts, s, true) : launch_phot_simt(*c, fs, n, nullptr, s, nullptr, true);
        }
        if (e == cudaSuccess) {
            ProfScope ps(*c, 3, s);
            e = launch_combine_grad(*c, fs, n, parts, tc, mag_bar + g0 * fs.Q, mags ? mags + g0 * fs.Q : nullptr,
                                    param_bar, n_gal, g0, s);
            if (e == cudaSuccess) e = launch_shat(*c, fs, n, tc, tc && c->opts.band_skip, s);
            if (e == cudaSuccess) e = tc ? launch_vjp_tc(*c, fs, n, s) : launch_vjp_simt(*c, n, s);
            if (e == cudaSuccess) e = launch_weights_vjp(*c, params, n_gal, g0, n, tc, tc, param_bar, s);
        }
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            return DSPS_ERR_CUDA;
        }
    }
    return DSPS_OK;
}

}  // namespace dsps
