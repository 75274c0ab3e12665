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
    (void)c; (void)n_gal; (void)params; (void)set_id; (void)precision; (void)mag_bar; (void)mags; (void)param_bar; (void)s;
    set_last_error("dsps_photometry_vjp: not built yet");
    return DSPS_ERR_UNSUPPORTED;
}

}  // namespace dsps
