// dispatch.cu -- per-call driver of the fused path: for each chunk of at most
// w.cap galaxies, the weights kernel writes the chunk's SSP weights (in the
// operand form of the chosen contraction) and per-galaxy epilogue constants,
// then the photometry kernel contracts, attenuates, redshifts and integrates
// them into magnitudes (and, for the adjoint, the chain of vjp.cu).  All
// launches go to the given stream.
#include "dsps_internal.cuh"

namespace dsps {

void set_last_error(const char *msg);

namespace {
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

size_t workspace_bytes(const Ctx &c, int64_t rows, bool adjoint) {
    const size_t R = (size_t)rows;
    const size_t W32 = (size_t)(c.K_pad > c.KZ_pad ? c.K_pad : c.KZ_pad);
    const size_t WZ = (size_t)(c.KA_pad > c.KZ_pad ? c.KA_pad : c.KZ_pad);   // split-weight row (kz or age-block order)
    size_t b = al256(R * W32 * 4) + 2 * al256(R * WZ * 2) + al256(R * AUX_STRIDE * 4) + al256(R * 4) + al256(R * sizeof(GalPrep)) +
               2 * al256(R * 4) + al256((size_t)ZSORT_BUCKETS * 4) + al256((size_t)TC_PARTS * R * 3 * QSTRIDE_MAX * 4) +
               al256(R * QSTRIDE_MAX * 4) + 2 * al256((R / 128 + 1) * sizeof(int2)) + al256((R / 128 + 1) * c.kmask_words * 4) + al256(sizeof(int));
    if (adjoint) b += al256(R * c.N_pad * 4);
    if (c.opts.dust_agedep) b += al256(R * 5 * QSTRIDE_MAX * 4) + al256(R * c.KZ_pad * 4);
    return b;
}

Workspace workspace_carve(const Ctx &c, void *base, int64_t rows, bool adjoint) {
    const size_t R = (size_t)rows;
    unsigned char *p = static_cast<unsigned char *>(base);
    auto take = [&](size_t bytes) {
        void *q = p;
        p += al256(bytes);
        return q;
    };
    Workspace w;
    w.cap = rows;
    w.w32 = static_cast<float *>(take(R * (size_t)(c.K_pad > c.KZ_pad ? c.K_pad : c.KZ_pad) * 4));
    const size_t WZ = (size_t)(c.KA_pad > c.KZ_pad ? c.KA_pad : c.KZ_pad);
    w.whi = static_cast<__nv_bfloat16 *>(take(R * WZ * 2));
    w.wlo = static_cast<__nv_bfloat16 *>(take(R * WZ * 2));
    w.aux = static_cast<float *>(take(R * AUX_STRIDE * 4));
    w.magoff = static_cast<float *>(take(R * 4));
    w.prep = static_cast<GalPrep *>(take(R * sizeof(GalPrep)));
    w.perm = static_cast<int *>(take(R * 4));
    w.gidx = static_cast<int *>(take(R * 4));
    w.hist = static_cast<int *>(take((size_t)ZSORT_BUCKETS * 4));
    w.partial = static_cast<float *>(take((size_t)TC_PARTS * R * 3 * QSTRIDE_MAX * 4));
    w.cq = static_cast<float *>(take(R * QSTRIDE_MAX * 4));
    w.trange = static_cast<int2 *>(take((R / 128 + 1) * sizeof(int2)));
    w.urange = static_cast<int2 *>(take((R / 128 + 1) * sizeof(int2)));
    w.kmask = static_cast<unsigned *>(take((R / 128 + 1) * c.kmask_words * 4));
    w.sched = static_cast<int *>(take(sizeof(int)));
    w.shat = adjoint ? take(R * c.N_pad * 4) : nullptr;
    if (c.opts.dust_agedep) {
        w.gacc = static_cast<float *>(take(R * 5 * QSTRIDE_MAX * 4));
        w.what2 = static_cast<float *>(take(R * c.KZ_pad * 4));
    }
    return w;
}

int run_photometry_ws(Ctx *c, const Workspace &w0, int64_t n_gal, const float *params, const FilterSet &fs,
                      int32_t precision, float *mags, cudaStream_t s, bool profile, const HistArgs *hist) {
    if (c->opts.dust_agedep) return run_photometry_agedep_ws(c, w0, n_gal, params, fs, precision, mags, s, profile, hist);
    Workspace w = w0;
    w.rest = fs.rest;
    w.stats = (profile && c->prof) ? c->d_stats : nullptr;
    const bool prof = profile && c->prof;
    for (int64_t g0 = 0; g0 < n_gal; g0 += w.cap) {
        const int64_t n = n_gal - g0 < w.cap ? n_gal - g0 : w.cap;
        cudaError_t e = cudaSuccess;
        if (precision == DSPS_PREC_FP32) {
            {
                ProfScope ps(*c, 0, s, prof);
                e = launch_zsort(*c, w, params, n_gal, g0, n, s);
                if (e == cudaSuccess) e = launch_weights(*c, w, W_OMEGA_F32, params, n_gal, g0, n, nullptr, s, true);
            }
            int parts = 1;
            if (e == cudaSuccess) {
                ProfScope ps(*c, 1, s, prof);
                e = launch_phot_simt(*c, w, fs, n, nullptr, s, false, true, nullptr, &parts);
            }
            if (e == cudaSuccess) {
                // per-part filter sums in a fixed order -> magnitudes (or the histogram)
                ProfScope ps(*c, 0, s, prof);
                e = launch_combine(*c, w, fs, n, parts, hist ? nullptr : mags + g0 * fs.Q, s, hist);
            }
        } else {
            int parts = 0;
            {
                ProfScope ps(*c, 0, s, prof);
                e = launch_zsort(*c, w, params, n_gal, g0, n, s);
                if (e == cudaSuccess) e = launch_weights(*c, w, W_OMEGA_BF16X2, params, n_gal, g0, n, nullptr, s, true);
            }
            if (e == cudaSuccess) {
                ProfScope ps(*c, 2, s, prof);
                e = launch_phot_tc(*c, w, fs, n, &parts, s);
            }
            if (e == cudaSuccess) {
                ProfScope ps(*c, 0, s, prof);
                e = launch_combine(*c, w, fs, n, parts, hist ? nullptr : mags + g0 * fs.Q, s, hist);
            }
        }
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            return DSPS_ERR_CUDA;
        }
    }
    return DSPS_OK;
}

int run_photometry_vjp_ws(Ctx *c, const Workspace &w0, int64_t n_gal, const float *params, const FilterSet &fs,
                          int32_t precision, const float *mag_bar, float *mags, float *param_bar, cudaStream_t s,
                          bool profile) {
    if (c->opts.dust_agedep)
        return run_photometry_vjp_agedep_ws(c, w0, n_gal, params, fs, precision, mag_bar, mags, param_bar, s, profile);
    Workspace w = w0;
    w.rest = fs.rest;
    w.stats = (profile && c->prof) ? c->d_stats : nullptr;
    const bool prof = profile && c->prof;
    const bool tc = precision == DSPS_PREC_BF16X3;
    for (int64_t g0 = 0; g0 < n_gal; g0 += w.cap) {
        const int64_t n = n_gal - g0 < w.cap ? n_gal - g0 : w.cap;
        cudaError_t e = cudaSuccess;
        int parts = 1;
        {
            ProfScope ps(*c, 0, s, prof);
            e = launch_zsort(*c, w, params, n_gal, g0, n, s);
            if (e == cudaSuccess)
                e = launch_weights(*c, w, tc ? W_OMEGA_BF16X2 : W_OMEGA_F32, params, n_gal, g0, n, nullptr, s, true);
        }
        if (e == cudaSuccess) {
            ProfScope ps(*c, tc ? 2 : 1, s, prof);
            e = tc ? launch_phot_tc(*c, w, fs, n, &parts, s, true)
                   : launch_phot_simt(*c, w, fs, n, nullptr, s, true, true, nullptr, &parts);
        }
        if (e == cudaSuccess) {
            ProfScope ps(*c, 3, s, prof);
            e = launch_combine_grad(*c, w, fs, n, parts, true, mag_bar + g0 * fs.Q, mags ? mags + g0 * fs.Q : nullptr,
                                    param_bar, n_gal, g0, s);
            if (e == cudaSuccess) e = launch_shat(*c, w, fs, n, tc, c->opts.band_skip != 0, s);
            if (e == cudaSuccess) e = tc ? launch_vjp_tc(*c, w, fs, n, s) : launch_vjp_simt(*c, w, n, s, 0, -1, &fs);
            if (e == cudaSuccess) e = launch_weights_vjp(*c, w, params, n_gal, g0, n, true, tc, param_bar, s);
        }
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            return DSPS_ERR_CUDA;
        }
    }
    return DSPS_OK;
}

int ensure_shat(Ctx *c, bool ewacc) {
    // [chunk][N_pad] x 4 bytes each, made on the first call that needs them:
    // Shat of the adjoint (FP32, or bf16 hi + lo), the window spectra of the
    // line widths; and the line widths' summed window under age-dependent dust.
    void **slots[2] = {&c->ws.shat, reinterpret_cast<void **>(&c->ws.ewacc)};
    for (int i = 0; i < (ewacc ? 2 : 1); ++i) {
        if (*slots[i]) continue;
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, (size_t)c->chunk * c->N_pad * 4);
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            return DSPS_ERR_CUDA;
        }
        *slots[i] = p;
    }
    return DSPS_OK;
}

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
    return run_photometry_ws(c, c->ws, n_gal, params, c->sets[set_id], precision, mags, s, true);
}

int run_photometry_host(Ctx *c, int64_t n_gal, const float *h_params, int32_t set_id, int32_t precision,
                        float *h_mags, cudaStream_t s) {
    if (n_gal < 0 || (n_gal > 0 && (!h_params || !h_mags))) {
        set_last_error("dsps_photometry_host: bad argument");
        return DSPS_ERR_INVALID_ARG;
    }
    if (set_id < 0 || set_id >= (int)c->sets.size()) {
        set_last_error("dsps_photometry_host: unknown filter set");
        return DSPS_ERR_INVALID_ARG;
    }
    if (precision != DSPS_PREC_FP32 && precision != DSPS_PREC_BF16X3) {
        set_last_error("dsps_photometry_host: unknown precision");
        return DSPS_ERR_INVALID_ARG;
    }
    if (n_gal == 0) return DSPS_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return DSPS_ERR_CUDA;
    const FilterSet &fs = c->sets[set_id];
    // one chunk of inputs [npar][chunk] and outputs [chunk][Q] on the device
    const int64_t chunk = n_gal < c->chunk ? n_gal : c->chunk;
    const size_t in_bytes = al256((size_t)chunk * c->npar * 4);
    const size_t need = in_bytes + al256((size_t)chunk * fs.Q * 4);
    if (c->hio_bytes < need) {
        if (c->d_hio) cudaFree(c->d_hio);
        c->d_hio = nullptr;
        c->hio_bytes = 0;
        cudaError_t e = cudaMalloc(&c->d_hio, need);
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            return DSPS_ERR_CUDA;
        }
        c->hio_bytes = need;
    }
    float *d_p = reinterpret_cast<float *>(c->d_hio);
    float *d_m = reinterpret_cast<float *>(c->d_hio + in_bytes);
    for (int64_t g0 = 0; g0 < n_gal; g0 += chunk) {
        const int64_t n = n_gal - g0 < chunk ? n_gal - g0 : chunk;
        // rows g0 .. g0 + n of every parameter row: one strided copy
        cudaError_t e = cudaMemcpy2DAsync(d_p, (size_t)n * 4, h_params + g0, (size_t)n_gal * 4, (size_t)n * 4,
                                          (size_t)c->npar, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            return DSPS_ERR_CUDA;
        }
        const int rc = run_photometry_ws(c, c->ws, n, d_p, fs, precision, d_m, s, true);
        if (rc != DSPS_OK) return rc;
        e = cudaMemcpyAsync(h_mags + g0 * fs.Q, d_m, (size_t)n * fs.Q * 4, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) {
            set_last_error(cudaGetErrorString(e));
            return DSPS_ERR_CUDA;
        }
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return DSPS_ERR_CUDA;
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
    const int rc = ensure_shat(c);
    if (rc != DSPS_OK) return rc;
    return run_photometry_vjp_ws(c, c->ws, n_gal, params, c->sets[set_id], precision, mag_bar, mags, param_bar, s,
                                 true);
}

}  // namespace dsps
