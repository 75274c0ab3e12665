// static_scratch.cu -- FP32 photometry that performs no device allocation.
//
// Some callers cannot call cudaMalloc when they need magnitudes: a worker
// thread of a host framework whose device memory is owned by its own pooling
// allocator, or a latency-critical loop where an allocation (which may
// synchronise the device or fail under memory pressure) is not allowed.  For
// them dsps_photometry_fp32_static() runs the FP32 form of the photometry path
// using a context made earlier (its resident SSP block, filter tables and
// cosmology table) and, for the per-call scratch (weights, per-galaxy epilogue
// constants), the fixed array below instead of the context's work space.
//
// The array is a file-scope __device__ object of STATIC_SCRATCH_BYTES: every
// GPU that loads this library holds it until the process exits.  Host code
// cannot use the symbol g_static_scratch as a device address (on the host it
// names a host-side stand-in), so the device address is fetched once per
// device with cudaGetSymbolAddress, with that device current, on the first
// call that runs on it.  Every call shares the array and it keeps the last
// call's contents; the kernels overwrite every byte they later read, so nothing
// needs clearing.  Calls whose executions overlap on the GPU (two streams, or
// two host threads) race on the array.
#include <cstdio>
#include <mutex>

#include "dsps_internal.cuh"

namespace dsps {
void set_last_error(const char *msg);
}

using namespace dsps;

namespace {

constexpr size_t STATIC_SCRATCH_BYTES = (size_t)64 << 20;   // 64 MiB
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

std::mutex g_addr_mu;
void *g_addr[MAX_DEVICES] = {};

// Device address of g_static_scratch on `dev` (which must be current).
cudaError_t scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_addr[dev]);
    return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Largest population that fits: [rows][K_pad] FP32 weights, then
// [rows][AUX_STRIDE] FP32 constants, [rows] FP32 magnitude offsets and
// [rows] GalPrep (the layout of the context's work space, Workspace).
int64_t max_rows(int K_pad) {
    const size_t per = (size_t)K_pad * 4 + AUX_STRIDE * 4 + 4 + sizeof(GalPrep);
    int64_t r = (int64_t)((STATIC_SCRATCH_BYTES - 4 * 256) / per);
    while (r > 0 && align256((size_t)r * K_pad * 4) + align256((size_t)r * AUX_STRIDE * 4) +
                            align256((size_t)r * 4) + align256((size_t)r * sizeof(GalPrep)) > STATIC_SCRATCH_BYTES)
        --r;
    return r;
}

}  // namespace

extern "C" int dsps_photometry_fp32_static(dsps_ctx *ctx, int64_t n_gal, const float *params, int32_t set_id,
                                           float *mags, dsps_stream_t stream) {
    DSPS_TRACE("dsps_photometry_fp32_static");
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c || n_gal < 0 || (n_gal > 0 && (!params || !mags))) {
        set_last_error("dsps_photometry_fp32_static: bad argument");
        return DSPS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(c->mu);
    if (set_id < 0 || set_id >= (int)c->sets.size()) {
        set_last_error("dsps_photometry_fp32_static: unknown filter set");
        return DSPS_ERR_INVALID_ARG;
    }
    if (c->opts.dust_agedep) {
        set_last_error("dsps_photometry_fp32_static: not with age-dependent dust");
        return DSPS_ERR_UNSUPPORTED;
    }
    const int64_t cap = max_rows(c->K_pad);
    if (n_gal > cap) {
        char buf[256];
        std::snprintf(buf, sizeof buf,
                      "dsps_photometry_fp32_static: %lld galaxies exceed the %lld that fit the %zu-byte static "
                      "scratch for this grid",
                      (long long)n_gal, (long long)cap, STATIC_SCRATCH_BYTES);
        set_last_error(buf);
        return DSPS_ERR_INVALID_ARG;
    }
    if (n_gal == 0) return DSPS_OK;
    if (c->device < 0 || c->device >= MAX_DEVICES) {
        set_last_error("dsps_photometry_fp32_static: device index beyond the static scratch table");
        return DSPS_ERR_UNSUPPORTED;
    }
    if (cudaSetDevice(c->device) != cudaSuccess) {
        set_last_error("dsps_photometry_fp32_static: cudaSetDevice failed");
        return DSPS_ERR_CUDA;
    }
    unsigned char *base = nullptr;
    cudaError_t e = scratch_address(c->device, &base);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return DSPS_ERR_CUDA;
    }
    Workspace ws;
    ws.cap = cap;
    ws.w32 = reinterpret_cast<float *>(base);
    const size_t off_aux = align256((size_t)cap * c->K_pad * 4);
    ws.aux = reinterpret_cast<float *>(base + off_aux);
    const size_t off_mo = off_aux + align256((size_t)cap * AUX_STRIDE * 4);
    ws.magoff = reinterpret_cast<float *>(base + off_mo);
    ws.prep = reinterpret_cast<GalPrep *>(base + off_mo + align256((size_t)cap * 4));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const FilterSet &fs = c->sets[set_id];
    ws.rest = fs.rest;
    e = launch_weights(*c, ws, W_OMEGA_F32, params, n_gal, 0, n_gal, nullptr, s);
    if (e == cudaSuccess) e = launch_phot_simt(*c, ws, fs, n_gal, mags, s);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return DSPS_ERR_CUDA;
    }
    return DSPS_OK;
}
