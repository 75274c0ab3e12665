// serve.cu -- request loop with continuous batching (dsps_submit / dsps_poll).
//
// A request is a population of galaxies in host memory, or in device memory
// (dsps_request.buffers = DSPS_BUF_DEVICE: copied device to device into the
// batch's inputs and out of its outputs, no host staging).  It is cut into
// pieces of at most PIECE_MAX galaxies.  A scheduler thread forms a batch from
// the oldest pending piece plus later pending pieces of the same kind (filter
// set, precision, gradient or not) up to PIECE_MAX galaxies, and launches it as
// soon as a stream is free and the batch's whole device footprint (work space
// + inputs + outputs) fits in the HBM-budget arena; pieces that arrive while
// other batches run are admitted as streams and memory free up, so their
// copies and kernels overlap on the device.  A finished batch (event polled)
// has its outputs copied back into the callers' buffers and its memory
// returned.  Every galaxy's result is independent of the batch it rides in
// (the kernels compute rows independently), so it equals a lone call.
//
// Host-side fault injection (tests; nothing touches the GPU):
//   DSPS_SERVE_FAULT=fail_batch:N   the N-th batch launch fails before any
//                                   launch; its requests complete with
//                                   DSPS_ERR_CUDA, the loop carries on
//   DSPS_SERVE_FAULT=delay_us:X     completion is reported X us late
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dsps_internal.cuh"
#include "serve_host.h"

namespace dsps {

void set_last_error(const char *msg);

namespace {

using Clock = std::chrono::steady_clock;
constexpr int64_t PIECE_MAX = 65536;

using serve_host::Arena;

struct Req {
    uint64_t ticket = 0;
    dsps_request r{};
    bool dev = false;           // buffers in device memory
    int Q = 0;
    int64_t pieces_left = 0;
    int status = DSPS_OK;
    bool done = false;
    Clock::time_point t_submit, t_done;
};

struct Piece {
    std::shared_ptr<Req> req;
    int64_t start = 0, n = 0;   // galaxies [start, start + n) of the request
};

struct Batch {
    int slot = -1;
    std::vector<Piece> pieces;
    std::vector<int64_t> off;   // row offset of each piece in the batch
    int64_t G = 0;
    int Q = 0, set_id = 0, precision = 0, grad = 0;
    bool any_host = false;      // some piece has host buffers (host staging used)
    unsigned char *dev = nullptr, *host = nullptr;
    float *h_params = nullptr, *h_mbar = nullptr, *h_mags = nullptr, *h_pbar = nullptr;
    cudaEvent_t ev = nullptr;
    int status = DSPS_OK;
    Clock::time_point ready_at;
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct Serve {
    Ctx *c = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Piece> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Req>> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_busy;
    std::vector<Batch> inflight;
    unsigned char *dev_block = nullptr, *host_block = nullptr;
    Arena dev, host;
    int64_t batches = 0;
    int64_t fault_fail_batch = -1;
    int64_t fault_delay_us = 0;

    size_t dev_bytes(int64_t G, int Q, bool grad) const {
        size_t b = workspace_bytes(*c, G, grad) + al256(G * c->npar * 4) + al256(G * Q * 4);
        if (grad) b += al256(G * Q * 4) + al256(G * c->ngrad * 4);
        return b;
    }
    size_t host_bytes(int64_t G, int Q, bool grad) const {
        size_t b = al256(G * c->npar * 4) + al256(G * Q * 4);
        if (grad) b += al256(G * Q * 4) + al256(G * c->ngrad * 4);
        return b;
    }
    void loop();
    bool try_launch(std::unique_lock<std::mutex> &lk);
    void launch(Batch &b);
    void finish(Batch &b);
};

namespace {

void parse_faults(Serve *s) {
    const serve_host::FaultSpec f = serve_host::parse_faults(std::getenv("DSPS_SERVE_FAULT"));
    s->fault_fail_batch = f.fail_batch;
    s->fault_delay_us = f.delay_us;
}

}  // namespace

int serve_start(Ctx *c) {
    if (c->serve) return DSPS_OK;
    auto *s = new Serve();
    s->c = c;
    parse_faults(s);
    const size_t dbytes = (size_t)std::max<int64_t>(c->opts.hbm_budget_bytes, 1 << 20);
    // Host staging: inputs and outputs are at most 220 bytes per galaxy of a
    // work space that costs at least ~9 KB per galaxy on the device.
    const size_t hbytes = std::max<size_t>(dbytes / 32, (size_t)64 << 20);
    if (cudaSetDevice(c->device) != cudaSuccess || cudaMalloc(&s->dev_block, dbytes) != cudaSuccess) {
        delete s;
        set_last_error("dsps_submit: could not allocate the request loop's HBM arena");
        return DSPS_ERR_CUDA;
    }
    if (cudaMallocHost(&s->host_block, hbytes) != cudaSuccess) {
        cudaFree(s->dev_block);
        delete s;
        set_last_error("dsps_submit: could not allocate pinned staging");
        return DSPS_ERR_CUDA;
    }
    s->dev.reset(s->dev_block, dbytes);
    s->host.reset(s->host_block, hbytes);
    const int ns = std::max(1, c->opts.n_streams);
    s->streams.resize(ns);
    s->slot_busy.assign(ns, false);
    for (auto &st : s->streams) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    c->serve = s;
    s->th = std::thread([s] { s->loop(); });
    return DSPS_OK;
}

void serve_stop(Ctx *c) {
    Serve *s = c->serve;
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    cudaSetDevice(c->device);
    for (auto &b : s->inflight) {
        cudaEventSynchronize(b.ev);
        cudaEventDestroy(b.ev);
    }
    for (auto &st : s->streams) cudaStreamDestroy(st);
    cudaFree(s->dev_block);
    cudaFreeHost(s->host_block);
    c->serve = nullptr;
    delete s;
}

void Serve::launch(Batch &b) {
    // Host staging: params [npar][G] SoA and, for the gradient, mag_bar [G][Q],
    // of the pieces with host buffers.
    for (size_t i = 0; i < b.pieces.size(); ++i) {
        const Piece &p = b.pieces[i];
        const dsps_request &r = p.req->r;
        if (p.req->dev) continue;
        for (int row = 0; row < c->npar; ++row)
            std::memcpy(b.h_params + (size_t)row * b.G + b.off[i], r.params + (size_t)row * r.n_gal + p.start,
                        (size_t)p.n * 4);
        if (b.grad)
            std::memcpy(b.h_mbar + (size_t)b.off[i] * b.Q, r.mag_bar + (size_t)p.start * b.Q, (size_t)p.n * b.Q * 4);
    }
    cudaStream_t st = streams[b.slot];
    const bool grad = b.grad != 0;
    Workspace w = workspace_carve(*c, b.dev, b.G, grad);
    unsigned char *io = b.dev + workspace_bytes(*c, b.G, grad);
    float *d_params = reinterpret_cast<float *>(io);
    float *d_mags = reinterpret_cast<float *>(io + al256(b.G * c->npar * 4));
    float *d_mbar = grad ? reinterpret_cast<float *>(io + al256(b.G * c->npar * 4) + al256(b.G * b.Q * 4)) : nullptr;
    float *d_pbar = grad ? reinterpret_cast<float *>(io + al256(b.G * c->npar * 4) + 2 * al256(b.G * b.Q * 4)) : nullptr;
    FilterSet fs;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        fs = c->sets[b.set_id];
    }
    cudaError_t e = cudaSuccess;
    if (b.any_host) {
        e = cudaMemcpyAsync(d_params, b.h_params, (size_t)b.G * c->npar * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && grad)
            e = cudaMemcpyAsync(d_mbar, b.h_mbar, (size_t)b.G * b.Q * 4, cudaMemcpyHostToDevice, st);
    }
    // device pieces, after the staging copy (which carries no data for their rows)
    for (size_t i = 0; i < b.pieces.size() && e == cudaSuccess; ++i) {
        const Piece &p = b.pieces[i];
        const dsps_request &r = p.req->r;
        if (!p.req->dev) continue;
        e = cudaMemcpy2DAsync(d_params + b.off[i], (size_t)b.G * 4, r.params + p.start, (size_t)r.n_gal * 4,
                              (size_t)p.n * 4, (size_t)c->npar, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && grad)
            e = cudaMemcpyAsync(d_mbar + (size_t)b.off[i] * b.Q, r.mag_bar + (size_t)p.start * b.Q,
                                (size_t)p.n * b.Q * 4, cudaMemcpyDeviceToDevice, st);
    }
    int rc = e == cudaSuccess ? DSPS_OK : DSPS_ERR_CUDA;
    if (batches++ == fault_fail_batch) rc = DSPS_ERR_CUDA;   // injected, before any kernel
    if (rc == DSPS_OK)
        rc = grad ? run_photometry_vjp_ws(c, w, b.G, d_params, fs, b.precision, d_mbar, d_mags, d_pbar, st, false)
                  : run_photometry_ws(c, w, b.G, d_params, fs, b.precision, d_mags, st, false);
    if (rc == DSPS_OK) {
        if (b.any_host) {
            e = cudaMemcpyAsync(b.h_mags, d_mags, (size_t)b.G * b.Q * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && grad)
                e = cudaMemcpyAsync(b.h_pbar, d_pbar, (size_t)b.G * c->ngrad * 4, cudaMemcpyDeviceToHost, st);
        }
        for (size_t i = 0; i < b.pieces.size() && e == cudaSuccess; ++i) {
            const Piece &p = b.pieces[i];
            const dsps_request &r = p.req->r;
            if (!p.req->dev) continue;
            e = cudaMemcpyAsync(r.mags + (size_t)p.start * b.Q, d_mags + (size_t)b.off[i] * b.Q,
                                (size_t)p.n * b.Q * 4, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess && grad)
                e = cudaMemcpy2DAsync(r.param_bar + p.start, (size_t)r.n_gal * 4, d_pbar + b.off[i], (size_t)b.G * 4,
                                      (size_t)p.n * 4, (size_t)c->ngrad, cudaMemcpyDeviceToDevice, st);
        }
        if (e != cudaSuccess) rc = DSPS_ERR_CUDA;
    }
    b.status = rc;
    cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming);
    cudaEventRecord(b.ev, st);
    b.ready_at = Clock::now() + std::chrono::microseconds(fault_delay_us);
}

void Serve::finish(Batch &b) {
    if (b.status == DSPS_OK) {
        for (size_t i = 0; i < b.pieces.size(); ++i) {
            const Piece &p = b.pieces[i];
            const dsps_request &r = p.req->r;
            if (p.req->dev) continue;   // written on the device before the batch's event
            std::memcpy(r.mags + (size_t)p.start * b.Q, b.h_mags + (size_t)b.off[i] * b.Q, (size_t)p.n * b.Q * 4);
            if (b.grad)
                for (int k = 0; k < c->ngrad; ++k)
                    std::memcpy(r.param_bar + (size_t)k * r.n_gal + p.start, b.h_pbar + (size_t)k * b.G + b.off[i],
                                (size_t)p.n * 4);
        }
    }
    const auto now = Clock::now();
    for (auto &p : b.pieces) {
        Req &q = *p.req;
        if (b.status != DSPS_OK) q.status = b.status;
        if (--q.pieces_left == 0) {
            q.done = true;
            q.t_done = now;
        }
    }
    cudaEventDestroy(b.ev);
    dev.release(b.dev);
    host.release(b.host);
    slot_busy[b.slot] = false;
}

bool Serve::try_launch(std::unique_lock<std::mutex> &lk) {
    if (pending.empty()) return false;
    int slot = -1;
    for (size_t i = 0; i < slot_busy.size(); ++i)
        if (!slot_busy[i]) { slot = (int)i; break; }
    if (slot < 0) return false;
    // The oldest piece fixes the kind; later pieces of that kind join while they fit.
    const Piece &head = pending.front();
    Batch b;
    b.set_id = head.req->r.set_id;
    b.precision = head.req->r.precision;
    b.grad = head.req->r.want_grad ? 1 : 0;
    b.Q = head.req->Q;
    std::vector<serve_host::PieceKey> keys(pending.size());
    for (size_t i = 0; i < pending.size(); ++i) {
        const dsps_request &r = pending[i].req->r;
        keys[i] = {r.set_id, r.precision, r.want_grad ? 1 : 0, pending[i].n};
    }
    int64_t G = 0;
    const std::vector<size_t> take = serve_host::pick_batch(keys, PIECE_MAX, &G);
    for (size_t i : take) b.any_host = b.any_host || !pending[i].req->dev;
    const int64_t Gpad = (G + 127) / 128 * 128;
    unsigned char *d = dev.alloc(dev_bytes(Gpad, b.Q, b.grad));
    if (!d) return false;    // admission by memory: wait for a batch to finish
    unsigned char *h = nullptr;
    if (b.any_host) {
        h = host.alloc(host_bytes(G, b.Q, b.grad));
        if (!h) {
            dev.release(d);
            return false;
        }
    }
    b.slot = slot;
    b.dev = d;
    b.host = h;
    b.G = G;
    b.h_params = reinterpret_cast<float *>(h);
    b.h_mags = reinterpret_cast<float *>(h + al256(G * c->npar * 4));
    if (b.grad && h) {
        b.h_mbar = reinterpret_cast<float *>(h + al256(G * c->npar * 4) + al256(G * b.Q * 4));
        b.h_pbar = reinterpret_cast<float *>(h + al256(G * c->npar * 4) + 2 * al256(G * b.Q * 4));
    }
    int64_t o = 0;
    for (size_t k = 0; k < take.size(); ++k) {
        b.pieces.push_back(pending[take[k]]);
        b.off.push_back(o);
        o += pending[take[k]].n;
    }
    for (size_t k = take.size(); k-- > 0;) pending.erase(pending.begin() + (std::ptrdiff_t)take[k]);
    slot_busy[slot] = true;
    lk.unlock();
    launch(b);
    lk.lock();
    inflight.push_back(b);
    return true;
}

void Serve::loop() {
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        // completions
        bool finished = false;
        for (size_t i = 0; i < inflight.size();) {
            Batch &b = inflight[i];
            if (cudaEventQuery(b.ev) == cudaSuccess && Clock::now() >= b.ready_at) {
                finish(b);
                inflight.erase(inflight.begin() + (std::ptrdiff_t)i);
                finished = true;
            } else {
                ++i;
            }
        }
        if (finished) cv_done.notify_all();
        // admissions
        while (try_launch(lk)) {
        }
        if (stop && inflight.empty()) break;
        if (stop && pending.empty() && inflight.empty()) break;
        if (inflight.empty() && pending.empty())
            cv_work.wait(lk, [this] { return stop || !pending.empty(); });
        else
            cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
}

namespace {

// Whether the device `dev` can address p as device memory (device or managed).
bool device_pointer(const void *p, int dev) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice && at.device == dev) || at.type == cudaMemoryTypeManaged;
}

}  // namespace

int serve_submit(Ctx *c, const dsps_request *r, uint64_t *ticket) {
    if (r->n_gal < 0 || (r->n_gal > 0 && (!r->params || !r->mags)) ||
        (r->want_grad && r->n_gal > 0 && (!r->mag_bar || !r->param_bar)) ||
        (r->precision != DSPS_PREC_FP32 && r->precision != DSPS_PREC_BF16X3) ||
        (r->buffers != DSPS_BUF_HOST && r->buffers != DSPS_BUF_DEVICE)) {
        set_last_error("dsps_submit: bad request");
        return DSPS_ERR_INVALID_ARG;
    }
    if (r->buffers == DSPS_BUF_DEVICE && r->n_gal > 0) {
        if (cudaSetDevice(c->device) != cudaSuccess) {
            set_last_error("dsps_submit: cudaSetDevice failed");
            return DSPS_ERR_CUDA;
        }
        const void *ptrs[4] = {r->params, r->mags, r->want_grad ? r->mag_bar : r->params,
                               r->want_grad ? r->param_bar : r->params};
        for (const void *p : ptrs)
            if (!device_pointer(p, c->device)) {
                set_last_error("dsps_submit: a DSPS_BUF_DEVICE request holds a pointer that is not device memory "
                               "of the context's device");
                return DSPS_ERR_INVALID_ARG;
            }
    }
    int Q = 0;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (r->set_id < 0 || r->set_id >= (int)c->sets.size()) {
            set_last_error("dsps_submit: unknown filter set");
            return DSPS_ERR_INVALID_ARG;
        }
        Q = c->sets[r->set_id].Q;
        int rc = serve_start(c);
        if (rc != DSPS_OK) return rc;
    }
    Serve *s = c->serve;
    const int64_t piece = std::min<int64_t>(PIECE_MAX, std::max<int64_t>(r->n_gal, 1));
    if (s->dev_bytes((piece + 127) / 128 * 128, Q, r->want_grad != 0) > s->dev.total() ||
        s->host_bytes(piece, Q, r->want_grad != 0) > s->host.total()) {
        set_last_error("dsps_submit: one piece of this request exceeds the HBM budget");
        return DSPS_ERR_OUT_OF_BUDGET;
    }
    auto q = std::make_shared<Req>();
    q->r = *r;
    q->dev = r->buffers == DSPS_BUF_DEVICE;
    q->Q = Q;
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        q->ticket = s->next_ticket++;
        s->reqs[q->ticket] = q;
        if (r->n_gal == 0) {
            q->done = true;
            q->t_done = q->t_submit;
        } else {
            for (int64_t st = 0; st < r->n_gal; st += PIECE_MAX) {
                Piece p;
                p.req = q;
                p.start = st;
                p.n = std::min<int64_t>(PIECE_MAX, r->n_gal - st);
                s->pending.push_back(p);
                ++q->pieces_left;
            }
        }
        *ticket = q->ticket;
    }
    s->cv_work.notify_one();
    return DSPS_OK;
}

int serve_poll(Ctx *c, uint64_t ticket, int64_t timeout_us, double *latency_us) {
    Serve *s = c->serve;
    if (!s) {
        set_last_error("dsps_poll: unknown ticket");
        return DSPS_ERR_NOT_FOUND;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_last_error("dsps_poll: unknown ticket");
        return DSPS_ERR_NOT_FOUND;
    }
    std::shared_ptr<Req> q = it->second;
    if (!q->done && timeout_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return q->done; });
    if (!q->done) {
        if (timeout_us <= 0) return DSPS_PENDING;
        set_last_error("dsps_poll: the wait timed out with the request unfinished");
        return DSPS_ERR_TIMEOUT;
    }
    if (latency_us)
        *latency_us = std::chrono::duration<double, std::micro>(q->t_done - q->t_submit).count();
    s->reqs.erase(it);
    if (q->status != DSPS_OK) set_last_error("dsps_poll: the request's batch failed");
    return q->status;
}

}  // namespace dsps
