// serve_host.h -- the host-only parts of the request loop (serve.cu): the
// first-fit arena over the HBM budget, the choice of the pieces that form a
// batch, and the host-side fault-injection switch.  Plain C++ without CUDA, so
// that the CPU tests build them under AddressSanitizer / UBSan.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cstdlib>
#include <iterator>
#include <map>
#include <string>
#include <vector>

namespace dsps {
namespace serve_host {

// First-fit allocator over one block, 256-byte granules, coalescing frees.
class Arena {
public:
    void reset(unsigned char *base, size_t bytes) {
        base_ = base;
        free_.clear();
        used_.clear();
        if (bytes) free_[0] = bytes;
        total_ = bytes;
    }
    unsigned char *alloc(size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, sz = it->second;
                free_.erase(it);
                if (sz > bytes) free_[off + bytes] = sz - bytes;
                used_[off] = bytes;
                return base_ + off;
            }
        }
        return nullptr;
    }
    void release(unsigned char *p) {
        if (!p) return;
        const size_t off = (size_t)(p - base_);
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t sz = u->second;
        used_.erase(u);
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + sz == nx->first) {
            sz += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += sz;
                return;
            }
        }
        free_[off] = sz;
    }
    size_t total() const { return total_; }
    size_t free_bytes() const {
        size_t b = 0;
        for (const auto &f : free_) b += f.second;
        return b;
    }
    size_t free_blocks() const { return free_.size(); }

private:
    unsigned char *base_ = nullptr;
    size_t total_ = 0;
    std::map<size_t, size_t> free_, used_;
};

// What decides whether two pieces may share a launch, and the piece's size.
struct PieceKey {
    int set_id = 0, precision = 0, grad = 0;
    int64_t n = 0;
};

// Indices (in queue order) of the pending pieces that form the next batch:
// the oldest piece fixes the kind (filter set, precision, gradient); later
// pieces of that kind join while the batch stays within piece_max galaxies.
inline std::vector<size_t> pick_batch(const std::vector<PieceKey> &pending, int64_t piece_max, int64_t *total) {
    std::vector<size_t> take;
    int64_t G = 0;
    if (!pending.empty()) {
        const PieceKey &h = pending.front();
        for (size_t i = 0; i < pending.size(); ++i) {
            const PieceKey &p = pending[i];
            if (p.set_id != h.set_id || p.precision != h.precision || p.grad != h.grad) continue;
            if (G + p.n > piece_max) break;
            take.push_back(i);
            G += p.n;
        }
    }
    if (total) *total = G;
    return take;
}

// DSPS_SERVE_FAULT: "fail_batch:N" (the N-th batch launch fails before any
// kernel) or "delay_us:X" (completions reported X us late); nothing else.
struct FaultSpec {
    int64_t fail_batch = -1;
    int64_t delay_us = 0;
};
inline FaultSpec parse_faults(const char *f) {
    FaultSpec s;
    if (!f) return s;
    const std::string v(f);
    if (v.rfind("fail_batch:", 0) == 0) s.fail_batch = std::atoll(v.c_str() + 11);
    if (v.rfind("delay_us:", 0) == 0) s.delay_us = std::atoll(v.c_str() + 9);
    if (s.delay_us < 0) s.delay_us = 0;
    return s;
}

}  // namespace serve_host
}  // namespace dsps
