// Host-side logic of the request loop (serve_host.h) driven under
// AddressSanitizer and UBSan by tests/test_sanitizers.py: random allocate /
// release sequences on the arena with its invariants checked after every
// operation, the batch choice on random queues, and the fault switch parser.
// Exits non-zero (or the sanitizer aborts) on any violation.
#include <cstdio>
#include <random>
#include <set>
#include <utility>
#include <vector>

#include "serve_host.h"

using dsps::serve_host::Arena;
using dsps::serve_host::PieceKey;

static int fails = 0;
#define CHECK(c)                                                         \
    do {                                                                 \
        if (!(c)) {                                                      \
            std::fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__); \
            ++fails;                                                     \
        }                                                                \
    } while (0)

static void arena_random(unsigned seed) {
    std::mt19937_64 rng(seed);
    const size_t total = (size_t)(1 + rng() % 64) << 20;
    std::vector<unsigned char> block(total);
    Arena a;
    a.reset(block.data(), total);
    std::vector<std::pair<unsigned char *, size_t>> live;   // pointer, rounded size
    for (int op = 0; op < 4000; ++op) {
        if (live.empty() || rng() % 3) {
            const size_t want = (size_t)(rng() % (total / 8 + 1));
            unsigned char *p = a.alloc(want);
            if (p) {
                const size_t sz = want ? (want + 255) & ~(size_t)255 : 256;
                CHECK(p >= block.data() && p + sz <= block.data() + total);
                CHECK(((size_t)(p - block.data()) & 255) == 0);
                for (auto &l : live) CHECK(p + sz <= l.first || l.first + l.second <= p);   // no overlap
                p[0] = 1;                      // the memory is usable
                p[sz - 1] = 2;
                live.push_back({p, sz});
            }
        } else {
            const size_t k = (size_t)(rng() % live.size());
            a.release(live[k].first);
            live.erase(live.begin() + (std::ptrdiff_t)k);
        }
        size_t used = 0;
        for (auto &l : live) used += l.second;
        CHECK(a.free_bytes() + used == total);
    }
    a.release(nullptr);                        // ignored
    for (auto &l : live) a.release(l.first);
    CHECK(a.free_bytes() == total);
    CHECK(a.free_blocks() == 1);               // coalesced back into one block
}

static void pick_random(unsigned seed) {
    std::mt19937 rng(seed);
    for (int rep = 0; rep < 500; ++rep) {
        std::vector<PieceKey> q(rng() % 20);
        // the loop cuts requests into pieces of at most 65536 galaxies
        for (auto &p : q) p = {int(rng() % 3), int(rng() % 2), int(rng() % 2), int64_t(1 + rng() % 65536)};
        int64_t G = -1;
        const auto take = dsps::serve_host::pick_batch(q, 65536, &G);
        if (q.empty()) {
            CHECK(take.empty() && G == 0);
            continue;
        }
        CHECK(!take.empty() && take[0] == 0);   // the oldest piece always leads
        int64_t sum = 0;
        for (size_t k = 0; k < take.size(); ++k) {
            const PieceKey &p = q[take[k]];
            CHECK(p.set_id == q[0].set_id && p.precision == q[0].precision && p.grad == q[0].grad);
            if (k) CHECK(take[k] > take[k - 1]);
            sum += p.n;
        }
        CHECK(sum == G && G <= 65536);
    }
}

static void faults() {
    using dsps::serve_host::parse_faults;
    CHECK(parse_faults(nullptr).fail_batch == -1 && parse_faults(nullptr).delay_us == 0);
    CHECK(parse_faults("fail_batch:3").fail_batch == 3);
    CHECK(parse_faults("delay_us:250").delay_us == 250);
    CHECK(parse_faults("delay_us:-5").delay_us == 0);
    CHECK(parse_faults("nonsense").fail_batch == -1);
    CHECK(parse_faults("").delay_us == 0);
}

int main() {
    for (unsigned s = 0; s < 24; ++s) arena_random(s);
    pick_random(7);
    faults();
    std::printf("sanitize_host: %d failures\n", fails);
    return fails ? 1 : 0;
}
