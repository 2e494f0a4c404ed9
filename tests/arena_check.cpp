// Randomised check of the serving arena's first-fit bookkeeping (host only).
#include <cstdio>
#include <cstdlib>
#include <map>
#include <vector>

#include "arena.h"

#define CHECK(c)                                                        \
    do {                                                                \
        if (!(c)) {                                                     \
            std::printf("FAIL line %d: %s\n", __LINE__, #c);            \
            return 1;                                                   \
        }                                                               \
    } while (0)

int main() {
    using msadp::Arena;
    const size_t cap = 1 << 20;
    Arena a(cap);
    CHECK(a.capacity() == cap && a.largest_free() == cap && a.in_use() == 0);
    CHECK(!a.release(0));
    CHECK(a.could_ever_fit(cap) && !a.could_ever_fit(cap + 1));
    std::map<size_t, size_t> live;  // offset -> rounded size
    unsigned long long x = 12345;
    auto rnd = [&](unsigned long long m) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        return (x >> 33) % m;
    };
    for (int step = 0; step < 200000; ++step) {
        if (live.empty() || rnd(3) != 0) {
            const size_t bytes = 1 + rnd(rnd(2) ? 4096 : 65536);
            size_t off = 0;
            // the lowest free block that fits must be the one chosen
            const bool ok = a.alloc(bytes, &off);
            const size_t need = (bytes + Arena::kAlign - 1) / Arena::kAlign * Arena::kAlign;
            size_t expect = (size_t)-1, prev_end = 0;
            for (const auto &b : live) {
                if (b.first - prev_end >= need) {
                    expect = prev_end;
                    break;
                }
                prev_end = b.first + b.second;
            }
            if (expect == (size_t)-1 && cap - prev_end >= need) expect = prev_end;
            CHECK(ok == (expect != (size_t)-1));
            if (!ok) continue;
            CHECK(off == expect && off % Arena::kAlign == 0 && off + need <= cap);
            live[off] = need;
        } else {
            auto it = live.begin();
            std::advance(it, rnd(live.size()));
            CHECK(a.release(it->first));
            CHECK(!a.release(it->first));
            live.erase(it);
        }
        size_t used = 0;
        for (const auto &b : live) used += b.second;
        CHECK(a.in_use() == used && a.blocks() == live.size());
    }
    for (const auto &b : live) CHECK(a.release(b.first));
    CHECK(a.in_use() == 0 && a.largest_free() == cap && a.blocks() == 0);
    std::printf("ok\n");
    return 0;
}
