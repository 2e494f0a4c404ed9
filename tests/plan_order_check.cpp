// Host check of the planner's ticket order (compiled by tests/test_tile_edges_host.py):
// for tile (and band) plans the order lists every tile once, by wave (sum of the
// tile's grid coordinates, decoded here by division) and by increasing linear
// index within a wave; for column plans by a + b; and wave_start marks where each
// wave begins. With the wave-shuffle test hook on, the same holds except the
// order inside a wave, which must differ from the canonical one somewhere.
#include <cstdio>
#include <string>
#include <vector>

#include "plan.h"
#include "plan_hooks.h"

using namespace msadp;

static int check(int k, const int32_t *lens, int A, int kernel, int edge, int64_t *moved = nullptr) {
    const bool shuffled = wave_shuffle_seed() != 0;
    HostPlan hp;
    std::string err;
    if (make_plan(k, lens, A, kernel, hp, err, edge) != 0) return printf("plan failed: %s\n", err.c_str()), 1;
    const int64_t nt = hp.ntiles;
    if ((int64_t)hp.order.size() != nt) return printf("order size\n"), 1;
    std::vector<char> seen((size_t)nt, 0);
    int64_t pos = 0;
    for (size_t w = 0; w + 1 < hp.wave_start.size(); ++w) {
        if (hp.wave_start[w] != pos) return printf("k=%d wave %zu starts at %lld, expected %lld\n", k, w, (long long)hp.wave_start[w], (long long)pos), 1;
        int64_t prev = -1;
        for (; pos < hp.wave_start[w + 1]; ++pos) {
            const int64_t t = (int64_t)hp.order[(size_t)pos];
            if (t < 0 || t >= nt || seen[(size_t)t]) return printf("k=%d tile %lld repeated or out of range\n", k, (long long)t), 1;
            seen[(size_t)t] = 1;
            int64_t wave = 0;
            if (hp.tb_layout == 1) {
                wave = t / hp.G[1] + t % hp.G[1];
            } else {
                int64_t rem = t;
                for (int i = 0; i < k; ++i) {
                    const int64_t c = rem / hp.gstride[i];
                    rem -= c * hp.gstride[i];
                    wave += c;
                }
                if (!shuffled && t <= prev) return printf("k=%d wave %zu not in index order\n", k, w), 1;
                if (shuffled && moved && t <= prev) ++*moved;
            }
            if (wave != (int64_t)w) return printf("k=%d tile %lld in wave %zu, belongs to %lld\n", k, (long long)t, w, (long long)wave), 1;
            prev = t;
        }
    }
    if (pos != nt) return printf("k=%d waves cover %lld of %lld tiles\n", k, (long long)pos, (long long)nt), 1;
    return 0;
}

int main() {
    int bad = 0;
    const int32_t l2[] = {1100, 700}, l3[] = {170, 99, 130}, l4[] = {80, 33, 61, 20}, l5[] = {10, 0, 9, 12, 3},
                  l6[] = {7, 9, 8, 6, 9, 5}, l7[] = {4, 5, 3, 6, 2, 5, 4}, l8[] = {3, 2, 4, 3, 1, 2, 3, 2},
                  l3c[] = {700, 760, 800}, l0[] = {0, 0, 0};
    bad += check(2, l2, 20, 1, 32);
    bad += check(2, l2, 20, 3, -1);  // band kernel: one ticket per 32-row band, in band order
    bad += check(2, l0, 4, 3, -1);
    bad += check(3, l3, 20, 1, 12);
    bad += check(3, l3, 20, 2, -1);
    bad += check(3, l3c, 20, 2, -1);
    bad += check(3, l0, 4, 1, 8);
    bad += check(4, l4, 4, 1, 4);
    bad += check(4, l4, 4, 1, 6);
    bad += check(5, l5, 4, 1, 4);
    bad += check(6, l6, 4, 1, 3);
    bad += check(7, l7, 4, 1, 2);
    bad += check(8, l8, 4, 1, 2);
    // another topological order: tickets permuted inside every wave
    set_wave_shuffle_seed(12345);
    int64_t moved = 0;
    bad += check(2, l2, 20, 1, 32, &moved);
    bad += check(3, l3, 20, 1, 12, &moved);
    bad += check(3, l3c, 20, 2, -1);
    bad += check(4, l4, 4, 1, 6, &moved);
    bad += check(6, l6, 4, 1, 3, &moved);
    bad += check(2, l2, 20, 3, -1);
    if (moved == 0) bad += printf("shuffled plans kept the canonical order\n") > 0;
    set_wave_shuffle_seed(0);
    if (!bad) printf("ok\n");
    return bad ? 1 : 0;
}
