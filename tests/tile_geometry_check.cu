// Host check of the generic tile kernel's shared-memory geometry (compiled by
// tests/test_tile_edges_host.py): for every compiled tile shape, the halo'd
// score layout with padded strides must place every halo'd cell at its own
// offset inside the tile buffer, predecessor offsets must be the sums of the
// moved axes' strides, and the halo cells counted for the halo table must be
// the cells with some local coordinate -1.
#include <cstdio>
#include <vector>

#include "device_common.cuh"

using namespace msadp;

static int check(int K, int E) {
    int ext[MSA_MAX_K], sh[MSA_MAX_K];
    long cells = 1;
    for (int j = 0; j < K; ++j) {
        ext[j] = tile_ext(K, E, j) + 1;
        sh[j] = geo_sh(K, E, j);
        cells *= ext[j];
    }
    const int volh = geo_volh(K, E);
    if (cells != geo_cellsh(K, E)) return printf("K=%d E=%d: cell count %ld != %d\n", K, E, cells, geo_cellsh(K, E)), 1;
    std::vector<char> used((size_t)volh, 0);
    long halo = 0;
    std::vector<int> d(K, 0);
    for (long c = 0; c < cells; ++c) {
        long r = c;
        int off = 0;
        bool h = false;
        for (int j = K - 1; j >= 0; --j) {
            d[j] = (int)(r % ext[j]);
            r /= ext[j];
            off += d[j] * sh[j];
            h = h || d[j] == 0;
        }
        if (off < 0 || off >= volh) return printf("K=%d E=%d: offset %d outside [0,%d)\n", K, E, off, volh), 1;
        if (used[(size_t)off]) return printf("K=%d E=%d: offset %d used twice\n", K, E, off), 1;
        used[(size_t)off] = 1;
        halo += h;
    }
    if (halo != geo_cellsh(K, E) - geo_vol(K, E)) return printf("K=%d E=%d: halo cells %ld\n", K, E, halo), 1;
    for (int m = 1; m < (1 << K); ++m) {
        int s = 0;
        for (int j = 0; j < K; ++j)
            if ((m >> j) & 1) s += sh[j];
        if (s != move_soff(K, E, m)) return printf("K=%d E=%d: move %d offset\n", K, E, m), 1;
    }
    if (sh[K - 1] != 1) return printf("K=%d E=%d: last stride %d\n", K, E, sh[K - 1]), 1;
    for (int j = 0; j + 1 < K; ++j)
        if (sh[j] < sh[j + 1] * ext[j + 1]) return printf("K=%d E=%d: stride %d overlaps\n", K, E, j), 1;
    return 0;
}

int main() {
    int bad = 0;
    for (int k = 2; k <= MSA_MAX_K; ++k)
        for (int i = 0; i < kMaxTileEdges; ++i)
            if (tile_edge_candidate(k, i) > 0) bad += check(k, tile_edge_candidate(k, i));
    if (!bad) printf("ok\n");
    return bad ? 1 : 0;
}
