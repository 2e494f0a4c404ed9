// Host planner (hot-path step a2): shape rho_i = len_i + 1 (section 3.2), the
// mixed-radix row-major linear index of the tensor (section 2's shape- and
// dimension-invariant indexing: l = sum_i x_i * stride_i with the last axis
// fastest), the tile grid, and the ticket order of tiles by wave (section 3:
// tiles whose coordinates sum to w form wave w and are mutually independent).
#include "plan.h"
#include "plan_hooks.h"

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <mutex>

namespace msadp {

// The k = 3 column kernel handles alphabets up to c3::MAXA and a last axis up to
// c3::MAXRHO2 (both staged in shared memory).
static bool col3_fits(int k, const int32_t *lens, int A) {
    if (k != 3 || A > c3::MAXA) return false;
    return (int64_t)lens[2] + 1 <= c3::MAXRHO2;
}

namespace {
std::mutex g_tune_mu;
int g_edge[MSA_MAX_K + 1] = {};  // 0: default edge
bool g_k3_tiles = false;
bool g_k2_tiles = false;
int g_line_z[MSA_MAX_K + 1] = {};            // 0: default segment
bool g_lines_tiles[MSA_MAX_K + 1] = {};      // k = 4 .. 6: prefer the generic tile kernel
constexpr bool stream_default(int k) { return k >= 4 && k <= 6; }  // where the streamed form is the default
bool g_stream[MSA_MAX_K + 1] = {false, false, false, false, stream_default(4), stream_default(5), stream_default(6)};
}  // namespace

int tile_edge_for(int k) {
    if (k < 2 || k > MSA_MAX_K) return 0;
    std::lock_guard<std::mutex> g(g_tune_mu);
    return g_edge[k] ? g_edge[k] : tile_edge_default(k);
}

int set_tile_edge(int k, int edge) {
    if (k < 2 || k > MSA_MAX_K || (edge != 0 && !tile_edge_valid(k, edge))) return MSA_EINVAL;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_edge[k] = edge;
    return MSA_OK;
}

bool prefer_tiles_k3() {
    std::lock_guard<std::mutex> g(g_tune_mu);
    return g_k3_tiles;
}

void set_prefer_tiles_k3(bool v) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_k3_tiles = v;
}

bool prefer_tiles_k2() {
    std::lock_guard<std::mutex> g(g_tune_mu);
    return g_k2_tiles;
}

void set_prefer_tiles_k2(bool v) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_k2_tiles = v;
}

int line_z_for(int k) {
    if (k < kLinesMinK || k > kLinesMaxK) return 0;
    std::lock_guard<std::mutex> g(g_tune_mu);
    return g_line_z[k] ? g_line_z[k] : line_z_default(k);
}

int set_line_z(int k, int z) {
    if (k < kLinesMinK || k > kLinesMaxK || (z != 0 && !line_z_valid(k, z))) return MSA_EINVAL;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_line_z[k] = z;
    return MSA_OK;
}

bool prefer_tiles_lines(int k) {
    if (k < kLinesMinK || k > kLinesMaxK) return true;
    std::lock_guard<std::mutex> g(g_tune_mu);
    return g_lines_tiles[k];
}

void set_prefer_tiles_lines(int k, bool v) {
    if (k < kLinesMinK || k > kLinesMaxK) return;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_lines_tiles[k] = v;
}

bool prefer_stream(int k) {
    if (k < kStreamMinK || k > kStreamMaxK) return false;
    std::lock_guard<std::mutex> g(g_tune_mu);
    return g_stream[k];
}

void set_prefer_stream(int k, bool v) {
    if (k < kStreamMinK || k > kStreamMaxK) return;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_stream[k] = v;
}

void reset_prefer_stream(int k) { set_prefer_stream(k, stream_default(k)); }

bool stream_fits(int k, const int32_t *lens) {
    if (k < kStreamMinK || k > kStreamMaxK) return false;
    // tile and super-block indices stay within 31 bits
    int64_t tiles = 1;
    for (int i = 0; i < k - 1; ++i) tiles *= ((int64_t)lens[i] + 1 + line_ext(k, i) - 1) / line_ext(k, i);
    return tiles < (1LL << 31);
}

int choose_kernel(int k, const int32_t *lens, int A, int requested, bool allow_stream) {
    if (requested == kKernelTiles) return kKernelTiles;
    if (requested == kKernelStream && k >= kStreamMinK && k <= kStreamMaxK) return kKernelStream;
    if (k >= kLinesMinK && k <= kLinesMaxK &&
        (requested == kKernelLines || requested == kKernelStream || (requested == kKernelAuto && !prefer_tiles_lines(k)))) {
        // at k = 6 only the whole-column form (last axis of at most kWideZ) beats the line kernel
        if (requested == kKernelAuto && allow_stream && prefer_stream(k) && stream_fits(k, lens) &&
            (k != 6 || lens[k - 1] + 1 <= kWideZ))
            return kKernelStream;
        return kKernelLines;
    }
    if (k == 2 && (requested == kKernelBand2 || (requested == kKernelAuto && !prefer_tiles_k2()))) return kKernelBand2;
    if (col3_fits(k, lens, A) && (requested == kKernelCol3 || !prefer_tiles_k3())) return kKernelCol3;
    return kKernelTiles;
}

void tile_extents(int k, const int32_t *lens, int kernel, int edge, int32_t *E) {
    if (kernel == kKernelCol3) {
        E[0] = c3::WR;
        E[1] = 32;
        E[2] = lens[2] + 1;
        return;
    }
    if (kernel == kKernelBand2) {  // bands of 32 lanes x kBand2RowsPerLane rows spanning every column
        E[0] = 32 * kBand2RowsPerLane;
        E[1] = lens[1] + 1;
        return;
    }
    if (kernel == kKernelStream) {  // 32-line blocks spanning the whole last axis
        for (int i = 0; i < k - 1; ++i) E[i] = line_ext(k, i);
        E[k - 1] = lens[k - 1] + 1;
        return;
    }
    if (kernel == kKernelLines) {  // 32-line blocks; the last axis cut into equal segments of at most `edge`
        for (int i = 0; i < k - 1; ++i) E[i] = line_ext(k, i);
        const int rho = lens[k - 1] + 1;
        const int nseg = (rho + edge - 1) / edge;
        E[k - 1] = (rho + nseg - 1) / nseg;
        return;
    }
    for (int i = 0; i < k; ++i) E[i] = tile_ext(k, edge, i);
}

void wave_sizes(int k, const int32_t *grid, std::vector<int64_t> &out) {
    // Number of grid points with coordinate sum w: the product of the axes'
    // generating polynomials (1 + z + ... + z^(G_i - 1)), coefficient by coefficient.
    std::vector<int64_t> cur(1, 1);
    for (int i = 0; i < k; ++i) {
        const int g = std::max(grid[i], 1);
        std::vector<int64_t> nxt(cur.size() + g - 1, 0);
        for (size_t w = 0; w < cur.size(); ++w)
            for (int v = 0; v < g; ++v) nxt[w + v] += cur[w];
        cur.swap(nxt);
    }
    out = cur;
}

static int64_t round_up64(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

static std::atomic<uint64_t> g_wave_shuffle_seed{0};
void set_wave_shuffle_seed(uint64_t seed) { g_wave_shuffle_seed = seed; }
uint64_t wave_shuffle_seed() { return g_wave_shuffle_seed; }

// SplitMix64 (Steele, Lea and Flood's splittable generator, Vigna's constants).
static uint64_t splitmix64(uint64_t &state) {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Test hook: permute the tickets inside every wave (Fisher-Yates, seeded). Every
// producer of a tile lies in an earlier wave, so the order stays topological.
static void shuffle_within_waves(HostPlan &hp) {
    uint64_t state = wave_shuffle_seed();
    if (state == 0) return;
    for (size_t w = 0; w + 1 < hp.wave_start.size(); ++w) {
        const int64_t b = hp.wave_start[w], e = hp.wave_start[w + 1];
        for (int64_t i = e - 1; i > b; --i) {
            const int64_t j = b + (int64_t)(splitmix64(state) % (uint64_t)(i - b + 1));
            std::swap(hp.order[(size_t)i], hp.order[(size_t)j]);
        }
    }
}

bool score_and_traceback_layout(HostPlan &hp) {
    const int k = hp.k;
    // score scratch: full tensor, last axis padded to 4 elements (16-byte rows)
    int64_t s = 1;
    for (int i = k - 1; i >= 0; --i) {
        hp.qstride[i] = s;
        s *= (i == k - 1) ? round_up64(hp.rho[i], 4) : hp.rho[i];
    }
    hp.qelems = s;
    // traceback tensor (row-major view, the layout msa_plan_read_tb returns):
    // last axis padded to 16-byte rows
    s = 1;
    for (int i = k - 1; i >= 0; --i) {
        hp.tbstride[i] = s;
        s *= (i == k - 1) ? round_up64(hp.rho[i], kTbRowAlign) : hp.rho[i];
    }
    hp.tbbytes = s;
    hp.tb_layout = 0;
    hp.tb_dev_bytes = hp.tbbytes;
    if (hp.kernel == kKernelTiles && k >= kTileMajorMinK) {
        // tile-major scratch and traceback on the device: tile t's cells form one
        // block of prod(E_i) entries in local row-major order (edge tiles padded)
        int64_t vol = 1;
        for (int i = k - 1; i >= 0; --i) {
            hp.lst[i] = (int32_t)vol;
            vol *= hp.E[i];
        }
        if (hp.ntiles * vol >= (1LL << 31)) return false;
        hp.qelems = hp.ntiles * vol;
        hp.tb_layout = 2;
        hp.tb_block = (int32_t)vol;
        hp.tb_dev_bytes = hp.ntiles * vol;
    }
    if (hp.kernel == kKernelLines || hp.kernel == kKernelStream) {
        // traceback: tile t's block holds (E_{k-1} + skew_max) rows of 32 bytes
        // (the streamed kernel: rounded up to whole blocks), cell (c, z) at
        // (z + sum c_i) * 32 + lane(c); faces: 32 lines of lzq words (the streamed
        // kernel: lzq (value, tag) entries of two words)
        const int z = hp.E[k - 1];
        const bool stream = hp.kernel == kKernelStream;
        const int rows = z + line_skew_max(k);
        const int ub = stream_block(k);
        hp.tb_block = (stream ? (rows + ub - 1) / ub * ub : rows) * 32;
        hp.lst[k - 1] = 32;
        for (int i = 0; i < k - 1; ++i) hp.lst[i] = 32 + line_lstride(k, i);
        // streamed: lzq times per face line (the whole sweep of a super-block),
        // stream_face_lines(k) lines per super-block
        hp.lzq = stream ? (z + stream_skew_max(k) + ub - 1) / ub * ub : (z + 3) / 4 * 4;
        hp.qelems = stream ? hp.nunits * stream_face_lines(k) * hp.lzq * 2 : hp.ntiles * 32 * hp.lzq;
        hp.tb_layout = 3;
        hp.tb_dev_bytes = hp.ntiles * hp.tb_block;
        if (hp.qelems >= (1LL << 38) || hp.tb_dev_bytes >= (1LL << 40)) return false;
    }
    return true;
}

int plan_shape(int k, const int32_t *lens, int A, int kernel_choice, HostPlan &hp, std::string &err, int edge,
               bool allow_stream) {
    char buf[256];
    if (k < 2 || k > MSA_MAX_K) {
        snprintf(buf, sizeof buf, "k=%d outside [2,%d]", k, MSA_MAX_K);
        err = buf;
        return MSA_EINVAL;
    }
    if (!lens) {
        err = "lens is NULL";
        return MSA_EINVAL;
    }
    if (A < 1 || A > MSA_MAX_ALPHABET) {
        snprintf(buf, sizeof buf, "alphabet size %d outside [1,%d]", A, MSA_MAX_ALPHABET);
        err = buf;
        return MSA_EINVAL;
    }
    hp = HostPlan();
    hp.k = k;
    hp.A = A;
    hp.kernel = choose_kernel(k, lens, A, kernel_choice, allow_stream);
    long double cells = 1;
    int64_t len_sum = 0, w_corner = 0, pair_min = 0;
    for (int i = 0; i < k; ++i) {
        if (lens[i] < 0) {
            snprintf(buf, sizeof buf, "lens[%d]=%d is negative", i, lens[i]);
            err = buf;
            return MSA_EINVAL;
        }
        hp.lens[i] = lens[i];
        hp.rho[i] = lens[i] + 1;
        cells *= (long double)hp.rho[i];
        len_sum += lens[i];
        w_corner += (int64_t)lens[i] << i;
        for (int j = i + 1; j < k; ++j) pair_min += std::min(lens[i], lens[j]);
    }
    if (cells > (long double)(1LL << 38) || len_sum >= (1 << 24) || w_corner >= (1 << 28)) {
        snprintf(buf, sizeof buf, "tensor of %.3Lg cells is beyond the supported size", cells);
        err = buf;
        return MSA_ETOOBIG;
    }
    if (hp.kernel == kKernelStream && !stream_fits(k, lens)) {
        snprintf(buf, sizeof buf, "the streamed line kernel's tile indices exceed 31 bits for these lengths");
        err = buf;
        return MSA_ETOOBIG;
    }
    hp.cells = (int64_t)cells;
    hp.len_sum = (int32_t)len_sum;
    hp.w_corner = (int32_t)w_corner;
    hp.pair_min_sum = (int32_t)std::min<int64_t>(pair_min, (1LL << 30));

    if (hp.kernel == kKernelTiles) {
        hp.edge = edge < 0 ? tile_edge_for(k) : edge;
        if (!tile_edge_valid(k, hp.edge)) {
            snprintf(buf, sizeof buf, "tile edge %d is not compiled for k=%d", hp.edge, k);
            err = buf;
            return MSA_EINVAL;
        }
    }
    if (hp.kernel == kKernelLines) {
        hp.edge = edge < 0 ? line_z_for(k) : edge;
        if (!line_z_valid(k, hp.edge)) {
            snprintf(buf, sizeof buf, "line segment %d is not compiled for k=%d", hp.edge, k);
            err = buf;
            return MSA_EINVAL;
        }
    }
    tile_extents(k, lens, hp.kernel, hp.edge, hp.E);
    int64_t nt = 1;
    for (int i = k - 1; i >= 0; --i) {
        hp.G[i] = (hp.rho[i] + hp.E[i] - 1) / hp.E[i];
        hp.gstride[i] = nt;
        nt *= hp.G[i];
    }
    if (nt >= (1LL << 32)) {
        err = "too many tiles";
        return MSA_ETOOBIG;
    }
    hp.ntiles = nt;
    // tickets: the tiles, or for the streamed line kernel the super-blocks of
    // stream_wg line blocks (one CTA each)
    int64_t nu = 1;
    for (int i = k - 1; i >= 0; --i) {
        hp.SG[i] = hp.kernel == kKernelStream && i < k - 1 ? (hp.G[i] + stream_wg(k, i) - 1) / stream_wg(k, i) : hp.G[i];
        hp.sgstride[i] = nu;
        nu *= hp.SG[i];
    }
    hp.nunits = nu;
    int gsum = 0;
    for (int i = 0; i < k; ++i) gsum += hp.SG[i];
    hp.waves = gsum - k + 1;

    if (!score_and_traceback_layout(hp)) {
        err = "score scratch beyond 32-bit element offsets";
        return MSA_ETOOBIG;
    }
    if (hp.kernel == kKernelBand2) {
        // scores: only each band's last row, the face the band below reads, as
        // (value, tag) entries of two words
        hp.face0_stride = 2 * round_up64(hp.rho[1], 32);
        hp.qelems = hp.ntiles * hp.face0_stride;
    }

    if (hp.kernel == kKernelCol3) {  // faces between columns
        const int rho2 = hp.rho[2];
        hp.face0_rows = c3::face0_rows(rho2);
        hp.face1_rows = c3::face1_rows(rho2);
        hp.face0_stride = (int64_t)hp.face0_rows * c3::F0W;
        hp.face1_stride = (int64_t)hp.face1_rows * c3::F1W;
        hp.qelems = nt * hp.face0_stride;
        hp.aux_elems = nt * hp.face1_stride;
        hp.tb_layout = 1;
        hp.tb_dev_bytes = nt * c3::tb_col_bytes(rho2);
    }
    return MSA_OK;
}

int make_plan(int k, const int32_t *lens, int A, int kernel_choice, HostPlan &hp, std::string &err, int edge,
              bool allow_stream) {
    const int rc = plan_shape(k, lens, A, kernel_choice, hp, err, edge, allow_stream);
    if (rc) return rc;
    const int64_t nt = hp.nunits;
    if (hp.kernel == kKernelCol3) {
        // the column order: a column (a, b) can start about a*(WR + U) + b*(32 + U)
        // CTA-time steps after the first, so tickets follow that estimate (every
        // producer gets a smaller ticket)
        std::vector<std::pair<int64_t, int64_t>> key(nt);
        for (int64_t t = 0; t < nt; ++t) {
            const int64_t a = t / hp.G[1], b = t % hp.G[1];
            key[t] = {a * (c3::WR + c3::U) + b * (32 + c3::U), t};
        }
        std::sort(key.begin(), key.end());
        hp.order.resize(nt);
        for (int64_t t = 0; t < nt; ++t) hp.order[t] = (uint64_t)key[t].second;
        // the key is (WR + U) (a + b): waves of equal a + b, contiguous in the order
        static_assert(c3::WR == 32, "column waves by a + b");
        hp.wave_start.assign((size_t)(hp.G[0] + hp.G[1]), 0);
        for (int64_t t = 0; t < nt; ++t) hp.wave_start[(size_t)(t / hp.G[1] + t % hp.G[1] + 1)]++;
        for (size_t w = 1; w < hp.wave_start.size(); ++w) hp.wave_start[w] += hp.wave_start[w - 1];
        shuffle_within_waves(hp);
        return MSA_OK;
    }

    // ticket order: by wave, then by linear tile index (counting sort); the wave
    // of each tile follows its grid coordinates, stepped like an odometer (last
    // axis fastest) instead of decoded from the linear index
    std::vector<int64_t> cnt(hp.waves + 1, 0);
    std::vector<int32_t> wave_of(nt);
    {
        int c[MSA_MAX_K] = {};
        int w = 0;
        for (int64_t t = 0; t < nt; ++t) {
            wave_of[t] = w;
            cnt[w + 1]++;
            for (int i = k - 1; i >= 0; --i) {
                if (c[i] + 1 < hp.SG[i]) {
                    ++c[i];
                    ++w;
                    break;
                }
                w -= c[i];
                c[i] = 0;
            }
        }
    }
    for (int w = 0; w < hp.waves; ++w) cnt[w + 1] += cnt[w];
    hp.wave_start = cnt;
    hp.order.assign(nt, 0);
    for (int64_t t = 0; t < nt; ++t) hp.order[cnt[wave_of[t]]++] = (uint64_t)t;
    shuffle_within_waves(hp);
    return MSA_OK;
}

}  // namespace msadp
