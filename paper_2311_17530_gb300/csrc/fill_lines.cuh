// Line-sweep fill for k >= 4: the recurrence of section 2 (each cell the max over
// its 2^k - 1 predecessors plus the sum-of-pairs score of the move) organised as
// lines along the last axis instead of independent cells.
//
// Work unit (tile): a block of 32 lines -- local coordinates c_0 .. c_{k-2} in a
// box of extents L_i over the first k - 1 axes (line_ext) -- times a segment of at
// most Z positions along the last axis (the sweep axis). Tiles are handed out in
// wave order by an atomic ticket (waves of equal tile-index sum, section 3) and
// wait for their k face predecessors' completion flags, as the generic tile
// kernel does. One warp fills one tile; lane l owns line c(l) and at step t
// computes position z = t - sum_i c_i (a skew by the line's index sum), so every
// predecessor line c - e_m' (m' a nonempty subset of the line axes) computed
// position z at step t - |m'|.
//
// For a cell x = (line c, position z) and a move m = m' (+ the sweep axis s):
//   m' alone      : Q(c - e_m', z)     + P(m')          P = pair sum of m' (the
//                                                       pairs among line axes,
//                                                       constant along the line)
//   m' + s        : Q(c - e_m', z - 1) + P(m') + T(m', z)   T = pairs of m' with s
//   s alone       : Q(c, z - 1)                        (no pair)
// The candidate of m' + s is the previous step's candidate of m' plus T(m', z),
// so each line keeps the 2^(k-1) - 1 candidates of the previous position in
// registers ("carried"), P is formed once per tile, and T from k - 1 pair-table
// lookups per cell. Each step therefore loads one value per line-axis subset
// m' (2^(k-1) - 1 shared-memory loads), not one per move.
//
// Scores are packed keys (internal.h): one integer max gives the best value and
// the lowest move mask among ties; the mask is the traceback byte.
//
// Shared memory per warp: the halo'd line box (extents L_i + 1, the extra index
// 0 holding the lower neighbours' lines) times positions 0 .. Z (position 0 holds
// z = -1 from the tile below along the sweep axis), with per-axis strides chosen
// so that the 32 lanes of every step's load of a given m' fall in 32 different
// banks (lane c reads word sum_i c_i (A_i - 1) + const mod 32, a bijection of
// the box); the pair tables of the sweep axis against each line axis for the
// tile; and the neighbour tile of every subset of the line axes.
//
// Global memory per tile (tile-major): the traceback bytes of cell (c, z) at
// (z + sum c_i) * 32 + l(c) -- each step's 32 bytes are one contiguous store --
// and the faces the successors read: for each line with some c_i = L_i - 1 all
// of its positions, for the other lines the last position, line-major (line l
// at l * ZQ + z), written from shared memory after the sweep.
#pragma once

#include "device_common.cuh"

namespace msadp {

// ---------------------------------------------------------------------------
// Geometry (compile-time per k and the longest segment Z).

// The line kernel is compiled for k = 4, 5, 6; at k = 7, 8 a lane would carry
// 63 or 127 candidates and as many pair sums, more than its registers, and the
// generic tile kernel runs instead. Block extents, segment candidates, lane
// strides and the skew bound are in internal.h (shared with the planner).
// Shared-memory stride (words) of line axis i in the halo'd line box. Found by
// exhaustive search for each (k, Z): every stride at least the size of the axes
// nested inside it (innermost at least Z + 1 positions), the 32 lines' word
// offsets sum_i c_i (A_i - 1) distinct mod 32, and the smallest footprint
// (within 7 % of the unpadded box).
__host__ __device__ constexpr int line_stride(int K, int Z, int i) {
    constexpr int k4z8[] = {45, 9, 136}, k4z16[] = {17, 52, 261}, k4z32[] = {34, 103, 521};
    constexpr int k5z16[] = {17, 256, 777, 51}, k5z32[] = {34, 103, 1553, 309};
    constexpr int k6z16[] = {17, 51, 153, 460, 1381}, k6z25[] = {26, 79, 237, 713, 2161};
    return K == 4 ? (Z == 8 ? k4z8[i] : Z == 16 ? k4z16[i] : k4z32[i])
         : K == 5 ? (Z == 16 ? k5z16[i] : k5z32[i])
                  : (Z == 16 ? k6z16[i] : k6z25[i]);
}
// word offset of the predecessor line c - e_m' relative to line c
template <int K, int Z>
__host__ __device__ constexpr int move_line_off(int m) {
    int s = 0;
    for (int i = 0; i < K - 1; ++i)
        if ((m >> i) & 1) s += line_stride(K, Z, i);
    return s;
}
__host__ __device__ constexpr int line_halo_lines(int K) {  // lines of the halo'd box
    int n = 1;
    for (int i = 0; i < K - 1; ++i) n *= line_ext(K, i) + 1;
    return n;
}
// Words of the halo'd line box: the last word any (line, position) addresses, plus
// slack for the 4-word reads of the face write-back.
template <int K, int Z>
__host__ __device__ constexpr int line_v_words() {
    int top = Z + 1;
    for (int i = 0; i < K - 1; ++i) top += line_ext(K, i) * line_stride(K, Z, i);
    return round_up(top + 4, 4);
}
// Pair-table row stride: at least Z + skew_max (a lane reads its row at positions
// -skew_max .. Z + skew_max - 1, unclamped, in the sweep), and congruent to
// skew_max + 1 mod 32, so that lanes reading row c_i at position t - sum c hit
// distinct banks unless they read the same word.
template <int K, int Z>
__host__ __device__ constexpr int line_pt_stride() {
    int s = Z + line_skew_max(K);
    while (s % 32 != (line_skew_max(K) + 1) % 32) ++s;
    return s;
}
template <int K, int Z>
__host__ __device__ constexpr int line_pt_words() {
    int n = 0;
    for (int i = 0; i < K - 1; ++i) n += line_ext(K, i) * line_pt_stride<K, Z>();
    return n;
}
template <int K, int Z>
__host__ __device__ constexpr int line_warp_bytes() {
    return line_v_words<K, Z>() * 4 + line_pt_words<K, Z>() * 4 + (1 << (K - 1)) * 4;
}
template <int K>
__host__ __device__ constexpr int line_cta_fixed_bytes() {
    return round_up(line_halo_lines(K) * 4, 16);
}
// Warps (tiles) per CTA: the count that keeps the most warps resident per SM
// within shared memory (228 KB per SM, 227 KB per CTA, 1 KB reserved per CTA; at
// most 48 warps per SM), preferring fewer per CTA.
constexpr int kLinesSmemPerSm = 228 * 1024, kLinesSmemPerCta = 227 * 1024;
template <int K, int Z>
__host__ __device__ constexpr int line_best_warps() {
    int best = 1, best_res = 0;
    for (int w = 1; w <= 16; ++w) {
        const int bytes = line_cta_fixed_bytes<K>() + w * line_warp_bytes<K, Z>();
        if (bytes > kLinesSmemPerCta) break;
        int ctas = kLinesSmemPerSm / (bytes + 1024);
        if (ctas > 32) ctas = 32;
        const int resident = ctas * w > 48 ? 48 : ctas * w;
        if (resident > best_res) {
            best_res = resident;
            best = w;
        }
    }
    return best;
}
template <int K, int Z>
__host__ __device__ constexpr int line_smem_bytes() {
    return line_cta_fixed_bytes<K>() + line_best_warps<K, Z>() * line_warp_bytes<K, Z>();
}

// ---------------------------------------------------------------------------

template <int K, int Z>
__global__ void __launch_bounds__(line_best_warps<K, Z>() * 32) fill_lines_kernel(const LaunchDesc L) {
    constexpr int NA = K - 1;               // line axes
    constexpr int M = (1 << NA) - 1;        // nonempty subsets of the line axes
    constexpr int NHL = line_halo_lines(K); // lines of the halo'd box
    constexpr int NH = NHL - 32;            // halo lines (some index 0)
    constexpr int SMAX = line_skew_max(K);
    constexpr int NQ = (Z + 3) / 4;         // 4-position groups of a segment
    constexpr int VW = line_v_words<K, Z>();
    constexpr int ZS = line_pt_stride<K, Z>();
    constexpr int MASKB = (1 << K) - 1;
    constexpr int NW = line_best_warps<K, Z>();
    static_assert(line_cta_fixed_bytes<K>() >= 4 * SMAX, "sweep reads below the first box stay in shared memory");

    extern __shared__ __align__(16) unsigned char smem[];
    // per CTA: one entry per halo'd line, halo lines first, then the 32 lines of
    // the block: bits 0..13 its base word, 14..18 the lane of the producer line
    // that holds it, 19.. the axes at index 0 (which lower neighbour holds it)
    uint32_t *htab = reinterpret_cast<uint32_t *>(smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int32_t *V = reinterpret_cast<int32_t *>(smem + line_cta_fixed_bytes<K>() + warp * line_warp_bytes<K, Z>());
    int32_t *PT = V + VW;
    int32_t *nb = PT + line_pt_words<K, Z>();

    // halo'd line table (once per CTA), halo lines first in index order, then the
    // block's own lines: a halo'd index j (digits h_i in [0, L_i], axis 0 most
    // significant) has interior_below(j) indices below it with every digit >= 1
    for (int j = tid; j < NHL; j += NW * 32) {
        int rem = j, off = 0, lp = 0;
        uint32_t S = 0;
        int h[NA];
#pragma unroll
        for (int i = NA - 1; i >= 0; --i) {
            h[i] = rem % (line_ext(K, i) + 1);
            rem /= line_ext(K, i) + 1;
            off += h[i] * line_stride(K, Z, i);
            lp += (h[i] == 0 ? line_ext(K, i) - 1 : h[i] - 1) * line_lstride(K, i);
            if (h[i] == 0) S |= 1u << i;
        }
        int below = 0;
        bool prefix = true;
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            if (prefix && h[i] > 1) below += (h[i] - 1) * line_lstride(K, i);  // digits 1 .. h_i - 1 here
            prefix = prefix && h[i] >= 1;
        }
        htab[S != 0 ? j - below : NH + below] = (uint32_t)off | ((uint32_t)lp << 14) | (S << 19);
    }
    __syncthreads();

    // this lane's line: local coordinates, halo'd base word, skew
    int cl[NA];
    int vbase = 0, skew = 0;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
        cl[i] = (lane / line_lstride(K, i)) % line_ext(K, i);
        vbase += (cl[i] + 1) * line_stride(K, Z, i);
        skew += cl[i];
    }

    // The next ticket is taken while the current tile runs, so its atomic (an L2
    // round trip) is off the tile's path; a warp holding an unstarted ticket only
    // delays tiles with later tickets, never one it waits for.
    int tnext = 0;
    if (lane == 0) tnext = atomicAdd(L.ticket, 1);
    int cached_prob = -1;
    bool cached_live = false;
    while (true) {
        const int t = __shfl_sync(kFull, tnext, 0);
        if ((int64_t)t >= L.ntickets) break;
        if (ld_volatile(L.err) != 0) break;
        if (lane == 0) tnext = atomicAdd(L.ticket, 1);
        const uint64_t ent = L.order[t];
        const int pidx = (int)(ent >> 32);
        const ProblemDesc &P = L.probs[pidx];
        const int64_t lin = (int64_t)(uint32_t)ent;

        int tco[K], o[K];
        {
            // tile coordinates (32-bit: a problem has fewer than 2^31 tiles)
            unsigned rem = (unsigned)lin;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const unsigned gs = (unsigned)P.gstride[j];
                tco[j] = (int)(rem / gs);
                rem -= (unsigned)tco[j] * gs;
                o[j] = tco[j] * P.E[j];
            }
        }
        const int64_t tile_base = P.tile_base;
        // Everything that does not depend on the face predecessors comes first, so
        // that its loads overlap the wait: problem fields, the neighbour table, the
        // sweep axis's pair tables and this line's pair sums.
        // the encode step's verdict on the problem (fixed before the fill starts)
        if (pidx != cached_prob) {
            cached_prob = pidx;
            cached_live = ld_volatile(&P.istat->status) == 0;
        }
        const bool live = cached_live;
        const int A = P.A;
        const int32_t *__restrict__ tab = P.tab;
        const uint8_t *__restrict__ codes = P.codes;
        const int Ez = P.E[NA];                      // segment length of full tiles
        const int z0 = o[NA];
        const int Zt = min(Ez, P.rho[NA] - z0);      // this tile's positions
        const int ZQ = P.lzq;                        // words per line in a face block
        const int64_t QB = 32 * (int64_t)ZQ;
        int Sp[M + 1];
        if (live) {
            // neighbour tile of each subset S of the line axes (-1: below the origin)
            for (int S = lane; S <= M; S += 32) {
                int64_t n = lin;
                bool in = true;
#pragma unroll
                for (int i = 0; i < NA; ++i)
                    if ((S >> i) & 1) {
                        in = in && tco[i] > 0;
                        n -= P.gstride[i];
                    }
                nb[S] = in ? (int)n : -1;
            }
            // Pair tables of the sweep axis, PT[i][a][z] = tab(code_i(o_i + a), code_s(z0 + z)),
            // and this line's pair sums over subsets of the line axes (constant
            // along the line). All residue codes are loaded first, then all table
            // entries, so the set-up costs two dependent round trips.
            constexpr int NR = (Z + 31) / 32;  // positions per lane
            constexpr int NROW = [] {
                int n = 0;
                for (int i = 0; i < K - 1; ++i) n += line_ext(K, i);
                return n;
            }();
            int cz[NR], ca[NROW], cd[NA];
            {
                const int lens = P.len[NA], cofs = P.cofs[NA];
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int x = z0 + lane + 32 * r;
                    cz[r] = (x >= 1 && x <= lens) ? codes[cofs + x - 1] : 0;
                }
                int row = 0;
#pragma unroll
                for (int i = 0; i < NA; ++i) {
                    const int len = P.len[i], cof = P.cofs[i];
#pragma unroll
                    for (int a = 0; a < line_ext(K, i); ++a) {
                        const int x = o[i] + a;
                        ca[row++] = (x >= 1 && x <= len) ? codes[cof + x - 1] : 0;
                    }
                    const int x = o[i] + cl[i];
                    cd[i] = (x >= 1 && x <= len) ? codes[cof + x - 1] : 0;
                }
            }
            int pt[NROW][NR];
#pragma unroll
            for (int row = 0; row < NROW; ++row)
#pragma unroll
                for (int r = 0; r < NR; ++r) pt[row][r] = __ldg(tab + ca[row] * A + cz[r]);
            {
                int row = 0, pb = 0;
#pragma unroll
                for (int i = 0; i < NA; ++i) {
#pragma unroll
                    for (int a = 0; a < line_ext(K, i); ++a, ++row)
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            const int z = lane + 32 * r;
                            if (z < Zt) PT[pb + a * ZS + z] = pt[row][r];
                        }
                    pb += line_ext(K, i) * ZS;
                }
            }
            Sp[0] = 0;
#pragma unroll
            for (int h = 0; h < NA; ++h) {
                // R[r] = sum over l in r of pair(l, h), r a subset of the axes below h
                int R[1 << (NA - 1)];
                R[0] = 0;
#pragma unroll
                for (int r = 1; r < (1 << h); ++r) R[r] = R[r & (r - 1)] + __ldg(tab + cd[lowbit_c(r)] * A + cd[h]);
#pragma unroll
                for (int r = 0; r < (1 << h); ++r) Sp[r | (1 << h)] = Sp[r] + R[r];
            }
        }
        __syncwarp();  // nb and PT are read by every lane below

        // face predecessors (one lane per axis)
        bool ok = true;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (lane == j && tco[j] > 0) ok = wait_at_least(&L.done[tile_base + lin - P.gstride[j]], 1, L.err, L.spin_ns);
        if (!__all_sync(kFull, ok)) {
            if (lane == 0) atomicCAS(L.err, 0, MSA_ETIMEOUT);
            break;
        }
        // The acquiring lanes' loads precede every lane's loads below: the warp
        // barrier orders them (no full fence needed).
        __syncwarp();

        if (live) {
            const int32_t *__restrict__ Qg = P.Q;

            // Halo: the halo lines' positions 0 .. Zt - 1 (4 at a time), then every
            // halo'd line's position -1 from the tile below along the sweep axis.
            // Loads bypass L1 (other SMs wrote them) and are issued in batches.
            {
                // position -1 of every halo'd line from the tile below along the sweep axis
                constexpr int NZF = (NHL + 31) / 32;
                const bool below = tco[NA] > 0;
                const int64_t gsz = P.gstride[NA];
                int zf[NZF];
#pragma unroll
                for (int u = 0; u < NZF; ++u) {
                    const int j = lane + 32 * u;
                    zf[u] = kNeg;
                    if (j < NHL) {
                        const uint32_t e = htab[j];
                        const int src = nb[e >> 19];
                        if (below && src >= 0) zf[u] = __ldcg(Qg + (src - gsz) * QB + (int)((e >> 14) & 31) * ZQ + (Ez - 1));
                    }
                }
                // loads in flight per lane: two batches at k = 6 (registers, not shared
                // memory, would bound the warps of the shorter segment at 24)
                constexpr int HB = K >= 6 && Z > 16 ? 24 : 16;
                for (int i0 = 0; i0 < NH * NQ; i0 += 32 * HB) {
                    int4 val[HB];
                    int dst[HB];
#pragma unroll
                    for (int u = 0; u < HB; ++u) {
                        const int it = i0 + 32 * u + lane;
                        const int j = it / NQ, q = it - j * NQ;
                        dst[u] = -1;
                        val[u] = make_int4(kNeg, kNeg, kNeg, kNeg);
                        if (it < NH * NQ && 4 * q < Zt) {
                            const uint32_t e = htab[j];
                            const int src = nb[e >> 19];
                            dst[u] = (int)(e & 0x3FFF) + 1 + 4 * q;
                            if (src >= 0)
                                val[u] = __ldcg(reinterpret_cast<const int4 *>(Qg + src * QB + (int)((e >> 14) & 31) * ZQ +
                                                                               4 * q));
                        }
                    }
#pragma unroll
                    for (int u = 0; u < HB; ++u)
                        if (dst[u] >= 0) {
                            const int it = i0 + 32 * u + lane;
                            const int n = Zt - 4 * (it - (it / NQ) * NQ);  // positions left in the segment
                            V[dst[u]] = val[u].x;
                            if (n > 1) V[dst[u] + 1] = val[u].y;
                            if (n > 2) V[dst[u] + 2] = val[u].z;
                            if (n > 3) V[dst[u] + 3] = val[u].w;
                        }
                }
#pragma unroll
                for (int u = 0; u < NZF; ++u) {
                    const int j = lane + 32 * u;
                    if (j < NHL) V[htab[j] & 0x3FFF] = zf[u];
                }
            }
            __syncwarp();

            // The sweep. Every lane reads its own skewed position, in range or not,
            // so the 32 loads of a step stay in 32 banks: at z = -1 word 0 holds the
            // position below; the words read at z < -1 (up to skew_max - 1 words
            // before the box, inside the CTA's shared memory) and at z >= Zt feed
            // only candidates that are overwritten or never stored, and the
            // traceback byte such a lane writes is a padding byte of the tile.
            const bool origin_lane = lin == 0 && lane == 0;
            int Wl = (z0 - skew) * (1 << NA);  // W(x) = Wl + ts * 2^NA at step ts
#pragma unroll
            for (int i = 0; i < NA; ++i) Wl += (o[i] + cl[i]) << i;
            int ptoff[NA];  // row c_i of the pair table of axis i
            {
                int pb = 0;
#pragma unroll
                for (int i = 0; i < NA; ++i) {
                    ptoff[i] = pb + cl[i] * ZS;
                    pb += line_ext(K, i) * ZS;
                }
            }
            int carry[M + 1];
            int vself = V[vbase];
#pragma unroll
            for (int m = 1; m <= M; ++m) carry[m] = V[vbase - move_line_off<K, Z>(m)] + Sp[m];
            uint8_t *tbblk = P.tb + lin * (int64_t)P.tb_block + lane;
            const int nsteps = Zt + SMAX;
            for (int ts = 0; ts < nsteps; ++ts) {
                const int z = ts - skew;
                const bool act = (unsigned)z < (unsigned)Zt;
                const int zz = z + 1;  // word offset of position z
                const int32_t *vp = V + vbase + zz;
                int p[NA];
#pragma unroll
                for (int i = 0; i < NA; ++i) p[i] = PT[ptoff[i] + z];
                int T[M + 1];
                T[0] = 0;
#pragma unroll
                for (int m = 1; m <= M; ++m) T[m] = (m & (m - 1)) ? T[m & (m - 1)] + p[lowbit_c(m)] : p[lowbit_c(m)];
                int acc0 = vself, acc1 = kNeg;
#pragma unroll
                for (int m = 1; m <= M; ++m) {
                    const int cm = vp[-move_line_off<K, Z>(m)] + Sp[m];
                    const int cb = carry[m] + T[m];
                    if (m & 1)
                        acc0 = __vimax3_s32(acc0, cm, cb);
                    else
                        acc1 = __vimax3_s32(acc1, cm, cb);
                    carry[m] = cm;
                }
                const int acc = max(acc0, acc1);
                int tm = (Wl + ts * (1 << NA) - acc) & MASKB;
                int val = acc + tm;
                if (origin_lane && ts == 0) {  // H(0) = 0: no move
                    val = 0;
                    tm = 0;
                }
                tbblk[ts * 32] = (uint8_t)tm;
                if (act) {
                    V[vbase + zz] = val;
                    vself = val;
                }
                __syncwarp();
            }

            // Faces for the successors (line-major), and the corner's key.
            int32_t *__restrict__ Qw = P.Q + lin * QB;
            for (int it = lane; it < 32 * NQ; it += 32) {
                const int ln = it / NQ, q = it - ln * NQ;
                if (4 * q >= Zt) continue;
                int lb = 0;
                bool face = false;
#pragma unroll
                for (int i = 0; i < NA; ++i) {
                    const int c = (ln / line_lstride(K, i)) % line_ext(K, i);
                    lb += (c + 1) * line_stride(K, Z, i);
                    face = face || c == line_ext(K, i) - 1;
                }
                if (!face && q != (Zt - 1) / 4) continue;
                const int32_t *s = V + lb + 1 + 4 * q;
                *reinterpret_cast<int4 *>(Qw + ln * ZQ + 4 * q) = make_int4(s[0], s[1], s[2], s[3]);
            }
            if (lane == 0) {
                bool corner = true;
                int lb = 0;
#pragma unroll
                for (int i = 0; i < NA; ++i) {
                    const int c = P.len[i] - o[i];
                    corner = corner && c >= 0 && c < line_ext(K, i);
                    lb += (c + 1) * line_stride(K, Z, i);
                }
                const int zc = P.len[NA] - z0;
                if (corner && zc >= 0 && zc < Zt) *P.qcorner = V[lb + 1 + zc];
            }
        }
        // Every lane's stores precede lane 0's release through the warp barrier;
        // the release store makes them visible with the flag.
        __syncwarp();
        if (lane == 0 && (int64_t)t != L.withhold) st_release(&L.done[tile_base + lin], 1);
    }
}

// Shared-memory attribute of fill_lines_kernel<K, Z>, set once per device (so
// that no launch inside a stream capture makes the call).
template <int K, int Z>
cudaError_t lines_attributes() {
    static DeviceOnce once;
    return once.run([] {
        return cudaFuncSetAttribute(fill_lines_kernel<K, Z>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    line_smem_bytes<K, Z>());
    });
}

template <int K, int Z>
cudaError_t launch_lines(const LaunchDesc &L, int grid, cudaStream_t s) {
    cudaError_t e = lines_attributes<K, Z>();
    if (e != cudaSuccess) return e;
    fill_lines_kernel<K, Z><<<grid, line_best_warps<K, Z>() * 32, line_smem_bytes<K, Z>(), s>>>(L);
    return cudaGetLastError();
}

template <int K, int Z>
int lines_ctas() {
    if (lines_attributes<K, Z>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fill_lines_kernel<K, Z>, line_best_warps<K, Z>() * 32,
                                                      line_smem_bytes<K, Z>()) != cudaSuccess)
        return 0;
    return n;
}

// Dispatch of one k over its compiled segment lengths (instantiated in fill_lines_k<k>.cu).
template <int K>
struct LinesK {
    static constexpr int Z0 = line_z_candidate(K, 0), Z1 = line_z_candidate(K, 1), Z2 = line_z_candidate(K, 2);
    static cudaError_t launch(int z, const LaunchDesc &L, int grid, cudaStream_t s) {
        if (z == Z0) return launch_lines<K, Z0>(L, grid, s);
        if (z == Z1) return launch_lines<K, Z1>(L, grid, s);
        if constexpr (Z2 > 0)
            if (z == Z2) return launch_lines<K, Z2>(L, grid, s);
        return cudaErrorInvalidValue;
    }
    static int ctas(int z) {
        if (z == Z0) return lines_ctas<K, Z0>();
        if (z == Z1) return lines_ctas<K, Z1>();
        if constexpr (Z2 > 0)
            if (z == Z2) return lines_ctas<K, Z2>();
        return 0;
    }
    static int warps(int z) {
        if (z == Z0) return line_best_warps<K, Z0>();
        if (z == Z1) return line_best_warps<K, Z1>();
        if constexpr (Z2 > 0)
            if (z == Z2) return line_best_warps<K, Z2>();
        return 0;
    }
};

}  // namespace msadp
