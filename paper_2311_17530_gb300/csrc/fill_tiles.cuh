// Generic persistent hyper-tile fill for any k in [2, 8].
//
// The k-dimensional tensor (section 2) is cut into hyper-tiles of compile-time
// extents E_i (the paper's partitions of size S, section 3, but without overlap:
// a tile reads a one-cell halo from its lower neighbours instead). Tiles are
// handed out by an atomic ticket in wave order (tiles of equal index sum: the
// partitions section 3 groups by their distance from the origin); a tile starts once
// its k face predecessors have published completion (bounded acquire waits),
// which also covers every edge and corner predecessor transitively (in a pruned
// fill, where left-out tiles wait for nothing, a live tile waits for every lower
// neighbour directly).
//
// One warp (two for a few large shapes, see tiles_group) fills one tile in
// shared memory: the halo comes from the score scratch in global memory (L2,
// bypassing L1), then the warp sweeps the tile's own intra-tile hyperplanes
// (cells of equal local index sum are independent), one cell per thread, each
// cell taking the max over its 2^k - 1 predecessors with the packed-key add-max
// (DPX viaddmax). Finally the tile's scores and traceback bytes are written back
// and the tile's flag is released.
#pragma once

#include "device_common.cuh"

namespace msadp {

// Shared memory: the intra-tile schedule (8 bytes per cell) and plane offsets
// for the CTA, then per warp the halo'd score tile, the traceback tile and the
// residue codes along each axis.
// Tile-major mode (k >= kTileMajorMinK) adds per CTA the halo table (one 8-byte
// entry per halo cell: its shared-memory offset, which lower neighbour tile
// holds it, and its offset in that tile's block) and the write-back table (the
// shared-memory offset of each interior cell), and per warp the element offsets
// of the neighbour tiles' blocks.
// Halo entries pack (shared-memory offset, neighbour mask, offset in the
// neighbour's block) into 4 bytes when the three fields fit, else 8.
__host__ __device__ constexpr int bits_for(int n) {  // bits to hold 0 .. n - 1
    int b = 0;
    while ((1 << b) < n) ++b;
    return b;
}
template <int K, int E>
__host__ __device__ constexpr bool tiles_halo_packed() {
    return bits_for(geo_volh(K, E)) + K + bits_for(geo_vol(K, E)) <= 32;
}
template <int K, int E>
__host__ __device__ constexpr int tiles_tm_cta_bytes() {
    return K >= kTileMajorMinK ? round_up((geo_cellsh(K, E) - geo_vol(K, E)) * (tiles_halo_packed<K, E>() ? 4 : 8), 16) +
                                     round_up(geo_vol(K, E) * 2, 16)
                               : 0;
}
// pair tables of a tile (k >= kTileMajorMinK): for each pair l < h of sequences,
// the scaled pair score of every local coordinate pair (a, b), E x E entries
template <int K, int E>
__host__ __device__ constexpr int tiles_ptab_ints() {
    return K >= kTileMajorMinK ? K * (K - 1) / 2 * E * E : 0;
}
template <int K, int E>
__host__ __device__ constexpr int tiles_warp_bytes() {
    return round_up(geo_volh(K, E) * 4, 16) + round_up(geo_vol(K, E), 16) + round_up(geo_codes(K, E), 16) +
           (K >= kTileMajorMinK ? (1 << K) * 4 + round_up(tiles_ptab_ints<K, E>() * 4, 16) : 0);
}
__host__ __device__ constexpr int pair_index(int K, int l, int h) { return l * K - l * (l + 1) / 2 + (h - l - 1); }
// Warps that fill one tile together: 2 where one warp's tile buffers leave too
// few warps resident (k = 6, E = 3: 16 KB of halo'd scores per tile; k = 4,
// E = 6 and k = 5, E = 4: 10-13 KB). Measured faster for these three.
template <int K, int E>
__host__ __device__ constexpr int tiles_group() {
    return (K == 6 && E == 3) || (K == 4 && E == 6) || (K == 5 && E == 4) ? 2 : 1;
}
// plane scratch: the schedule's running plane counts, later the halo-table scan
// (one count per warp plus the total: up to 32 warps where tiles take groups)
template <int K, int E>
__host__ __device__ constexpr int tiles_pcur_ints() {
    return round_up(tiles_group<K, E>() > 1 && geo_planes(K, E) < 33 ? 33 : geo_planes(K, E), 4);
}
template <int K, int E>
__host__ __device__ constexpr int tiles_cta_fixed_bytes() {
    return round_up(geo_vol(K, E) * 8, 16) + round_up(geo_planes(K, E) + 1, 4) * 4 + tiles_pcur_ints<K, E>() * 4 +
           tiles_tm_cta_bytes<K, E>();
}
// Warps per CTA: the count (a multiple of the group, up to TilesCfg::kMax) that
// keeps the most warps resident per SM within its shared memory (227 KB per CTA,
// 228 KB per SM, 1 KB reserved per CTA), preferring fewer warps per CTA on ties.
// tiles_warp_bytes is the buffer of one tile (one group).
constexpr int kSmemPerSm = 228 * 1024, kSmemPerCta = 227 * 1024, kSmemReservedPerCta = 1024;
template <int K, int E>
__host__ __device__ constexpr int tiles_best_warps(int kmax) {
    constexpr int G = tiles_group<K, E>();
    int best = G, best_res = 0;
    for (int w = G; w <= kmax; w += G) {
        const int bytes = tiles_cta_fixed_bytes<K, E>() + (w / G) * tiles_warp_bytes<K, E>();
        if (bytes > kSmemPerCta) break;
        int ctas = kSmemPerSm / (bytes + kSmemReservedPerCta);
        if (ctas > 32) ctas = 32;
        const int resident = ctas * w > 48 ? 48 : ctas * w;  // warps per SM are capped by the hardware
        if (resident > best_res) {
            best_res = resident;
            best = w;
        }
    }
    return best;
}
template <int K, int E>
struct TilesCfg {
    // warps per CTA considered (k = 6 and tile groups need more to fill an SM)
    static constexpr int kMax = K == 6 || tiles_group<K, E>() > 1 ? 24 : 8;
    static constexpr int kFit = (kSmemPerCta - tiles_cta_fixed_bytes<K, E>()) / tiles_warp_bytes<K, E>();
    static constexpr int WARPS = tiles_best_warps<K, E>(kMax);
    static_assert(kFit >= 1, "tile does not fit in shared memory");
    static_assert(WARPS % tiles_group<K, E>() == 0 && (tiles_group<K, E>() == 1 || WARPS / tiles_group<K, E>() <= 15),
                  "whole groups, one named barrier each");
    static_assert(K < kTileMajorMinK || tiles_pcur_ints<K, E>() >= WARPS + 1, "plane scratch holds the halo-table scan");
    static_assert(geo_volh(K, E) < 65536 && geo_vol(K, E) < 65536, "schedule entries hold 16-bit offsets");
    static_assert(E < (K <= 4 ? 256 : 16) && tile_ext(K, E, K - 1) < (K <= 4 ? 256 : 16),
                  "packed local coordinates");
};

template <int K, int E>
__host__ __device__ constexpr int tiles_smem_bytes() {
    return tiles_cta_fixed_bytes<K, E>() + TilesCfg<K, E>::WARPS / tiles_group<K, E>() * tiles_warp_bytes<K, E>();
}

// Barrier and vote of the G warps that fill one tile (named barrier 1 + group).
template <int G>
__device__ __forceinline__ void group_sync(int grp) {
    if constexpr (G == 1)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(32 * G) : "memory");
}
template <int G>
__device__ __forceinline__ bool group_all(int grp, bool p) {
    if constexpr (G == 1) {
        return __all_sync(kFull, p);
    } else {
        unsigned r;
        asm volatile(
            "{\n\t.reg .pred q, rq;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred rq, %2, %3, q;\n\tselp.u32 %0, 1, 0, "
            "rq;\n\t}"
            : "=r"(r)
            : "r"((unsigned)p), "r"(1 + grp), "r"(32 * G)
            : "memory");
        return r != 0;
    }
}

template <int K, int E>
__global__ void __launch_bounds__(TilesCfg<K, E>::WARPS * 32)
fill_tiles_kernel(const LaunchDesc L) {
    constexpr int VOL = geo_vol(K, E);
    constexpr int VOLH = geo_volh(K, E);
    constexpr int PLANES = geo_planes(K, E);
    constexpr int NM = (1 << K) - 1;
    constexpr int CB = K <= 4 ? 8 : 4;  // bits per packed local coordinate
    constexpr unsigned CMASK = (1u << CB) - 1;
    constexpr int MASKB = (1 << K) - 1;  // tie bits B = k

    constexpr bool TM = K >= kTileMajorMinK;  // tile-major scratch and traceback
    constexpr int NH = geo_cellsh(K, E) - VOL;  // halo cells

    extern __shared__ __align__(16) unsigned char smem[];
    uint2 *sched = reinterpret_cast<uint2 *>(smem);
    int *pstart = reinterpret_cast<int *>(smem + round_up(VOL * 8, 16));
    int *pcur = pstart + round_up(PLANES + 1, 4);
    constexpr bool HPK = tiles_halo_packed<K, E>();  // 4-byte halo entries
    constexpr int SB = bits_for(VOLH), LB = bits_for(VOL);
    uint2 *htab = reinterpret_cast<uint2 *>(pcur + tiles_pcur_ints<K, E>());
    uint32_t *htab4 = reinterpret_cast<uint32_t *>(htab);
    uint16_t *wtab = reinterpret_cast<uint16_t *>(reinterpret_cast<unsigned char *>(htab) +
                                                  (TM ? round_up(NH * (HPK ? 4 : 8), 16) : 0));
    unsigned char *wbase = reinterpret_cast<unsigned char *>(htab) + tiles_tm_cta_bytes<K, E>();

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int G = tiles_group<K, E>(), TG = 32 * G;  // warps and threads per tile
    const int grp = warp / G, gl = tid - grp * TG;        // tile group, thread in the group

    // Intra-tile schedule: every cell of a full tile, grouped by local index sum.
    for (int s = tid; s < PLANES; s += blockDim.x) pcur[s] = 0;
    __syncthreads();
    for (int i = tid; i < VOL; i += blockDim.x) {
        int s = 0, rem = i;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int c = rem / geo_st(K, E, j);
            rem -= c * geo_st(K, E, j);
            s += c;
        }
        atomicAdd(&pcur[s], 1);
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int s = 0; s < PLANES; ++s) {
            pstart[s] = acc;
            acc += pcur[s];
            pcur[s] = pstart[s];
        }
        pstart[PLANES] = acc;
    }
    __syncthreads();
    // placement by one warp, 32 cells at a time in index order, so every plane
    // lists its cells in increasing local index (neighbouring lanes then read
    // nearby shared-memory words)
    if (warp == 0)
        for (int i0 = 0; i0 < VOL; i0 += 32) {
            const int i = i0 + lane;
            int s = 0, rem = i, soff = 0;
            uint32_t pk = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const int c = rem / geo_st(K, E, j);
                rem -= c * geo_st(K, E, j);
                s += c;
                soff += (c + 1) * geo_sh(K, E, j);
                pk |= (uint32_t)c << (CB * j);
            }
            const bool live = i < VOL;
            const unsigned act = __ballot_sync(kFull, live);
            const unsigned same = __match_any_sync(kFull, live ? s : -1);
            if (live) {
                const int pos = pcur[s] + __popc(same & ((1u << lane) - 1));
                sched[pos] = make_uint2((uint32_t)soff | ((uint32_t)i << 16), pk);
            }
            __syncwarp();
            if (live && lane == __ffs(same & act) - 1) pcur[s] += __popc(same);
            __syncwarp();
        }
    __syncthreads();
    // Interleave each plane's cells by the shared-memory bank of their score
    // slot (soff mod 32, round-robin over banks: every bank's first cell, then
    // every bank's second, ...). All predecessor reads of a round of 32 cells
    // are one common offset from soff, so cells of distinct banks read distinct
    // banks in every one of them. Scratch: the warp's tile area, unused until
    // the tiles start.
    {
        const int nwarps = (int)(blockDim.x >> 5);
        constexpr int kScratch = tiles_warp_bytes<K, E>() / G / 16 * 16;  // per warp
        int *tot = reinterpret_cast<int *>(wbase + grp * tiles_warp_bytes<K, E>() + (warp - grp * G) * kScratch);
        int *rank = tot + 32;
        for (int p = warp; p < PLANES; p += nwarps) {
            const int b0 = pstart[p], n = pstart[p + 1] - b0;
            if (n <= 32 || 136 + n * 12 > kScratch) continue;
            uint2 *tmp = reinterpret_cast<uint2 *>(rank + round_up(n, 2));
            tot[lane] = 0;
            __syncwarp();
            for (int c0 = 0; c0 < n; c0 += 32) {  // rank among the plane's earlier cells of the same bank
                const int i = c0 + lane;
                const bool live = i < n;
                const uint2 e = live ? sched[b0 + i] : make_uint2(0, 0);
                const int bank = live ? (int)(e.x & 31) : -1;
                const unsigned peers = __match_any_sync(kFull, bank);
                const int r = live ? tot[bank] + __popc(peers & ((1u << lane) - 1)) : 0;
                __syncwarp();
                if (live && lane == __ffs(peers) - 1) tot[bank] += __popc(peers);
                if (live) {
                    tmp[i] = e;
                    rank[i] = r;
                }
                __syncwarp();
            }
            for (int i = lane; i < n; i += 32) {  // position of (rank, bank) in round-robin order
                const uint2 e = tmp[i];
                const int bank = (int)(e.x & 31), r = rank[i];
                int pos = 0;
                for (int b2 = 0; b2 < 32; ++b2) {
                    const int t = tot[b2];
                    pos += min(t, r) + (b2 < bank && t > r ? 1 : 0);
                }
                sched[b0 + pos] = e;
            }
            __syncwarp();
        }
    }
    __syncthreads();

    if constexpr (TM) {
        // write-back table: the shared-memory offset of each interior cell (local row-major)
        for (int i = tid; i < VOL; i += blockDim.x) {
            int rem = i, soff = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const int c = rem / geo_st(K, E, j);
                rem -= c * geo_st(K, E, j);
                soff += (c + 1) * geo_sh(K, E, j);
            }
            wtab[i] = (uint16_t)soff;
        }
        // halo table, in shared-memory order: cells with some local coordinate -1
        // belong to the lower neighbour tile S (the axes at -1), at local
        // coordinate E - 1 on those axes. Ranked chunk by chunk with a block scan
        // (pcur is free once the schedule is built: warp counts, then the running total).
        const int nwarps = (int)(blockDim.x >> 5);
        if (tid == 0) pcur[nwarps] = 0;
        __syncthreads();
        for (int base = 0; base < VOLH; base += blockDim.x) {
            const int i = base + tid;
            bool halo = false;
            uint32_t S = 0, loff = 0;
            if (i < VOLH) {
                int rem = i;
                bool pad = false;
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const int d = rem / geo_sh(K, E, j);  // halo'd coordinate 0 .. E_j (above: a pad position)
                    rem -= d * geo_sh(K, E, j);
                    pad = pad || d > tile_ext(K, E, j);
                    const int cl = d == 0 ? tile_ext(K, E, j) - 1 : d - 1;
                    if (d == 0) S |= 1u << j;
                    loff += (uint32_t)(cl * geo_st(K, E, j));
                }
                halo = S != 0 && !pad;
            }
            const unsigned bal = __ballot_sync(kFull, halo);
            if (lane == 0) pcur[warp] = __popc(bal);
            __syncthreads();
            int pos = pcur[nwarps] + __popc(bal & ((1u << lane) - 1));
            for (int w2 = 0; w2 < warp; ++w2) pos += pcur[w2];
            if (halo) {
                if constexpr (HPK)
                    htab4[pos] = (uint32_t)i | (S << SB) | (loff << (SB + K));
                else
                    htab[pos] = make_uint2((uint32_t)i | (S << 16), loff);
            }
            __syncthreads();
            if (tid == 0)
                for (int w2 = 0; w2 < nwarps; ++w2) pcur[nwarps] += pcur[w2];
            __syncthreads();
        }
    }

    int32_t *qs = reinterpret_cast<int32_t *>(wbase + grp * tiles_warp_bytes<K, E>());
    unsigned char *tbs = reinterpret_cast<unsigned char *>(qs) + round_up(VOLH * 4, 16);
    unsigned char *tcs = tbs + round_up(VOL, 16);
    int *nbase = reinterpret_cast<int *>(tcs + round_up(geo_codes(K, E), 16));
    int *ptab = nbase + (TM ? (1 << K) : 0);

    __shared__ int2 gtick[G > 1 ? 16 : 1];  // per group: ticket, launch error seen
    while (true) {
        int t = 0;
        if constexpr (G == 1) {
            if (lane == 0) t = atomicAdd(L.ticket, 1);
            t = __shfl_sync(kFull, t, 0);
            if ((int64_t)t >= L.ntickets) break;
            if (ld_volatile(L.err) != 0) break;
        } else {
            // one thread takes the ticket and reads the launch error for the group,
            // so that every decision below is the same in all of its warps
            if (gl == 0) gtick[grp] = make_int2(atomicAdd(L.ticket, 1), ld_volatile(L.err));
            group_sync<G>(grp);
            const int2 te = gtick[grp];
            t = te.x;
            if ((int64_t)t >= L.ntickets) break;
            if (te.y != 0) break;
        }
        const uint64_t ent = L.order[t];
        const ProblemDesc &P = L.probs[(int)(ent >> 32)];
        const int64_t lin = (int64_t)(uint32_t)ent;

        int o[K], e[K], tco[K], len[K], cofs[K];
        int64_t qstr[K], tstr[K];
        int64_t rem = lin;
        bool corner = true, origin = true, full = true;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int64_t gs = P.gstride[j];
            tco[j] = (int)(rem / gs);
            rem -= tco[j] * gs;
            o[j] = tco[j] * tile_ext(K, E, j);
            const int rho = P.rho[j];
            e[j] = min(tile_ext(K, E, j), rho - o[j]);
            corner = corner && (o[j] + e[j] == rho);
            full = full && e[j] == tile_ext(K, E, j);
            origin = origin && (o[j] == 0);
            len[j] = P.len[j];
            cofs[j] = P.cofs[j];
            qstr[j] = P.qstride[j];
            tstr[j] = P.tbstride[j];
        }
        const int64_t tile_base = P.tile_base;

        // Wait for the face predecessors (one thread per axis); their own waits
        // make every lower neighbour complete. In a pruned fill (P.skip set) a
        // tile the bound leaves out waits for nothing -- it only stores "no cell"
        // scores -- so that chain is broken: a live tile there waits for every
        // lower neighbour it reads (one thread per nonempty subset of the axes).
        // The flags are fixed before the fill, so the branch is the same for the
        // whole group.
        const bool left_out = P.skip != nullptr && P.skip[lin] != 0;
        bool ok = true;
        if (P.skip == nullptr) {
#pragma unroll
            for (int j = 0; j < K; ++j)
                if (gl == j && tco[j] > 0)
                    ok = wait_at_least(&L.done[tile_base + lin - P.gstride[j]], 1, L.err, L.spin_ns);
        } else if (!left_out) {
            for (int S = gl + 1; S < (1 << K) && ok; S += TG) {
                bool in = true;
                int64_t n = lin;
#pragma unroll
                for (int j = 0; j < K; ++j)
                    if ((S >> j) & 1) {
                        in = in && tco[j] > 0;
                        n -= P.gstride[j];
                    }
                if (in) ok = wait_at_least(&L.done[tile_base + n], 1, L.err, L.spin_ns);
            }
        }
        if (!group_all<G>(grp, ok)) {
            if (gl == 0) atomicCAS(L.err, 0, MSA_ETIMEOUT);
            break;
        }
        __threadfence();

        bool live;
        if constexpr (G == 1)
            live = ld_volatile(&P.istat->status) == 0;
        else
            live = group_all<G>(grp, ld_volatile(&P.istat->status) == 0);
        // A tile the pruning bound leaves out (its bound is below a lower bound on
        // the optimum, so none of its cells lies on an optimal alignment) stores
        // "no cell" scores for its successors, computes nothing and publishes
        // below. The branch is the same for the whole group and holds no barrier.
        if (live && left_out) {
            int32_t *__restrict__ Qw = P.Q;
            if constexpr (TM) {
                int32_t *qb = Qw + lin * VOL;
                for (int i = gl; i < VOL; i += TG) qb[i] = kNeg;
            } else {
                for (int i = gl; i < VOL; i += TG) {
                    int r = i;
                    bool in = true;
                    int64_t gq = 0;
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        const int cj = r / geo_st(K, E, j);
                        r -= cj * geo_st(K, E, j);
                        in = in && (cj < e[j]);
                        gq += (int64_t)(o[j] + cj) * qstr[j];
                    }
                    if (in) Qw[gq] = kNeg;
                }
            }
        }
        if (live && !left_out) {
            const int A = P.A;
            const int32_t *__restrict__ tab = P.tab;
            const uint8_t *__restrict__ codes = P.codes;
            const int32_t *__restrict__ Qg = P.Q;

            // Residue codes entering each local coordinate (x_j = o_j + c consumes
            // residue x_j - 1 of sequence j).
#pragma unroll
            for (int j = 0; j < K; ++j)
                for (int c = gl; c < tile_ext(K, E, j); c += TG) {
                    const int x = o[j] + c;
                    tcs[geo_code_base(K, E, j) + c] =
                        (x >= 1 && x <= len[j]) ? codes[cofs[j] + x - 1] : (uint8_t)0;
                }

            if constexpr (TM) {
                // this tile's pair tables: ptab[pair(l,h)][a*E + b] = tab[code_l(a)][code_h(b)]
                group_sync<G>(grp);
                for (int idx = gl; idx < tiles_ptab_ints<K, E>(); idx += TG) {
                    const int pr = idx / (E * E), ab = idx - pr * (E * E);
                    int l = 0, rest = pr;
                    while (rest >= K - 1 - l) {
                        rest -= K - 1 - l;
                        ++l;
                    }
                    const int h = l + 1 + rest;
                    const int ca = tcs[geo_code_base(K, E, l) + ab / E], cb = tcs[geo_code_base(K, E, h) + ab % E];
                    ptab[idx] = __ldg(tab + ca * A + cb);
                }
            }

            // Halo: every cell with some local coordinate -1. Loads bypass L1
            // (other SMs wrote these cells) and are issued in batches of HB before
            // their shared-memory stores, so the halo costs about one L2 round trip
            // per batch rather than one per element.
            constexpr int HB = (K >= 6 ? 48 : K == 5 ? (G > 1 ? 24 : 16) : K == 4 ? 16 : 8) / G;  // measured per shape
            if constexpr (TM) {
                // lower neighbour tiles' blocks (none across the origin faces)
                for (int S = gl + 1; S < (1 << K); S += TG) {
                    int64_t nb = lin;
                    bool ok = true;
#pragma unroll
                    for (int j = 0; j < K; ++j)
                        if ((S >> j) & 1) {
                            ok = ok && tco[j] > 0;
                            nb -= P.gstride[j];
                        }
                    nbase[S] = ok ? (int)(nb * VOL) : -1;
                }
                group_sync<G>(grp);
                for (int i0 = 0; i0 < NH; i0 += TG * HB) {
                    int val[HB], dst[HB];
#pragma unroll
                    for (int u = 0; u < HB; ++u) {
                        const int i = i0 + TG * u + gl;
                        dst[u] = -1;
                        val[u] = kNeg;
                        if (i < NH) {
                            int so, sm, lo;
                            if constexpr (HPK) {
                                const uint32_t h = htab4[i];
                                so = (int)(h & ((1u << SB) - 1));
                                sm = (int)((h >> SB) & ((1u << K) - 1));
                                lo = (int)(h >> (SB + K));
                            } else {
                                const uint2 h = htab[i];
                                so = (int)(h.x & 0xFFFFu);
                                sm = (int)(h.x >> 16);
                                lo = (int)h.y;
                            }
                            const int b = nbase[sm];
                            dst[u] = so;
                            if (b >= 0) val[u] = __ldcg(Qg + b + lo);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < HB; ++u)
                        if (dst[u] >= 0) qs[dst[u]] = val[u];
                }
            }
#pragma unroll
            for (int f = 0; f < (TM ? 0 : K); ++f) {
                for (int i0 = 0; i0 < face_size(K, E, f); i0 += TG * HB) {
                    int val[HB], dst[HB];
#pragma unroll
                    for (int u = 0; u < HB; ++u) {
                        const int i = i0 + TG * u + gl;
                        int r = i, soff = 0;
                        bool in = i < face_size(K, E, f), neg = false;
                        int64_t g = 0;
#pragma unroll
                        for (int j = 0; j < K; ++j) {
                            const int fs = face_stride(K, E, f, j);
                            int cj = r / fs;
                            r -= cj * fs;
                            if (j >= f) cj -= 1;
                            in = in && (cj < e[j]);
                            neg = neg || (cj < 0 && o[j] == 0);
                            soff += (cj + 1) * geo_sh(K, E, j);
                            g += (int64_t)(o[j] + cj) * qstr[j];
                        }
                        dst[u] = in ? soff : -1;
                        val[u] = (in && !neg) ? __ldcg(Qg + g) : kNeg;
                    }
#pragma unroll
                    for (int u = 0; u < HB; ++u)
                        if (dst[u] >= 0) qs[dst[u]] = val[u];
                }
            }
            group_sync<G>(grp);

            int Wo = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) Wo += o[j] << j;

            for (int s = 0; s < PLANES; ++s) {
                const int b = pstart[s], en = pstart[s + 1];
                for (int idx = b + gl; idx < en; idx += TG) {
                    const uint2 sc = sched[idx];
                    const int soff = (int)(sc.x & 0xFFFFu), toff = (int)(sc.x >> 16);
                    int c[K], wl = 0;
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        c[j] = (int)((sc.y >> (CB * j)) & CMASK);
                        wl += c[j] << j;
                    }
                    if (!full) {  // an edge tile: skip cells outside the tensor
                        bool in = true;
#pragma unroll
                        for (int j = 0; j < K; ++j) in = in && (c[j] < e[j]);
                        if (!in) continue;
                    }
                    if (origin && s == 0) {  // H(0) = 0
                        qs[soff] = 0;
                        tbs[toff] = 0;
                        continue;
                    }
                    int a[K];
                    if constexpr (!TM) {
#pragma unroll
                        for (int j = 0; j < K; ++j) a[j] = tcs[geo_code_base(K, E, j) + c[j]];
                    }
                    // Candidates grouped by the move's highest sequence h. The pair
                    // sum of m = r | 2^h is S[r] + T[r] with T[r] = sum_{l in r}
                    // (scaled pair l, h); S is stored only below 2^(K-1), the top
                    // group is consumed as it is formed, so the live state stays
                    // small enough for registers.
                    // NACC independent max chains (max is associative and commutative)
                    constexpr int NACC = K <= 3 ? 1 : K <= 5 ? 2 : 4;
                    int accs[NACC];
#pragma unroll
                    for (int i = 0; i < NACC; ++i) accs[i] = kNeg;
#pragma unroll
                    for (int i = 0; i < K; ++i) accs[i % NACC] = max(accs[i % NACC], qs[soff - geo_sh(K, E, i)]);
                    int S[1 << (K - 1)];
                    S[0] = 0;
                    S[1] = 0;  // the singleton {0}: no pair
#pragma unroll
                    for (int h = 1; h < K; ++h) {
                        int ph[K];
#pragma unroll
                        for (int l = 0; l < h; ++l) {
                            if constexpr (TM)
                                ph[l] = ptab[pair_index(K, l, h) * (E * E) + c[l] * E + c[h]];
                            else
                                ph[l] = __ldg(tab + a[l] * A + a[h]);
                        }
                        int T[1 << (K - 1)];
                        T[0] = 0;
#pragma unroll
                        for (int r2 = 1; r2 < (1 << h); ++r2) T[r2] = T[r2 & (r2 - 1)] + ph[lowbit_c(r2)];
#pragma unroll
                        for (int r2 = 0; r2 < (1 << h); ++r2) {
                            const int sm = S[r2] + T[r2];
                            if (h < K - 1) S[r2 | (1 << h)] = sm;
                            if (r2 != 0)
                                accs[r2 % NACC] =
                                    __viaddmax_s32(qs[soff - move_soff(K, E, r2 | (1 << h))], sm, accs[r2 % NACC]);
                        }
                    }
                    int acc = accs[0];
#pragma unroll
                    for (int i = 1; i < NACC; ++i) acc = max(acc, accs[i]);
                    const int tmask = (Wo + wl - acc) & MASKB;
                    qs[soff] = acc + tmask;
                    tbs[toff] = (unsigned char)tmask;
                }
                group_sync<G>(grp);
            }

            // Write back scores (for successor halos) and traceback bytes.
            int32_t *__restrict__ Qw = P.Q;
            uint8_t *__restrict__ tbw = P.tb;
            if constexpr (TM) {
                // this tile's blocks, contiguous (cells outside the tensor included)
                int32_t *qb = Qw + lin * VOL;
                uint8_t *tbb = tbw + lin * VOL;
                for (int i = gl; i < VOL; i += TG) {
                    qb[i] = qs[wtab[i]];
                    tbb[i] = tbs[i];
                }
            }
            for (int i = gl; i < (TM ? 0 : VOL); i += TG) {
                int r = i, soff = 0;
                bool in = true;
                int64_t gq = 0, gt = 0;
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const int cj = r / geo_st(K, E, j);
                    r -= cj * geo_st(K, E, j);
                    in = in && (cj < e[j]);
                    soff += (cj + 1) * geo_sh(K, E, j);
                    gq += (int64_t)(o[j] + cj) * qstr[j];
                    gt += (int64_t)(o[j] + cj) * tstr[j];
                }
                if (in) {
                    Qw[gq] = qs[soff];
                    tbw[gt] = tbs[i];
                }
            }
            if (corner && gl == 0) {
                int soff = 0;
#pragma unroll
                for (int j = 0; j < K; ++j) soff += e[j] * geo_sh(K, E, j);
                *P.qcorner = qs[soff];
            }
        }
        group_sync<G>(grp);
        if (gl == 0 && (int64_t)t != L.withhold) {
            __threadfence();
            st_release(&L.done[tile_base + lin], 1);
        }
    }
}

// Shared-memory attribute of fill_tiles_kernel<K, E>, set once per device (so
// that no launch inside a stream capture makes the call).
template <int K, int E>
cudaError_t tiles_attributes() {
    static DeviceOnce once;
    return once.run([] {
        return cudaFuncSetAttribute(fill_tiles_kernel<K, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    tiles_smem_bytes<K, E>());
    });
}

template <int K, int E>
cudaError_t launch_tiles(const LaunchDesc &L, int grid, cudaStream_t s) {
    constexpr int smem = tiles_smem_bytes<K, E>();
    cudaError_t e = tiles_attributes<K, E>();
    if (e != cudaSuccess) return e;
    fill_tiles_kernel<K, E><<<grid, TilesCfg<K, E>::WARPS * 32, smem, s>>>(L);
    return cudaGetLastError();
}

template <int K, int E>
int tiles_ctas() {
    constexpr int smem = tiles_smem_bytes<K, E>();
    if (tiles_attributes<K, E>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fill_tiles_kernel<K, E>, TilesCfg<K, E>::WARPS * 32,
                                                      smem) != cudaSuccess)
        return 0;
    return n;
}

// Dispatch of one k over its candidate edges (instantiated in fill_tiles_k<k>.cu).
template <int K>
struct TilesK {
    static constexpr int E0 = tile_edge_candidate(K, 0), E1 = tile_edge_candidate(K, 1),
                         E2 = tile_edge_candidate(K, 2);
    static cudaError_t launch(int edge, const LaunchDesc &L, int grid, cudaStream_t s) {
        if (edge == E0) return launch_tiles<K, E0>(L, grid, s);
        if constexpr (E1 > 0)
            if (edge == E1) return launch_tiles<K, E1>(L, grid, s);
        if constexpr (E2 > 0)
            if (edge == E2) return launch_tiles<K, E2>(L, grid, s);
        return cudaErrorInvalidValue;
    }
    static int ctas(int edge) {
        if (edge == E0) return tiles_ctas<K, E0>();
        if constexpr (E1 > 0)
            if (edge == E1) return tiles_ctas<K, E1>();
        if constexpr (E2 > 0)
            if (edge == E2) return tiles_ctas<K, E2>();
        return 0;
    }
    static int warps(int edge) {
        if (edge == E0) return TilesCfg<K, E0>::WARPS;
        if constexpr (E1 > 0)
            if (edge == E1) return TilesCfg<K, E1>::WARPS;
        if constexpr (E2 > 0)
            if (edge == E2) return TilesCfg<K, E2>::WARPS;
        return 0;
    }
};

}  // namespace msadp
