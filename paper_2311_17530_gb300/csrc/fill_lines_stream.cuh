// Streamed line fill for k = 4..6: the line kernel's recurrence and lanes
// (fill_lines.cuh: lane l of a warp owns one line of a 32-line block, skewed by
// the sum of its local coordinates; candidates of the moves that also advance
// the last axis s are carried from the previous step), organised for the
// latency of the hardware:
//
// * A CTA of W warps owns a SUPER-BLOCK of W line blocks (a grid of extents
//   stream_wg over the line axes) and sweeps it over the WHOLE last axis in
//   lockstep: at step t every lane of the CTA computes position z = t - sigma of
//   its line, sigma being the sum of the line's coordinates inside the
//   super-block, and a CTA barrier ends the step. Every predecessor line of the
//   super-block then holds position z at time t - |m'|, so warps exchange
//   nothing but shared memory; only super-blocks talk through global memory.
//   The skew, the set-up and the ticket are paid once per super-block column.
// * Super-blocks are handed out in wave order of their grid (section 3: blocks
//   whose coordinates sum to w form wave w). After each block of U steps a
//   super-block publishes what its upper-face lines held at those U TIMES, as
//   (value, tag) 8-byte entries (the tag is the launch's epoch), then a count
//   of published blocks (a plain relaxed store). Publishing by time makes a
//   block's data complete as soon as the block ends; a consumer's halo time tau
//   is its producer's time tau + SB_S (the super-block extents along the axes
//   S in which the producer lies below).
// * A consumer loads its producers' counts at a block's start and, once they
//   cover the next block's halo, copies it into a staging buffer during the
//   sweep (16-byte cp.async copies through L2); at the block's end it accepts
//   the entries once every one carries the epoch, copying again otherwise (a
//   bounded wait). The counts only spare the memory system from copies that
//   would fail: correctness rests on the tags, so no fence or release/acquire
//   pair is needed. An aligned 8-byte entry is written by one store and read
//   whole, and each entry is written once per launch; earlier launches left
//   smaller epochs (the plan clears the faces before the first launch and when
//   epochs wrap).
//
// Shared memory per CTA:
//   V      a ring of D words per line of the halo'd super-block (local
//          coordinates -1 .. SB_i - 1), indexed by time: position z of line c sits
//          in slot (z + sigma(c)) mod D. At step t every lane reads slot
//          (t - |m'|) mod D of its predecessor line c - e_m' (one slot for all
//          lanes) and writes slot t mod D of its own line, so the 32 accesses of
//          a warp are conflict-free when sum_i c_i A_i is distinct mod 32 over a
//          line block (strides A_i found by exhaustive search, below).
//   PT     an R-position ring of the pair tables of s against every line axis.
//   stage  the halo of the next block: U times of every halo line.
//   tables of the halo and face lines, the neighbour super-block of every
//          subset of the line axes, the residue code of every pair-table row.
// Blocks of U = 8 steps and a D = 16 slot ring for k = 4, 5; for k = 6 (547 halo
// lines around 128, so the ring and staging per CTA are large) U = 4 and D = 12,
// which leaves room for three CTAs per SM instead of two.
//
// Global memory: the traceback bytes of each line block (a tile of the line
// kernel's layout 3 spanning the whole last axis: cell (c, z) at
// (z + sum c_i) * 32 + lane); the faces of each super-block: its upper-face
// lines, line-major, ZQ times each.
#pragma once

#include <type_traits>

#include "device_common.cuh"

namespace msadp {

// Ring slots per line: a line's times from t - (k - 1) on plus the next block's
// U times, so D >= U + k - 1, and a whole number of blocks, so that every slot a
// step touches is a constant within a block of known parity b mod (D / U).
__host__ __device__ constexpr int stream_ring_d(int K) { return K == 6 ? 12 : 16; }
// Pair-table ring positions: a block reads positions bU - SMAX .. bU + U - 1.
__host__ __device__ constexpr int stream_pt_ring(int K) { return K == 6 ? 16 : 32; }

// Ring stride (words) of line axis i over the halo'd super-block: the smallest
// footprint with every line's D slots disjoint and sum_i c_i A_i distinct mod 32
// over a warp's line block.
__host__ __device__ constexpr int stream_stride(int K, int i) {
    constexpr int k4[] = {16, 81, 732}, k5[] = {16, 81, 406, 1220}, k6[] = {12, 61, 306, 920, 2768};
    return K == 4 ? k4[i] : K == 5 ? k5[i] : k6[i];
}
template <int K>
__host__ __device__ constexpr int stream_move_off(int m) {
    int s = 0;
    for (int i = 0; i < K - 1; ++i)
        if ((m >> i) & 1) s += stream_stride(K, i);
    return s;
}
template <int K>
__host__ __device__ constexpr int stream_halo_lines() {  // lines of the halo'd super-block with some index -1
    int all = 1;
    for (int i = 0; i < K - 1; ++i) all *= stream_sb(K, i) + 1;
    return all - 32 * stream_warps(K);
}
template <int K>
__host__ __device__ constexpr int stream_rows() {  // pair-table rows: one per (line axis, coordinate)
    int n = 0;
    for (int i = 0; i < K - 1; ++i) n += stream_sb(K, i);
    return n;
}
template <int K>
__host__ __device__ constexpr int stream_ring_words() {
    int s = stream_ring_d(K);
    for (int i = 0; i < K - 1; ++i) s += stream_sb(K, i) * stream_stride(K, i);
    return round_up(s, 4);
}
// Shared memory of a CTA, in 4-byte words (every part 16-byte aligned).
template <int K>
struct StreamLayout {
    static constexpr int NH = stream_halo_lines<K>();
    static constexpr int NFL = stream_face_lines(K);
    static constexpr int NROW = stream_rows<K>();
    // pair-table rows: an R-position ring stored twice (slots p mod R and
    // p mod R + R, so that a block's positions need no wrap), rows staggered by
    // (a line block's skew) + 1 banks
    static constexpr int ZS = 2 * stream_pt_ring(K) + line_skew_max(K) + 1;
    static constexpr int NT = 32 * stream_warps(K);
    static constexpr int V = 0;
    static constexpr int PT = V + stream_ring_words<K>();
    static constexpr int STAGE = PT + round_up(NROW * ZS, 4);
    static constexpr int NT_ = 32 * stream_warps(K);
    static constexpr int HC = (NH * (stream_block(K) / 2) + NT_ - 1) / NT_;  // halo copies per thread and block
    static constexpr int HOFS = STAGE + NH * stream_block(K) * 2;  // per copy: source offset (8 bytes)
    static constexpr int HMETA = HOFS + 2 * HC * NT_;               // ... ring base | time offset << 14
    static constexpr int HTAB = HMETA + HC * NT_;
    static constexpr int FTAB = HTAB + round_up(NH, 4);
    static constexpr int NB = FTAB + round_up(NFL, 4);
    static constexpr int CROW = NB + round_up(1 << (K - 1), 4);
    static constexpr int MISC = CROW + round_up(NROW, 4);  // ticket, verdicts
    static constexpr int WORDS = MISC + 8;
};
template <int K>
__host__ __device__ constexpr int stream_smem_bytes() {
    return StreamLayout<K>::WORDS * 4;
}
template <int K>
__host__ __device__ constexpr int stream_threads() {
    return 32 * stream_warps(K);
}
// CTAs per SM: what shared memory allows (228 KB per SM, 1 KB reserved per CTA,
// at most 48 warps) and what a budget of registers per thread allows (the sweep
// keeps 2^(k-1) carried candidates and pair sums live); the launch bound caps
// registers to match.
template <int K>
__host__ __device__ constexpr int stream_min_ctas() {
    int c = (228 * 1024) / (stream_smem_bytes<K>() + 1024);
    if (c * stream_warps(K) > 48) c = 48 / stream_warps(K);
    const int regs = K == 4 ? 80 : 168;
    const int cr = 65536 / (regs * stream_threads<K>());
    return c < cr ? c : cr;
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void st_relaxed_v2(unsigned long long *p, unsigned long long a, unsigned long long b) {
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ unsigned long long tagged(int value, int tag) {
    return (unsigned long long)(unsigned)value | ((unsigned long long)(unsigned)tag << 32);
}

template <int P>
using IntC = std::integral_constant<int, P>;

template <int K>
__global__ void __launch_bounds__(stream_threads<K>(), stream_min_ctas<K>()) fill_lines_stream_kernel(const LaunchDesc L) {
    constexpr int NA = K - 1;
    constexpr int M = (1 << NA) - 1;
    constexpr int NT = stream_threads<K>();
    constexpr int NLINES = NT;
    constexpr int SMAX = stream_skew_max(K);
    constexpr int U = stream_block(K), D = stream_ring_d(K), R = stream_pt_ring(K);
    constexpr int NPAR = D / U;  // block parities: slot of time bU + s is ((b mod NPAR) U + s) mod D
    constexpr int MASKB = (1 << K) - 1;
    using LY = StreamLayout<K>;
    constexpr int NH = LY::NH, NFL = LY::NFL, NROW = LY::NROW, ZS = LY::ZS;
    constexpr int NP = NH * (U / 2);              // halo copies (two entries each) per block
    constexpr int HC = LY::HC;                    // ... per thread
    constexpr int NF = NFL * (U / 2);             // face stores (two entries each) per block
    constexpr int FC = (NF + NT - 1) / NT;        // ... per thread
    constexpr int PQ = (NROW * U + NT - 1) / NT;  // pair-table entries per thread and refill
    constexpr int C0 = -((NA + U - 1) / U);       // first halo chunk: halo times start at -(k - 1)
    // The ring holds a line's times from t - (k - 1) on plus the next block's U
    // times; the pair-table ring holds the positions a block reads, bU - SMAX ..
    // bU + U - 1, and after the block the next U positions replace positions
    // below (b + 1) U - SMAX.
    static_assert(D % U == 0 && NPAR <= 4 && D >= U + NA && SMAX + U <= R && (R & (R - 1)) == 0 && NFL < 128 &&
                      LY::PT < (1 << 14) && NT % (U / 2) == 0 && SMAX < 32 && M < 32,
                  "geometry");
    // ring slot of a time (which may be negative)
    auto rslot = [](int x) { return (D & (D - 1)) == 0 ? x & (D - 1) : ((x % D) + D) % D; };

    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t *sm = reinterpret_cast<int32_t *>(smem_raw);
    int32_t *V = sm + LY::V;
    int32_t *PT = sm + LY::PT;
    unsigned long long *stage = reinterpret_cast<unsigned long long *>(sm + LY::STAGE);
    // halo lines: ring base | producer face line << 14 | axes S at -1 << 21 |
    // (the sum of SB_i over S: the producer's time offset) << 26
    int64_t *hofs = reinterpret_cast<int64_t *>(sm + LY::HOFS);
    int32_t *hmeta = sm + LY::HMETA;
    uint32_t *htab = reinterpret_cast<uint32_t *>(sm + LY::HTAB);
    uint32_t *ftab = reinterpret_cast<uint32_t *>(sm + LY::FTAB);  // face lines: ring base
    int32_t *nb = sm + LY::NB;
    int32_t *crow = sm + LY::CROW;
    // [0] ticket, [2] poll verdict, [3] / [4] the two count checkpoints' verdicts
    volatile int32_t *misc = sm + LY::MISC;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) {
        // face lines of the super-block in line order (coordinates c_i in
        // [0, SB_i), axis 0 most significant); their numbers index the faces
        // (fnum: a line's face number, kept in the staging buffer until it is used)
        int32_t *fnum = reinterpret_cast<int32_t *>(stage);
        int nf = 0;
        for (int j = 0; j < NLINES; ++j) {
            int rem = j, base = 0;
            bool face = false;
            for (int i = NA - 1; i >= 0; --i) {
                const int c = rem % stream_sb(K, i);
                rem /= stream_sb(K, i);
                base += (c + 1) * stream_stride(K, i);
                face = face || c == stream_sb(K, i) - 1;
            }
            fnum[j] = face ? nf : -1;
            if (face) ftab[nf++] = (uint32_t)base;
        }
        // halo lines (digits h_i in [0, SB_i], some 0): the producer's face line
        // has c_i = SB_i - 1 where h_i = 0 and h_i - 1 elsewhere
        int n = 0;
        int hall = 1;
        for (int i = 0; i < NA; ++i) hall *= stream_sb(K, i) + 1;
        for (int j = 0; j < hall; ++j) {
            int rem = j, base = 0, lp = 0, lstr = 1;
            uint32_t S = 0, sbs = 0;
            for (int i = NA - 1; i >= 0; --i) {
                const int h = rem % (stream_sb(K, i) + 1);
                rem /= stream_sb(K, i) + 1;
                base += h * stream_stride(K, i);
                lp += (h == 0 ? stream_sb(K, i) - 1 : h - 1) * lstr;
                lstr *= stream_sb(K, i);
                if (h == 0) {
                    S |= 1u << i;
                    sbs += stream_sb(K, i);
                }
            }
            if (S) htab[n++] = (uint32_t)base | (uint32_t)fnum[lp] << 14 | S << 21 | sbs << 26;
        }
    }

    // this thread's line: warp coordinates in the warp grid, lane coordinates in
    // the line block; ring base and skew inside the super-block
    int cl[NA], cw[NA];
    int vbase = 0, sig = 0, sigw = 0;
    {
        int rw = warp;
#pragma unroll
        for (int i = NA - 1; i >= 0; --i) {
            cw[i] = rw % stream_wg(K, i);
            rw /= stream_wg(K, i);
        }
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            const int lc = (lane / line_lstride(K, i)) % line_ext(K, i);
            cl[i] = cw[i] * line_ext(K, i) + lc;
            vbase += (cl[i] + 1) * stream_stride(K, i);
            sig += cl[i];
            sigw += cw[i] * line_ext(K, i);
        }
    }
    int32_t *const vb = V + vbase;

    int tnext = 0;
    if (tid == 0) tnext = atomicAdd(L.ticket, 1);
    int cached_prob = -1;
    bool cached_live = false;
    while (true) {
        if (tid == 0) {
            misc[0] = ld_volatile(L.err) != 0 ? 0x7fffffff : tnext;
            if ((int64_t)tnext < L.ntickets) tnext = atomicAdd(L.ticket, 1);
        }
        __syncthreads();  // also: the previous column's last reads of shared memory are done
        const int t = misc[0];
        __syncthreads();  // every thread has the ticket before thread 0 may take the next
        if ((int64_t)t >= L.ntickets) break;
        const uint64_t ent = L.order[t];
        const int pidx = (int)(ent >> 32);
        const ProblemDesc &P = L.probs[pidx];
        const int col = (int)(uint32_t)ent;  // super-block index
        if (pidx != cached_prob) {            // the encode step's verdict (fixed before the fill)
            cached_prob = pidx;
            cached_live = ld_volatile(&P.istat->status) == 0;
        }
        if (!cached_live) continue;  // a failed problem: its columns publish nothing and read nothing

        int sco[NA], o[NA];  // super-block coordinates, its first line's coordinates
        {
            unsigned rem = (unsigned)col;
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                const unsigned gs = (unsigned)P.sgstride[j];
                sco[j] = (int)(rem / gs);
                rem -= (unsigned)sco[j] * gs;
                o[j] = sco[j] * stream_sb(K, j);
            }
        }
        const int A = P.A;
        const int32_t *__restrict__ tab = P.tab;
        const uint8_t *__restrict__ codes = P.codes;
        const int rho = P.rho[NA], lens = P.len[NA], cofs = P.cofs[NA];
        const int ZQ = P.lzq;
        const int nblk = ZQ / U;  // blocks of the sweep: rho + SMAX steps, rounded up
        const int epoch = L.epoch;
        const int tagout = (int64_t)t == L.withhold ? 0 : epoch;  // a withheld column publishes nothing valid
        const int64_t FB = (int64_t)NFL * ZQ;  // face entries per super-block
        unsigned long long *Fq = reinterpret_cast<unsigned long long *>(P.Q);
        unsigned long long *Fo = Fq + (int64_t)col * FB;
        int32_t *const prog = L.done + P.tile_base;  // published blocks per super-block

        // this warp's tile (line block) for the traceback, or none past the grid
        int64_t tile = 0;
        bool has_tile = true;
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            const int g = sco[i] * stream_wg(K, i) + cw[i];
            has_tile = has_tile && g < P.G[i];
            tile += (int64_t)g * P.gstride[i];
        }

        // neighbour super-blocks, the pair-table rows' residue codes; every ring
        // slot starts as "no cell"
        for (int S = tid; S <= M; S += NT) {
            int n = col;
            bool in = true;
#pragma unroll
            for (int i = 0; i < NA; ++i)
                if ((S >> i) & 1) {
                    in = in && sco[i] > 0;
                    n -= (int)P.sgstride[i];
                }
            nb[S] = in ? n : -1;
        }
        if (tid < NROW) {
            int x = 0, len = 0, cof = 0, row = 0;
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                if (tid >= row && tid < row + stream_sb(K, i)) {
                    x = o[i] + tid - row;
                    len = P.len[i];
                    cof = P.cofs[i];
                }
                row += stream_sb(K, i);
            }
            crow[tid] = (x >= 1 && x <= len) ? codes[cof + x - 1] : 0;
        }
        for (int i = tid; i < LY::PT; i += NT) V[i] = kNeg;
        __syncthreads();  // nb, crow and the ring are read by every thread below

        // Halo copies of the consumer times [cU, cU + U): pair idx = (halo line j,
        // q2) holds times cU + 2 q2 and + 1, copied from the producer's face line
        // at those times + SB_S (none where there is no producer or the producer
        // time lies outside [0, ZQ), i.e. outside the producer's sweep).
        const int q2 = tid % (U / 2);  // the same for every copy of this thread
        // this thread's copies, once per column (copy v: pair idx = tid + NT v):
        // the producer's face entry of time 0 (-1: none), ring base | time offset
        // (formed at every copy instead, they cost more than the room they free)
#pragma unroll
        for (int v = 0; v < HC; ++v)
            if (tid + NT * v < NP) {
                const uint32_t e = htab[(tid + NT * v) / (U / 2)];
                const int src = nb[(e >> 21) & 31];
                hofs[v * NT + tid] = src < 0 ? -1 : (int64_t)src * FB + (int64_t)((e >> 14) & 127) * ZQ;
                hmeta[v * NT + tid] = (int)(e & 0x3FFF) | (2 * q2 + (int)(e >> 26)) << 14;
            }
        auto halo_pair = [&](int v, int &base, int &toff) -> int64_t {
            const int meta = hmeta[v * NT + tid];
            base = meta & 0x3FFF;
            toff = meta >> 14;
            return hofs[v * NT + tid];
        };
        auto halo_issue = [&](int c, bool mine) {
            if (mine) {
#pragma unroll
                for (int v = 0; v < HC; ++v) {
                    const int idx = tid + NT * v;
                    if (idx < NP) {
                        int base, toff;
                        const int64_t o = halo_pair(v, base, toff);
                        const int tp = c * U + toff;
                        if (o >= 0 && (unsigned)tp < (unsigned)ZQ) cp_async16(stage + 2 * idx, Fq + o + tp);
                    }
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        auto sb_of = [](uint32_t S) {
            int s = 0;
#pragma unroll
            for (int i = 0; i < NA; ++i)
                if ((S >> i) & 1) s += stream_sb(K, i);
            return s;
        };
        // Warp 0's lanes 1 .. M watch one producer each (subset S = lane). The
        // counts cover consumer chunk c (times [cU, cU + U)) once producer S has
        // published the blocks holding its times up to cU + U - 1 + SB_S.
        const int my_src = warp == 0 && lane >= 1 && lane <= M ? nb[lane] : -1;
        const int my_ahead = 1 + (U - 1 + sb_of((uint32_t)lane)) / U;
        auto count_ok = [&](int cnt, int c) { return cnt >= min(nblk, c + my_ahead); };
        // Wait (bounded) until the counts cover chunk c; every thread gets the verdict.
        uint64_t t0 = 0;
        auto halo_ready = [&](int c) -> bool {
            if (warp == 0) {
                bool ready = false;
                for (int polls = 0;; ++polls) {
                    ready = __all_sync(kFull, my_src < 0 || count_ok(ld_relaxed(prog + my_src), c));
                    if (ready) break;
                    if (t0 == 0) t0 = global_ns();
                    if (ld_volatile(L.err) != 0 || (int64_t)(global_ns() - t0) > L.spin_ns) break;
                    __nanosleep(polls < 8 ? 32 : 128);
                }
                if (lane == 0) misc[2] = ready;
            }
            __syncthreads();
            return misc[2] != 0;
        };
        // Accept chunk c: store the staged entries into the ring once all carry
        // this launch's tag. Copies not yet issued wait for the counts; entries
        // that fail the tag check are copied again. Bounded.
        auto halo_accept = [&](int c, bool issued) -> bool {
            t0 = 0;
            bool mine = true;
            for (int tries = 0;; ++tries) {
                if (!issued) {
                    if (!halo_ready(c)) return false;
                    halo_issue(c, mine);
                }
                asm volatile("cp.async.wait_all;" ::: "memory");  // each thread reads only its own copies
                bool ok = true;
#pragma unroll
                for (int v = 0; v < HC; ++v) {
                    const int idx = tid + NT * v;
                    if (idx < NP) {
                        const int tc = c * U + 2 * q2;
                        int base, toff;
                        const int64_t o = halo_pair(v, base, toff);
                        const int tp = c * U + toff;
                        int v0 = kNeg, v1 = kNeg;
                        if (o >= 0 && (unsigned)tp < (unsigned)ZQ) {
                            const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(stage + 2 * idx);
                            ok = ok && (int)(x.x >> 32) == epoch && (int)(x.y >> 32) == epoch;
                            v0 = (int)(unsigned)x.x;
                            v1 = (int)(unsigned)x.y;
                        }
                        const int sl = rslot(tc);  // tc is even and D even: sl + 1 is the slot of tc + 1
                        V[base + sl] = v0;
                        V[base + sl + 1] = v1;
                    }
                }
                if (__syncthreads_and(ok)) return true;
                bool expired = false;
                if (tid == 0) {
                    if (t0 == 0) t0 = global_ns();
                    expired = ld_volatile(L.err) != 0 || (int64_t)(global_ns() - t0) > L.spin_ns;
                }
                if (__syncthreads_or(expired)) return false;  // no copy is in flight here
                __nanosleep(32);
                issued = false;
                mine = !ok;
            }
        };
        // face times [bU, bU + U) of the upper-face lines
        auto face_write = [&](int b) {
#pragma unroll
            for (int v = 0; v < FC; ++v) {
                const int idx = tid + NT * v;
                if (idx < NF) {
                    const int f = idx / (U / 2), tt = b * U + 2 * (idx % (U / 2));
                    const int base = (int)ftab[f], sl = rslot(tt);
                    st_relaxed_v2(Fo + (int64_t)f * ZQ + tt, tagged(V[base + sl], tagout),
                                  tagged(V[base + sl + 1], tagout));
                }
            }
        };
        // pair tables of positions [p0, p0 + U): codes, then entries (in place), then stores
        int pent[PQ];
        auto pt_codes = [&](int p0) {
#pragma unroll
            for (int u = 0; u < PQ; ++u) {
                const int it = tid + NT * u, p = p0 + it % U;
                pent[u] = (it < NROW * U && p >= 1 && p <= lens) ? codes[cofs + p - 1] : 0;
            }
        };
        auto pt_entries = [&]() {
#pragma unroll
            for (int u = 0; u < PQ; ++u) {
                const int it = tid + NT * u;
                if (it < NROW * U) pent[u] = __ldg(tab + crow[it / U] * A + pent[u]);
            }
        };
        auto pt_store = [&](int p0) {
#pragma unroll
            for (int u = 0; u < PQ; ++u) {
                const int it = tid + NT * u, p = p0 + it % U;
                if (it < NROW * U && p < rho) {
                    PT[(it / U) * ZS + (p & (R - 1))] = pent[u];
                    PT[(it / U) * ZS + (p & (R - 1)) + R] = pent[u];
                }
            }
        };

        // Halo times [C0 U, U): one poll of the counts covers every initial chunk
        // (a halo line with a -1 coordinate holds positions >= 0 at negative
        // times); the first chunk's copies fly while this line's pair sums and the
        // first pair-table positions are formed.
        bool ok = halo_ready(0);
        if (ok) halo_issue(C0, true);
        pt_codes(0);
        int Sp[M + 1];
        {
            int cd[NA];
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                const int x = o[i] + cl[i];
                cd[i] = (x >= 1 && x <= P.len[i]) ? codes[P.cofs[i] + x - 1] : 0;
            }
            Sp[0] = 0;
#pragma unroll
            for (int h = 0; h < NA; ++h) {
                int Rs[1 << (NA - 1)];
                Rs[0] = 0;
#pragma unroll
                for (int r = 1; r < (1 << h); ++r) Rs[r] = Rs[r & (r - 1)] + __ldg(tab + cd[lowbit_c(r)] * A + cd[h]);
#pragma unroll
                for (int r = 0; r < (1 << h); ++r) Sp[r | (1 << h)] = Sp[r] + Rs[r];
            }
        }
        pt_entries();
        pt_store(0);
        if (ok) ok = halo_accept(C0, true);
        for (int c = C0 + 1; c <= 0 && ok; ++c) {
            halo_issue(c, true);
            ok = halo_accept(c, true);
        }
        __syncthreads();

        // The sweep. The origin's lane starts from H(0) = 0 as its "previous
        // position", which makes its key 0 with no move.
        int Wl = -sig * (1 << NA);  // W(x) = Wl + t 2^NA at step t
#pragma unroll
        for (int i = 0; i < NA; ++i) Wl += (o[i] + cl[i]) << i;
        int32_t *ptrow[NA];
        {
            int row = 0;
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                ptrow[i] = PT + (row + cl[i]) * ZS;
                row += stream_sb(K, i);
            }
        }
        int carry[M + 1];
        int vself = col == 0 && tid == 0 ? 0 : kNeg;
#pragma unroll
        for (int m = 1; m <= M; ++m) carry[m] = kNeg + Sp[m];
        // this warp's traceback rows: row r = t - (the line block's first skew)
        const int rows = P.tb_block / 32;
        uint8_t *tbw = P.tb + tile * P.tb_block + lane;

        // One block of U steps, unrolled: PAR = b mod NPAR makes every ring slot a
        // constant.
        // Warp 0 judges the counts at steps J1 and J2 (each verdict in its own
        // word), every thread reads a verdict after that step's barrier and
        // issues the next chunk's copies.
        constexpr int J1 = U / 4, J2 = U / 2 + U / 8;
        static_assert(J1 < J2 && J2 + 1 < U, "checkpoints");
        auto block = [&](int b, auto par) {
            constexpr int PAR = decltype(par)::value;
            const bool want = b + 1 < nblk;  // the next block needs chunk b + 1
            int cnt = 0x7fffffff;
            if (want && my_src >= 0) cnt = ld_relaxed(prog + my_src);
            const bool refill = (b + 1) * U < rho;
            if (refill) pt_codes((b + 1) * U);
            bool issued = false;
            const int Wb0 = Wl + b * U * (1 << NA);
            const int r0 = b * U - sigw;  // traceback row of step bU
            const int zp0 = (b * U - sig) & (R - 1);
            constexpr int sl0 = PAR * U;  // ring slot of time bU
            const int32_t *ptb[NA];
#pragma unroll
            for (int i = 0; i < NA; ++i) ptb[i] = ptrow[i] + zp0;
            auto step = [&](int s) {
                if ((s == J1 || s == J2) && want && !issued && warp == 0) {
                    const bool r = __all_sync(kFull, my_src < 0 || count_ok(cnt, b + 1));
                    if (lane == 0) misc[s == J1 ? 3 : 4] = r;
                    if (!r && my_src >= 0) cnt = ld_relaxed(prog + my_src);
                }
                if ((s == J1 + 1 || s == J2 + 1) && want && !issued) {
                    issued = misc[s == J1 + 1 ? 3 : 4] != 0;
                    if (issued) halo_issue(b + 1, true);
                }
                if (s == U / 2 - 1 && refill) pt_entries();
                const int ts = b * U + s;
                // a warp none of whose lanes holds a cell at this step skips it (every
                // thread still meets the step's one barrier)
                if ((unsigned)(ts - sigw) < (unsigned)(rho + line_skew_max(K))) {
                    const int z = ts - sig;
                    const bool act = (unsigned)z < (unsigned)rho;
                    const int own = sl0 + s < D ? sl0 + s : sl0 + s - D;  // slot of time ts
                    int slp[NA + 1];  // slot of time ts - q
#pragma unroll
                    for (int q = 0; q <= NA; ++q) slp[q] = own - q < 0 ? own - q + D : own - q;
                    int p[NA];
#pragma unroll
                    for (int i = 0; i < NA; ++i) p[i] = ptb[i][s];
                    int T[M + 1];
                    T[0] = 0;
#pragma unroll
                    for (int m = 1; m <= M; ++m) T[m] = (m & (m - 1)) ? T[m & (m - 1)] + p[lowbit_c(m)] : p[lowbit_c(m)];
                    int acc0 = vself, acc1 = kNeg;  // two independent max chains
#pragma unroll
                    for (int m = 1; m <= M; ++m) {
                        const int cm = vb[slp[popc_c(m)] - stream_move_off<K>(m)] + Sp[m];
                        const int cb = carry[m] + T[m];
                        if (m & 1)
                            acc0 = __vimax3_s32(acc0, cm, cb);
                        else
                            acc1 = __vimax3_s32(acc1, cm, cb);
                        carry[m] = cm;
                    }
                    const int acc_all = max(acc0, acc1);
                    const int tm = (Wb0 + s * (1 << NA) - acc_all) & MASKB;
                    const int val = acc_all + tm;
                    if (has_tile && (unsigned)(r0 + s) < (unsigned)rows) tbw[(int64_t)(r0 + s) * 32] = (uint8_t)tm;
                    if (act) {
                        vb[own] = val;
                        vself = val;
                    }
                }
                __syncthreads();
            };
#pragma unroll
            for (int s = 0; s < U; ++s) step(s);
            if (refill) pt_store((b + 1) * U);
            face_write(b);
            __syncthreads();  // the block's face stores precede the count in program order (a hint)
            if (tid == 0 && tagout != 0) st_relaxed(prog + col, b + 1);
            if (want) ok = halo_accept(b + 1, issued);
        };
        for (int b = 0; b < nblk && ok; b += NPAR) {
            block(b, IntC<0>{});
            if constexpr (NPAR > 1)
                if (b + 1 < nblk && ok) block(b + 1, IntC<1 % NPAR>{});
            if constexpr (NPAR > 2)
                if (b + 2 < nblk && ok) block(b + 2, IntC<2 % NPAR>{});
            if constexpr (NPAR > 3)
                if (b + 3 < nblk && ok) block(b + 3, IntC<3 % NPAR>{});
        }
        if (!ok) {
            if (tid == 0) atomicCAS(L.err, 0, MSA_ETIMEOUT);
            break;
        }
        // the corner's key: position len of the line holding the far corner
        {
            bool corner = true;
#pragma unroll
            for (int i = 0; i < NA; ++i) corner = corner && o[i] + cl[i] == P.len[i];
            if (corner) *P.qcorner = V[vbase + rslot(lens + sig)];
        }
    }
}

template <int K>
cudaError_t stream_attributes() {
    static DeviceOnce once;
    return once.run([] {
        return cudaFuncSetAttribute(fill_lines_stream_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    stream_smem_bytes<K>());
    });
}

template <int K>
cudaError_t launch_stream(const LaunchDesc &L, int grid, cudaStream_t s) {
    cudaError_t e = stream_attributes<K>();
    if (e != cudaSuccess) return e;
    fill_lines_stream_kernel<K><<<grid, stream_threads<K>(), stream_smem_bytes<K>(), s>>>(L);
    return cudaGetLastError();
}

template <int K>
int stream_ctas() {
    if (stream_attributes<K>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fill_lines_stream_kernel<K>, stream_threads<K>(),
                                                      stream_smem_bytes<K>()) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace msadp
