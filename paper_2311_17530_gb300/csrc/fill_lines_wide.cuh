// Whole-column super-block fill for k = 6 with a short last axis (rho_s <= Z):
// the line kernel's sweep (fill_lines.cuh: lane l of a warp owns one line of a
// 32-line block, skewed by the sum of its local coordinates; candidates of the
// moves that also advance the last axis s are carried from the previous step)
// on the streamed kernel's super-blocks (fill_lines_stream.cuh: a CTA of 4 warps
// owns 4 x 4 x 2 x 2 x 2 lines and sweeps them in lockstep, one barrier per
// step), with the halo exchanged as plain values once per column:
//
// * Shared memory holds the halo'd super-block (local coordinates -1 .. SB_i - 1)
//   indexed by POSITION: line h at word sum_i h_i A_i, its position z at word
//   + z + 1 (word 0 is position -1, "no cell"). At step t lane c reads position
//   t - sigma(c) of its predecessor lines; the 32 lanes of a warp hit 32 banks
//   when sum_i c_i (A_i - 1) is distinct mod 32 over a line block (strides found
//   by exhaustive search, footprint within 1 % of the unpadded box).
// * A column waits for the completion flags of its face neighbours along the
//   line axes (their own waits make the diagonal neighbours complete as well),
//   loads its 547 halo lines' positions in 16-byte groups from their producers'
//   faces, sweeps rho_s + SMAX steps, writes its upper-face lines back (every
//   position, line-major), and publishes its flag with a release store after a
//   CTA barrier. Per halo value that is a quarter of a 16-byte load and one
//   shared store, against a tagged 8-byte entry, its check and its ring store
//   per value in the pipelined form; a column cannot start before its
//   producers have finished theirs, which on a last axis of 25 positions costs
//   less than the per-block exchange.
//
// Global memory: the traceback bytes of each line block (layout 3 spanning the
// whole last axis, as the streamed kernel), the faces of each super-block: its
// upper-face lines, line-major, ZQ = rho_s rounded up to 4 positions each.
#pragma once

#include "device_common.cuh"

namespace msadp {


// Strides (words) of the line axes in the position-indexed super-block box.
__host__ __device__ constexpr int wide_stride(int K, int i) {
    constexpr int k6[] = {26, 393, 131, 1965, 5905};
    return k6[i] + 0 * K;
}
template <int K>
__host__ __device__ constexpr int wide_move_off(int m) {
    int s = 0;
    for (int i = 0; i < K - 1; ++i)
        if ((m >> i) & 1) s += wide_stride(K, i);
    return s;
}
template <int K>
__host__ __device__ constexpr int wide_v_words() {
    // the last word any line's positions -1 .. Z - 1 use, plus one, plus the 3
    // words past the last position that a face write-back's last group reads
    int s = kWideZ + 1;
    for (int i = 0; i < K - 1; ++i) s += stream_sb(K, i) * wide_stride(K, i);
    return round_up(s + 3, 4);
}
template <int K>
struct WideLayout {
    static constexpr int NA = K - 1;
    static constexpr int NT = 32 * stream_warps(K);
    static constexpr int NHL = [] {
        int n = 1;
        for (int i = 0; i < K - 1; ++i) n *= stream_sb(K, i) + 1;
        return n;
    }();
    static constexpr int NH = NHL - NT;
    static constexpr int NFL = stream_face_lines(K);
    static constexpr int NROW = [] {
        int n = 0;
        for (int i = 0; i < K - 1; ++i) n += stream_sb(K, i);
        return n;
    }();
    // pair-table rows: positions 0 .. Z - 1, row stride congruent to a line
    // block's skew + 1 mod 32 (lanes of one row read different positions)
    static constexpr int ZS = [] {
        int s = kWideZ;
        while (s % 32 != (line_skew_max(K) + 1) % 32) ++s;
        return s;
    }();
    static constexpr int PT = 0;
    static constexpr int HDESC = PT + round_up(NROW * ZS, 4);  // halo lines: base | face line << 15 | S << 22
    static constexpr int FTAB = HDESC + round_up(NH, 4);       // face lines: base
    static constexpr int NB = FTAB + round_up(NFL, 4);
    static constexpr int CROW = NB + round_up(1 << NA, 4);
    static constexpr int MISC = CROW + round_up(NROW, 4);
    static constexpr int V = MISC + 8;  // reads at most SMAX - 1 words below the box stay in the tables
    static constexpr int WORDS = V + wide_v_words<K>();
};
template <int K>
__host__ __device__ constexpr int wide_smem_bytes() {
    return WideLayout<K>::WORDS * 4;
}
template <int K>
__host__ __device__ constexpr int wide_min_ctas() {
    int c = (228 * 1024) / (wide_smem_bytes<K>() + 1024);
    return c < 1 ? 1 : c;
}

template <int K>
__global__ void __launch_bounds__(stream_threads<K>(), wide_min_ctas<K>()) fill_lines_wide_kernel(const LaunchDesc L) {
    using LY = WideLayout<K>;
    constexpr int NA = K - 1;
    constexpr int M = (1 << NA) - 1;
    constexpr int NT = LY::NT, NH = LY::NH, NHL = LY::NHL, NFL = LY::NFL, NROW = LY::NROW, ZS = LY::ZS;
    constexpr int SMAX = stream_skew_max(K);
    constexpr int MASKB = (1 << K) - 1;
    constexpr int HB = 8;  // halo loads in flight per thread
    static_assert(SMAX < LY::V && wide_v_words<K>() < (1 << 15) && NFL < 128 && M < 32, "geometry");

    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t *sm = reinterpret_cast<int32_t *>(smem_raw);
    int32_t *PT = sm + LY::PT;
    uint32_t *hdesc = reinterpret_cast<uint32_t *>(sm + LY::HDESC);
    int32_t *ftab = sm + LY::FTAB;
    int32_t *nb = sm + LY::NB;
    int32_t *crow = sm + LY::CROW;
    volatile int32_t *misc = sm + LY::MISC;  // [0] ticket, [1] wait verdict
    int32_t *V = sm + LY::V;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // Once per CTA: the face lines (some c_i = SB_i - 1) in line order with their
    // box bases, then every halo line (some digit h_i = 0) with its base, the
    // number of its producer's face line (c_i = SB_i - 1 where h_i = 0, h_i - 1
    // elsewhere) and the subset S of axes at -1 (which neighbour produces it).
    if (tid == 0) {
        int32_t *fnum = V;  // a line's face number (-1: none), kept in the box until it is used
        int nf = 0;
        for (int j = 0; j < NT; ++j) {
            int rem = j, base = 0;
            bool face = false;
            for (int i = NA - 1; i >= 0; --i) {
                const int c = rem % stream_sb(K, i);
                rem /= stream_sb(K, i);
                base += (c + 1) * wide_stride(K, i);
                face = face || c == stream_sb(K, i) - 1;
            }
            fnum[j] = face ? nf : -1;
            if (face) ftab[nf++] = base;
        }
        int n = 0;
        for (int j = 0; j < NHL; ++j) {
            int rem = j, base = 0, lp = 0, lstr = 1;
            uint32_t S = 0;
            for (int i = NA - 1; i >= 0; --i) {
                const int h = rem % (stream_sb(K, i) + 1);
                rem /= stream_sb(K, i) + 1;
                base += h * wide_stride(K, i);
                lp += (h == 0 ? stream_sb(K, i) - 1 : h - 1) * lstr;
                lstr *= stream_sb(K, i);
                if (h == 0) S |= 1u << i;
            }
            if (S) hdesc[n++] = (uint32_t)base | (uint32_t)fnum[lp] << 15 | S << 22;
        }
    }

    // this thread's line: warp and lane coordinates, box base, skew
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
            vbase += (cl[i] + 1) * wide_stride(K, i);
            sig += cl[i];
            sigw += cw[i] * line_ext(K, i);
        }
    }

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
        if (pidx != cached_prob) {
            cached_prob = pidx;
            cached_live = ld_volatile(&P.istat->status) == 0;
        }
        if (!cached_live) continue;  // a failed problem: its columns read and publish nothing

        int sco[NA], o[NA];
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
        const int rho = P.rho[NA], cofs = P.cofs[NA];
        const int ZQ = (rho + 3) & ~3;  // words per face line
        const int NQ = ZQ / 4;
        const int64_t FB = (int64_t)NFL * ZQ;
        const int32_t *Fq = P.Q;
        int32_t *Fo = P.Q + (int64_t)col * FB;
        int32_t *const done = L.done + P.tile_base;

        int64_t tile = 0;
        bool has_tile = true;
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            const int g = sco[i] * stream_wg(K, i) + cw[i];
            has_tile = has_tile && g < P.G[i];
            tile += (int64_t)g * P.gstride[i];
        }

        // neighbour super-blocks, pair-table rows' residue codes, position -1 of
        // every box line
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
        for (int j = tid; j < NHL; j += NT) {
            int rem = j, base = 0;
#pragma unroll
            for (int i = NA - 1; i >= 0; --i) {
                base += (rem % (stream_sb(K, i) + 1)) * wide_stride(K, i);
                rem /= stream_sb(K, i) + 1;
            }
            V[base] = kNeg;
        }
        // this line's pair sums over subsets of the line axes
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
        __syncthreads();  // nb and crow are read below
        // pair tables of the last axis against every line axis, positions 0 .. rho - 1
        for (int it = tid; it < NROW * rho; it += NT) {
            const int row = it / rho, z = it - row * rho;
            const int cz = z >= 1 ? codes[cofs + z - 1] : 0;
            PT[row * ZS + z] = __ldg(tab + crow[row] * A + cz);
        }
        // face neighbours along the line axes (one lane each); their completion
        // implies that of every diagonal neighbour
        if (warp == 0) {
            bool ok = true;
            if (lane < NA && sco[lane] > 0) ok = wait_at_least(done + nb[1 << lane], 1, L.err, L.spin_ns);
            ok = __all_sync(kFull, ok);
            if (lane == 0) misc[1] = ok;
        }
        __syncthreads();  // the waiting lanes' acquires precede every thread's halo loads
        if (!misc[1]) {
            if (tid == 0) atomicCAS(L.err, 0, MSA_ETIMEOUT);
            break;
        }

        // the halo: positions 0 .. rho - 1 of every halo line, 4 at a time
        for (int i0 = 0; i0 < NH * NQ; i0 += NT * HB) {
            int4 val[HB];
            int dst[HB];
#pragma unroll
            for (int u = 0; u < HB; ++u) {
                const int it = i0 + NT * u + tid;
                dst[u] = -1;
                val[u] = make_int4(kNeg, kNeg, kNeg, kNeg);
                if (it < NH * NQ) {
                    const int j = it / NQ, q = it - j * NQ;
                    const uint32_t e = hdesc[j];
                    const int src = nb[e >> 22];
                    dst[u] = (int)(e & 0x7FFF) + 1 + 4 * q;
                    if (src >= 0)
                        val[u] = __ldcg(reinterpret_cast<const int4 *>(Fq + (int64_t)src * FB +
                                                                       (int)((e >> 15) & 127) * ZQ + 4 * q));
                }
            }
#pragma unroll
            for (int u = 0; u < HB; ++u)
                if (dst[u] >= 0) {
                    const int it = i0 + NT * u + tid;
                    const int n = rho - 4 * (it - (it / NQ) * NQ);  // positions left on the line
                    V[dst[u]] = val[u].x;
                    if (n > 1) V[dst[u] + 1] = val[u].y;
                    if (n > 2) V[dst[u] + 2] = val[u].z;
                    if (n > 3) V[dst[u] + 3] = val[u].w;
                }
        }
        __syncthreads();

        // The sweep: rho + SMAX steps, one barrier each. Every lane reads its own
        // skewed position, in range or not (a read below position -1 or past the
        // last position feeds only candidates that are overwritten or never
        // stored); the origin's lane starts from H(0) = 0 as its previous position.
        int Wl = -sig * (1 << NA);  // W(x) = Wl + t 2^NA at step t
#pragma unroll
        for (int i = 0; i < NA; ++i) Wl += (o[i] + cl[i]) << i;
        int ptoff[NA];
        {
            int row = 0;
#pragma unroll
            for (int i = 0; i < NA; ++i) {
                ptoff[i] = (row + cl[i]) * ZS;
                row += stream_sb(K, i);
            }
        }
        int carry[M + 1];
        int vself = col == 0 && tid == 0 ? 0 : kNeg;
#pragma unroll
        for (int m = 1; m <= M; ++m) carry[m] = kNeg + Sp[m];
        const int rows = P.tb_block / 32;
        uint8_t *tbw = P.tb + tile * P.tb_block + lane;
        const int nsteps = rho + SMAX;
        for (int ts = 0; ts < nsteps; ++ts) {
            if ((unsigned)(ts - sigw) < (unsigned)(rho + line_skew_max(K))) {
                const int z = ts - sig;
                const bool act = (unsigned)z < (unsigned)rho;
                const int zp = z < 0 ? 0 : (z >= rho ? rho - 1 : z);
                int p[NA];
#pragma unroll
                for (int i = 0; i < NA; ++i) p[i] = PT[ptoff[i] + zp];
                int T[M + 1];
                T[0] = 0;
#pragma unroll
                for (int m = 1; m <= M; ++m) T[m] = (m & (m - 1)) ? T[m & (m - 1)] + p[lowbit_c(m)] : p[lowbit_c(m)];
                const int32_t *vp = V + vbase + z + 1;
                int acc0 = vself, acc1 = kNeg;
#pragma unroll
                for (int m = 1; m <= M; ++m) {
                    const int cm = vp[-wide_move_off<K>(m)] + Sp[m];
                    const int cb = carry[m] + T[m];
                    if (m & 1)
                        acc0 = __vimax3_s32(acc0, cm, cb);
                    else
                        acc1 = __vimax3_s32(acc1, cm, cb);
                    carry[m] = cm;
                }
                const int acc = max(acc0, acc1);
                const int tm = (Wl + ts * (1 << NA) - acc) & MASKB;
                const int val = acc + tm;
                const int r = ts - sigw;
                if (has_tile && r < rows) tbw[(int64_t)r * 32] = (uint8_t)tm;
                if (act) {
                    V[vbase + z + 1] = val;
                    vself = val;
                }
            }
            __syncthreads();
        }

        // faces for the successors: every position of the upper-face lines
        for (int it = tid; it < NFL * NQ; it += NT) {
            const int f = it / NQ, q = it - f * NQ;
            const int32_t *s = V + ftab[f] + 1 + 4 * q;
            *reinterpret_cast<int4 *>(Fo + (int64_t)f * ZQ + 4 * q) = make_int4(s[0], s[1], s[2], s[3]);
        }
        {
            bool corner = true;
#pragma unroll
            for (int i = 0; i < NA; ++i) corner = corner && o[i] + cl[i] == P.len[i];
            if (corner) *P.qcorner = V[vbase + rho];
        }
        __syncthreads();  // every thread's face stores precede the release
        if (tid == 0 && (int64_t)t != L.withhold) st_release(done + col, 1);
    }
}

template <int K>
cudaError_t wide_attributes() {
    static DeviceOnce once;
    return once.run([] {
        return cudaFuncSetAttribute(fill_lines_wide_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    wide_smem_bytes<K>());
    });
}

template <int K>
cudaError_t launch_wide(const LaunchDesc &L, int grid, cudaStream_t s) {
    cudaError_t e = wide_attributes<K>();
    if (e != cudaSuccess) return e;
    fill_lines_wide_kernel<K><<<grid, stream_threads<K>(), wide_smem_bytes<K>(), s>>>(L);
    return cudaGetLastError();
}

template <int K>
int wide_ctas() {
    if (wide_attributes<K>() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fill_lines_wide_kernel<K>, stream_threads<K>(),
                                                      wide_smem_bytes<K>()) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace msadp
