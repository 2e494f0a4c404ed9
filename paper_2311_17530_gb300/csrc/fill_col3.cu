// k = 3 column kernel: the fill of section 2 for three sequences, organised as
// a skewed register pipeline instead of independent tiles.
//
// Geometry. Axis 0 (sequence 0) is split into CTA blocks of WR = W * R rows: warp
// w of a CTA owns rows x0 = A*WR + w*R + r (r < R) in registers. Axis 1 is split
// into blocks of 32: lane l owns x1 = 32*B + l. Axis 2 (the last, fastest axis)
// is swept: at warp step t, lane l computes for each of its rows r the cell at
// x2 = j = t - l - r. With this skew every predecessor of a cell was computed one
// or two steps earlier by the same lane (rows r and r-1), by lane l-1 (received
// with a warp shuffle), by the warp above (through a shared-memory ring), or by a
// neighbouring CTA (through global "faces", below). The warps of a CTA run in
// lockstep, warp w lagging warp w-1 by R steps, one __syncthreads per step.
//
// Faces between CTAs, written in skewed layouts so that every read and write is
// one contiguous row:
//   F0[cta][p + l][l]       last row of the CTA (x0 = A*WR + WR - 1) at x1 = 32B+l, x2 = p
//   F1[cta][p + rho][rho]   last lane (x1 = 32B + 31) of CTA row rho at x2 = p
// A CTA publishes how many of its lockstep steps are complete in a progress
// counter; a consumer waits (bounded) until the producer is far enough ahead and
// stages the next chunk of faces into shared memory with cp.async, one chunk
// ahead of use.
//
// Cell update (packed keys, see internal.h): with pair scores scaled by 2^3,
//   Q(x) = max( Q(x-e0), Q(x-e1), Q(x-e2),
//               Q(x-e0-e1) + p01, Q(x-e0-e2) + p02, Q(x-e1-e2) + p12,
//               Q(x-e0-e1-e2) + p01 + p02 + p12 )
// then m* = (W(x) - max) mod 8 and Q(x) = max + m*; m* is the traceback byte.
// Traceback bytes are packed four positions per word and stored to the row-major
// traceback tensor as aligned 32-bit words.
#include "api_internal.h"
#include "device_common.cuh"

namespace msadp {

struct C3Smem {
    int32_t ring[c3::W][c3::S][32];   // row -1 values of each warp, by lockstep step
    int32_t f1[c3::S][c3::WR];        // axis-1 face of CTA (A, B-1)
    int32_t corner0[c3::S][4];        // last row of CTA (A-1, B-1) at its last lane
    int32_t ctl[4];
    int32_t cur_prob;
};

int col3_warps_per_cta() { return c3::W; }

__device__ __forceinline__ void c3_cp16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void c3_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void c3_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void c3_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// byte-insert selectors: put the low byte of the second operand at byte b
__device__ __forceinline__ constexpr unsigned c3_ins(int b) {
    return b == 0 ? 0x3214u : b == 1 ? 0x3240u : b == 2 ? 0x3410u : 0x4210u;
}

struct C3Col {
    // column-constant state
    int A, B, nsteps, TS;
    int rho0, rho1, rho2, len2;
    const int32_t *f0src, *f1src, *c0src;  // producer faces (nullptr: none)
    int32_t *f0dst, *f1dst;                // this column's faces
    int32_t *prog;                          // progress counters of this problem
    int pA1, pB1, pAB1;                     // producer column indices (-1: none)
    int me;
};

// Stage chunk c's faces into the shared rings (all threads; one commit group).
__device__ __forceinline__ void c3_stage(C3Smem &sm, const C3Col &cc, int c, int tid) {
    const int T0 = c * c3::CH;
    // F0 of (A-1, B): rows X in [T0, T0+CH) -> ring[0][(X-1) & (S-1)], 8 x 16 B per row
    if (cc.f0src) {
        for (int i = tid; i < c3::CH * 8; i += c3::THREADS) {
            const int X = T0 + i / 8, part = i % 8;
            c3_cp16(&sm.ring[0][(X - 1) & (c3::S - 1)][part * 4], cc.f0src + (int64_t)X * 32 + part * 4);
        }
    }
    // F1 of (A, B-1): rows X in [T0, T0+CH) -> f1[X & (S-1)], 16 x 16 B per row
    if (cc.f1src) {
        for (int i = tid; i < c3::CH * 16; i += c3::THREADS) {
            const int X = T0 + i / 16, part = i % 16;
            c3_cp16(&sm.f1[X & (c3::S - 1)][part * 4], cc.f1src + (int64_t)X * c3::WR + part * 4);
        }
    }
    // corner for warp 0 lane 0: F1 of (A-1, B-1) at row X + WR - 1, entries WR-4..WR-1
    if (cc.c0src) {
        for (int i = tid; i < c3::CH; i += c3::THREADS) {
            const int X = T0 + i;
            c3_cp16(&sm.corner0[X & (c3::S - 1)][0],
                    cc.c0src + (int64_t)(X + c3::WR - 1) * c3::WR + (c3::WR - 4));
        }
    }
    c3_commit();
}

// Wait (thread 0) until the producers have completed the steps chunk c reads.
__device__ __forceinline__ bool c3_wait_producers(const C3Col &cc, int c, const LaunchDesc &L) {
    const int Xmax = c * c3::CH + c3::CH - 1;
    bool ok = true;
    if (cc.pA1 >= 0) ok = ok && wait_at_least(&cc.prog[cc.pA1], min(cc.nsteps, Xmax + c3::WR), L.err, L.spin_ns);
    if (cc.pB1 >= 0) ok = ok && wait_at_least(&cc.prog[cc.pB1], min(cc.nsteps, Xmax + 32), L.err, L.spin_ns);
    if (cc.pAB1 >= 0)
        ok = ok && wait_at_least(&cc.prog[cc.pAB1], min(cc.nsteps, Xmax + c3::WR - 1 + 32), L.err, L.spin_ns);
    return ok;
}

// Per-warp register state of one column.
struct C3Regs {
    int V[3][c3::R];      // own values by generation (step mod 3)
    int U[3][c3::R];      // values received from lane l-1
    int VM[3], UM[3];     // row -1 (warp above), own lane and lane l-1
    int code[c3::R];      // axis-2 code of each row's current position
    unsigned cur[c3::R];  // traceback bytes being packed (4 positions)
    unsigned prv[c3::R];  // previous packed word
};

template <bool MASK, int s>
__device__ __forceinline__ void c3_step(C3Regs &g, C3Smem &sm, const int *__restrict__ tabr,
                                        const int (&rowoff)[c3::R], int laneoff, const int (&p01)[c3::R],
                                        const int (&Wc)[c3::R], const unsigned char *sc2, int T, int t,
                                        int lane, int w, unsigned rowvalid, bool lanevalid, int rho2,
                                        unsigned char *tbl, const int (&tbro)[c3::R], const unsigned (&selA)[4],
                                        int32_t *f0dst, int32_t *f1dst, bool origin) {
    constexpr int cur = s % 3, prv = (s + 2) % 3, pv2 = (s + 1) % 3;
    // receive lane l-1's values of the previous step; lane 0 takes the axis-1 face
    const int4 fa = *reinterpret_cast<const int4 *>(&sm.f1[T & (c3::S - 1)][w * c3::R]);
    const int4 fb = *reinterpret_cast<const int4 *>(&sm.f1[T & (c3::S - 1)][w * c3::R + 4]);
    const int fl[8] = {fa.x, fa.y, fa.z, fa.w, fb.x, fb.y, fb.z, fb.w};
#pragma unroll
    for (int r = 0; r < c3::R; ++r) {
        const int v = __shfl_up_sync(kFull, g.V[prv][r], 1);
        g.U[cur][r] = lane == 0 ? fl[r] : v;
    }
    // row -1 from the warp above (or the staged face of CTA (A-1, B))
    g.VM[cur] = sm.ring[w][(T - 1) & (c3::S - 1)][lane];
    {
        const int um = sm.ring[w][(T - 2) & (c3::S - 1)][(lane + 31) & 31];
        const int cw = w == 0 ? sm.corner0[T & (c3::S - 1)][3] : sm.f1[(T - 1) & (c3::S - 1)][w * c3::R - 1];
        g.UM[cur] = lane == 0 ? cw : um;
    }
    // shift the per-row axis-2 codes: row r now sits one position behind row r-1
#pragma unroll
    for (int r = c3::R - 1; r > 0; --r) g.code[r] = g.code[r - 1];
    g.code[0] = sc2[t - lane];
    const int t4 = 4 * t;
    const int jl = t - lane;
#pragma unroll
    for (int r = 0; r < c3::R; ++r) {
        const int c2 = g.code[r] << 7;  // table stride per code: 32 lanes * 4 bytes
        const int p02 = *reinterpret_cast<const int *>(reinterpret_cast<const char *>(tabr) + rowoff[r] + c2);
        const int p12 = *reinterpret_cast<const int *>(reinterpret_cast<const char *>(tabr) + laneoff + c2);
        const int v1m = r == 0 ? g.VM[cur] : g.V[prv][r - 1];
        const int v2m = r == 0 ? g.VM[prv] : g.V[pv2][r - 1];
        const int u1m = r == 0 ? g.UM[cur] : g.U[prv][r - 1];
        const int u2m = r == 0 ? g.UM[prv] : g.U[pv2][r - 1];
        int acc = max(max(v1m, g.U[cur][r]), g.V[prv][r]);
        acc = max(acc, u1m + p01[r]);
        acc = max(acc, v2m + p02);
        acc = max(acc, g.U[prv][r] + p12);
        acc = max(acc, u2m + (p01[r] + p02 + p12));
        // strip the tie bits: Q = W + ceil8(acc - W), m* = Q - acc
        const int wx = Wc[r] + t4;
        int q = ((acc - wx + 7) & ~7) + wx;
        int m = q - acc;
        if (MASK) {
            const bool valid = (unsigned)(jl - r) < (unsigned)rho2;
            q = valid ? q : kNeg;
            if (r == 0 && origin && jl == 0) {  // H(0) = 0, no move
                q = 0;
                m = 0;
            }
        }
        g.V[cur][r] = q;
        g.cur[r] = __byte_perm(g.cur[r], (unsigned)m, c3_ins(s & 3));
    }
    // faces: last row of the warp feeds the warp below; last lane feeds CTA (A, B+1)
    if (w + 1 < c3::W) {
        sm.ring[w + 1][T & (c3::S - 1)][lane] = g.V[cur][c3::R - 1];
    } else if (T - c3::WR + 1 >= 0) {
        f0dst[(int64_t)(T - c3::WR + 1) * 32 + lane] = g.V[cur][c3::R - 1];
    }
    if (lane == 31 && T >= 31) {
        int4 *d = reinterpret_cast<int4 *>(f1dst + (int64_t)(T - 31) * c3::WR + w * c3::R);
        d[0] = make_int4(g.V[cur][0], g.V[cur][1], g.V[cur][2], g.V[cur][3]);
        d[1] = make_int4(g.V[cur][4], g.V[cur][5], g.V[cur][6], g.V[cur][7]);
    }
    // every 4th step: store the aligned 4-position word of every row
    if ((s & 3) == 3) {
        const int base = jl - 3;  // positions [jl-r-3, jl-r] were packed in cur[r]
#pragma unroll
        for (int r = 0; r < c3::R; ++r) {
            const unsigned word = __byte_perm(g.prv[r], g.cur[r], selA[r & 3]);
            const int q0 = (base - r) & ~3;  // aligned start (see selA)
            const bool ok = ((rowvalid >> r) & 1) && lanevalid && (!MASK || (q0 >= 0 && q0 < rho2));
            if (ok) *reinterpret_cast<unsigned *>(tbl + tbro[r] + q0) = word;
            g.prv[r] = g.cur[r];
        }
    }
}

template <bool MASK>
__device__ __forceinline__ void c3_chunk(C3Regs &g, C3Smem &sm, const int *__restrict__ tabr,
                                         const int (&rowoff)[c3::R], int laneoff, const int (&p01)[c3::R],
                                         const int (&Wc)[c3::R], const unsigned char *sc2, int T0, int lane,
                                         int w, unsigned rowvalid, bool lanevalid, int rho2, int TS,
                                         unsigned char *tbl, const int (&tbro)[c3::R],
                                         const unsigned (&selA)[4], int32_t *f0dst, int32_t *f1dst,
                                         bool origin) {
#define C3_STEP(s)                                                                                        \
    {                                                                                                     \
        const int T = T0 + (s), t = T - w * c3::R;                                                        \
        if (t >= 0 && t < TS)                                                                             \
            c3_step<MASK, (s)>(g, sm, tabr, rowoff, laneoff, p01, Wc, sc2, T, t, lane, w, rowvalid,        \
                               lanevalid, rho2, tbl, tbro, selA, f0dst, f1dst, origin);                    \
        __syncthreads();                                                                                  \
    }
    C3_STEP(0) C3_STEP(1) C3_STEP(2) C3_STEP(3) C3_STEP(4) C3_STEP(5)
    C3_STEP(6) C3_STEP(7) C3_STEP(8) C3_STEP(9) C3_STEP(10) C3_STEP(11)
#undef C3_STEP
}

__global__ void __launch_bounds__(c3::THREADS, 1) fill_col3_kernel(const LaunchDesc L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C3Smem &sm = *reinterpret_cast<C3Smem *>(smem_raw);
    int *tabr = reinterpret_cast<int *>(smem_raw + sizeof(C3Smem));
    unsigned char *sc2base = reinterpret_cast<unsigned char *>(tabr + L.tab_ints);  // axis-2 codes

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) sm.cur_prob = -1;
    __syncthreads();

    while (true) {
        if (tid == 0) {
            sm.ctl[0] = atomicAdd(L.ticket, 1);
            sm.ctl[1] = ld_volatile(L.err);
        }
        __syncthreads();
        const int ticket = sm.ctl[0];
        const int errnow = sm.ctl[1];
        __syncthreads();
        if ((int64_t)ticket >= L.ntickets || errnow != 0) break;

        const uint64_t ent = L.order[ticket];
        const int pidx = (int)(ent >> 32);
        const ProblemDesc &P = L.probs[pidx];
        const int lin = (int)(uint32_t)ent;
        const int NB = P.G[1];
        C3Col cc;
        cc.A = lin / NB;
        cc.B = lin - cc.A * NB;
        cc.me = lin;
        cc.rho0 = P.rho[0];
        cc.rho1 = P.rho[1];
        cc.rho2 = P.rho[2];
        cc.len2 = P.len[2];
        cc.TS = cc.rho2 + c3::R + 31 + c3::EXTRA;
        cc.nsteps = c3::nsteps(cc.rho2);
        const int nchunks = cc.nsteps / c3::CH;
        cc.prog = L.done + P.tile_base;
        const int32_t *F0 = P.Q;
        const int32_t *F1 = P.aux;
        cc.f0dst = P.Q + (int64_t)lin * P.face0_stride;
        cc.f1dst = P.aux + (int64_t)lin * P.face1_stride;
        cc.pA1 = cc.A > 0 ? lin - NB : -1;
        cc.pB1 = cc.B > 0 ? lin - 1 : -1;
        cc.pAB1 = (cc.A > 0 && cc.B > 0) ? lin - NB - 1 : -1;
        cc.f0src = cc.pA1 >= 0 ? F0 + (int64_t)cc.pA1 * P.face0_stride : nullptr;
        cc.f1src = cc.pB1 >= 0 ? F1 + (int64_t)cc.pB1 * P.face1_stride : nullptr;
        cc.c0src = cc.pAB1 >= 0 ? F1 + (int64_t)cc.pAB1 * P.face1_stride : nullptr;
        const bool live = ld_volatile(&P.istat->status) == 0;

        if (live) {
            const int A = P.A;
            // replicated pair table (entry-major, one copy per lane) and axis-2 codes
            const int have = sm.cur_prob;
            __syncthreads();
            if (have != pidx)
                for (int i = tid; i < A * A * 32; i += c3::THREADS) tabr[i] = P.tab[i >> 5];
            if (tid == 0) sm.cur_prob = pidx;
            for (int i = tid; i < cc.rho2 + 2 * c3::CODEPAD + 32; i += c3::THREADS) {
                const int j = i - c3::CODEPAD;  // position x2 = j consumes residue j - 1
                sc2base[i] = (j >= 1 && j <= cc.len2) ? P.codes[P.cofs[2] + j - 1] : (unsigned char)0;
            }
            // rings start at "no predecessor"
            for (int i = tid; i < c3::W * c3::S * 32; i += c3::THREADS) (&sm.ring[0][0][0])[i] = kNeg;
            for (int i = tid; i < c3::S * c3::WR; i += c3::THREADS) (&sm.f1[0][0])[i] = kNeg;
            for (int i = tid; i < c3::S * 4; i += c3::THREADS) (&sm.corner0[0][0])[i] = kNeg;
            __syncthreads();

            // column constants of this lane
            const int x1 = cc.B * 32 + lane;
            const bool lanevalid = x1 < cc.rho1;
            const int code1 = (x1 >= 1 && x1 <= P.len[1]) ? P.codes[P.cofs[1] + x1 - 1] : 0;
            const int x0b = cc.A * c3::WR + w * c3::R;
            int rowoff[c3::R], p01[c3::R], Wc[c3::R], tbro[c3::R];
            unsigned rowvalid = 0;
#pragma unroll
            for (int r = 0; r < c3::R; ++r) {
                const int x0 = x0b + r;
                const int code0 = (x0 >= 1 && x0 <= P.len[0]) ? P.codes[P.cofs[0] + x0 - 1] : 0;
                rowoff[r] = (code0 * A * 32 + lane) * 4;
                p01[r] = P.tab[code0 * A + code1];
                // W(x) = x0 + 2 x1 + 4 x2 with x2 = t - lane - r
                Wc[r] = x0 + 2 * x1 - 4 * lane - 4 * r;
                if (x0 < cc.rho0) rowvalid |= 1u << r;
                tbro[r] = (int)((int64_t)r * P.tbstride[0]);
            }
            const int laneoff = (code1 * A * 32 + lane) * 4;
            unsigned char *tbl = P.tb + (int64_t)min(x0b, cc.rho0 - 1) * P.tbstride[0] +
                                 (int64_t)min(x1, cc.rho1 - 1) * P.tbstride[1];
            if (x0b >= cc.rho0) rowvalid = 0;
            // byte selectors aligning a packed word with the 4-aligned positions:
            // row r's word ends at j = t - lane - r with (j - 3) = -(lane + r) mod 4
            unsigned selA[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int o = 4 - ((-(lane + k)) & 3);
                selA[k] = (unsigned)(o | (o + 1) << 4 | (o + 2) << 8 | (o + 3) << 12);
            }

            C3Regs g;
#pragma unroll
            for (int r = 0; r < c3::R; ++r) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    g.V[k][r] = kNeg;
                    g.U[k][r] = kNeg;
                }
                g.code[r] = 0;
                g.cur[r] = 0;
                g.prv[r] = 0;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                g.VM[k] = kNeg;
                g.UM[k] = kNeg;
            }
            const unsigned char *sc2 = sc2base + c3::CODEPAD;
            const bool origin = cc.A == 0 && cc.B == 0 && w == 0 && lane == 0;

            // prologue: stage chunk 0
            if (tid == 0) sm.ctl[2] = c3_wait_producers(cc, 0, L) ? 0 : 1;
            __syncthreads();
            bool failed = sm.ctl[2] != 0;
            if (!failed) c3_stage(sm, cc, 0, tid);
            for (int c = 0; c < nchunks && !failed; ++c) {
                // prefetch chunk c+1 while chunk c computes
                if (c + 1 < nchunks) {
                    if (tid == 0) sm.ctl[2] = c3_wait_producers(cc, c + 1, L) ? 0 : 1;
                    __syncthreads();
                    if (sm.ctl[2] != 0) {
                        failed = true;
                        break;
                    }
                    c3_stage(sm, cc, c + 1, tid);
                    c3_wait_prev();
                } else {
                    c3_wait_all();
                }
                __syncthreads();
                const int T0 = c * c3::CH;
                const int t0 = T0 - w * c3::R;
                // interior chunk for this warp: every (lane, row) position inside [4, rho2)
                const bool interior = t0 - 31 - (c3::R - 1) >= 7 && t0 + c3::CH - 1 <= cc.rho2 - 1;
                if (interior)
                    c3_chunk<false>(g, sm, tabr, rowoff, laneoff, p01, Wc, sc2, T0, lane, w, rowvalid, lanevalid,
                                    cc.rho2, cc.TS, tbl, tbro, selA, cc.f0dst, cc.f1dst, origin);
                else
                    c3_chunk<true>(g, sm, tabr, rowoff, laneoff, p01, Wc, sc2, T0, lane, w, rowvalid, lanevalid,
                                   cc.rho2, cc.TS, tbl, tbro, selA, cc.f0dst, cc.f1dst, origin);
                // publish progress (all steps of the chunk are done: the last step ended in a barrier)
                if (tid == 0 && (int64_t)ticket != L.withhold) {
                    __threadfence();
                    st_release(&cc.prog[cc.me], T0 + c3::CH);
                }
            }
            c3_wait_all();
            __syncthreads();
            if (failed) {
                if (tid == 0) atomicCAS(L.err, 0, MSA_ETIMEOUT);
                break;
            }
        } else {
            if (tid == 0 && (int64_t)ticket != L.withhold) {
                __threadfence();
                st_release(&cc.prog[cc.me], cc.nsteps);
            }
        }
        __syncthreads();
    }
}

// Dynamic shared memory: rings and face staging, the replicated pair table
// (A*A entries x 32 lanes) and the padded axis-2 codes.
int col3_smem_bytes(int alphabet_size) {
    return (int)sizeof(C3Smem) + alphabet_size * alphabet_size * 32 * 4 + c3::MAXRHO2 + 2 * c3::CODEPAD + 48;
}

int fill_col3_ctas_per_sm(int smem) {
    if (cudaFuncSetAttribute(fill_col3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fill_col3_kernel, c3::THREADS, smem) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_fill_col3(const LaunchDesc &L, int grid, int smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(fill_col3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    fill_col3_kernel<<<grid, c3::THREADS, smem, s>>>(L);
    return cudaGetLastError();
}

}  // namespace msadp
