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
// Every face entry is a (value, tag) pair written by one 8-byte store; the tag is
// the launch's epoch, so a reader knows an entry is current from the entry alone
// (no flags, no fences). A ninth "staging" warp per CTA reads the faces its CTA
// needs from its three producer CTAs, waits (bounded) until their tags are
// current, and copies the values into shared rings up to AHEAD chunks ahead of
// the eight compute warps, which only ever wait on a shared counter.
//
// Cell update (packed keys, see internal.h): with pair scores scaled by 2^3,
//   Q(x) = max( Q(x-e0), Q(x-e1), Q(x-e2),
//               Q(x-e0-e1) + p01, Q(x-e0-e2) + p02, Q(x-e1-e2) + p12,
//               Q(x-e0-e1-e2) + p01 + p02 + p12 )
// then m* = (W(x) - max) mod 8 and Q(x) = max + m*; m* is the traceback byte.
// Each lane stores its R traceback bytes of a step as one 8-byte word into the
// column-blocked traceback layout (see c3::tb_col_bytes), 256 contiguous bytes
// per warp step.
#include "api_internal.h"
#include "device_common.cuh"

namespace msadp {

struct C3Smem {
    int32_t ring0[c3::S][32];          // staged F0 of (A-1, B): row X at slot (X - 1) & (S - 1)
    int32_t ringi[c3::W][c3::SI][32];  // warp w-1 -> warp w (index w >= 1), by lockstep step
    int32_t f1[c3::S][c3::WR];         // staged F1 of (A, B-1): row X at slot X & (S - 1)
    int32_t corner0[c3::S];            // F1 of (A-1, B-1), row X + WR - 1, entry WR - 1
    int32_t staged;                    // chunks staged (written by the staging warp)
    int32_t consumed;                  // chunks computed (written by compute thread 0)
    int32_t failed;                    // a wait ran out: every warp leaves the column
    int32_t go;                        // chunk-start decision of compute thread 0
    int32_t ctl[4];
    int32_t cur_prob;
};

int col3_warps_per_cta() { return c3::W + 1; }

__device__ __forceinline__ int vload(const int32_t *p) { return *reinterpret_cast<const volatile int32_t *>(p); }
__device__ __forceinline__ void vstore(int32_t *p, int v) { *reinterpret_cast<volatile int32_t *>(p) = v; }
__device__ __forceinline__ void compute_barrier() { asm volatile("bar.sync 1, %0;" ::"n"(c3::W * 32) : "memory"); }
__device__ __forceinline__ int2 ld_relaxed_v2(const int32_t *p) {
    int2 v;
    asm volatile("ld.relaxed.gpu.global.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p) : "memory");
    return v;
}

struct C3Col {
    int A, B, nsteps, TS;
    int rho0, rho1, rho2, len2;
    const int32_t *f0src, *f1src, *c0src;  // producer faces (nullptr: none)
    int32_t *f0dst, *f1dst;                // this column's faces
};

// Staging warp: copy chunk c's face entries into the shared rings once every
// needed entry carries this launch's tag. Entries outside the tensor (position
// p < 0 or p >= rho2) are never needed and are staged as "no predecessor".
// Returns false when the wait runs out or another warp gave up.
__device__ bool c3_stage_chunk(C3Smem &sm, const C3Col &cc, int c, int lane, int epoch, const LaunchDesc &L) {
    const int T0 = c * c3::CH;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        constexpr int H = (c3::WR + 31) / 32;  // F1 entries per lane and row
        int f0v[c3::CH], f1v[c3::CH][H], cv = kNeg;
        bool ok = true;
#pragma unroll
        for (int i = 0; i < c3::CH; ++i) {
            const int X = T0 + i;
            // F0 entry (X, lane): position X - lane
            int v = kNeg;
            if (cc.f0src && (unsigned)(X - lane) < (unsigned)cc.rho2) {
                const int2 e = ld_relaxed_v2(cc.f0src + (int64_t)X * c3::F0W + 2 * lane);
                ok = ok && e.y == epoch;
                v = e.x;
            }
            f0v[i] = v;
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const int rho = lane + 32 * h;  // F1 entry (X, rho): position X - rho
                int u = kNeg;
                if (cc.f1src && rho < c3::WR && (unsigned)(X - rho) < (unsigned)cc.rho2) {
                    const int2 e = ld_relaxed_v2(cc.f1src + (int64_t)X * c3::F1W + 2 * rho);
                    ok = ok && e.y == epoch;
                    u = e.x;
                }
                f1v[i][h] = u;
            }
        }
        if (lane < c3::CH) {  // corner: F1 of (A-1, B-1) row X + WR - 1, entry WR - 1: position X
            const int X = T0 + lane;
            if (cc.c0src && (unsigned)X < (unsigned)cc.rho2) {
                const int2 e = ld_relaxed_v2(cc.c0src + (int64_t)(X + c3::WR - 1) * c3::F1W + 2 * (c3::WR - 1));
                ok = ok && e.y == epoch;
                cv = e.x;
            }
        }
        if (__all_sync(kFull, ok)) {
#pragma unroll
            for (int i = 0; i < c3::CH; ++i) {
                const int X = T0 + i;
                sm.ring0[(X - 1) & (c3::S - 1)][lane] = f0v[i];
#pragma unroll
                for (int h = 0; h < H; ++h)
                    if (lane + 32 * h < c3::WR) sm.f1[X & (c3::S - 1)][lane + 32 * h] = f1v[i][h];
            }
            if (lane < c3::CH) sm.corner0[(T0 + lane) & (c3::S - 1)] = cv;
            return true;
        }
        if ((it & 7) == 7) {
            if (vload(&sm.failed) || ld_volatile(L.err) != 0) return false;
            if ((int64_t)(global_ns() - t0) > L.spin_ns) return false;
        }
        __nanosleep(128);
    }
}

// Per-warp register state of one column.
struct C3Regs {
    int V[3][c3::R];   // own values by generation (step mod 3)
    int U[3][c3::R];   // values received from lane l-1
    int VM[3], UM[3];  // row -1 (warp above), own lane and lane l-1
    int code[c3::R];   // axis-2 code of each row's current position
};

// Column-constant inputs of a compute warp.
struct C3Lane {
    const int *tabr;          // replicated pair table
    int rowoff[c3::R];        // byte offset of row r's table row (code of x0) in tabr
    int laneoff;              // byte offset of this lane's table row (code of x1)
    int p01[c3::R];           // scaled pair score of (x0, x1) per row
    int Wb;                   // W(x) = Wb - 3 r + 4 t for row r at warp step t
    const unsigned char *sc2; // axis-2 codes, indexed by position
    const int32_t *vmring;    // row -1 source: staged face (warp 0) or the warp above
    int vmask;
    unsigned char *tbw;       // this lane's traceback bytes at warp step 0
    int32_t *f0dst, *f1dst;
    int lane, w, rho2, TS, tag;
    bool origin;
};

template <bool MASK, int s>
__device__ __forceinline__ void c3_step(C3Regs &g, C3Smem &sm, const C3Lane &c, int T, int t) {
    constexpr int cur = s % 3, prv = (s + 2) % 3, pv2 = (s + 1) % 3;
    const int lane = c.lane, w = c.w;
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
    g.VM[cur] = c.vmring[((T - 1) & c.vmask) * 32 + lane];
    {
        const int um = c.vmring[((T - 2) & c.vmask) * 32 + ((lane + 31) & 31)];
        const int cw = w == 0 ? sm.corner0[T & (c3::S - 1)] : sm.f1[(T - 1) & (c3::S - 1)][w * c3::R - 1];
        g.UM[cur] = lane == 0 ? cw : um;
    }
    // shift the per-row axis-2 codes: row r now sits one position behind row r-1
#pragma unroll
    for (int r = c3::R - 1; r > 0; --r) g.code[r] = g.code[r - 1];
    g.code[0] = c.sc2[t - lane];
    const int w4 = c.Wb + 4 * t;
    const int jl = t - lane;
    int m8[c3::R];
#pragma unroll
    for (int r = 0; r < c3::R; ++r) {
        const int c2 = g.code[r] << 7;  // table stride per code: 32 lanes * 4 bytes
        const char *tb = reinterpret_cast<const char *>(c.tabr);
        const int p02 = *reinterpret_cast<const int *>(tb + c.rowoff[r] + c2);
        const int p12 = *reinterpret_cast<const int *>(tb + c.laneoff + c2);
        const int v1m = r == 0 ? g.VM[cur] : g.V[prv][r - 1];
        const int v2m = r == 0 ? g.VM[prv] : g.V[pv2][r - 1];
        const int u1m = r == 0 ? g.UM[cur] : g.U[prv][r - 1];
        const int u2m = r == 0 ? g.UM[prv] : g.U[pv2][r - 1];
        // max over the seven moves, as a balanced tree
        const int a = max(v1m, g.U[cur][r]);
        const int b = max(g.V[prv][r], u1m + c.p01[r]);
        const int d = max(v2m + p02, g.U[prv][r] + p12);
        const int e = u2m + (c.p01[r] + p02 + p12);
        const int acc = max(max(a, b), max(d, e));
        // strip the tie bits: Q = W + ceil8(acc - W), m* = Q - acc
        const int wx = w4 - 3 * r;
        int q = ((acc - wx + 7) & ~7) + wx;
        int m = q - acc;
        if (MASK) {
            const bool valid = (unsigned)(jl - r) < (unsigned)c.rho2;
            q = valid ? q : kNeg;
            if (r == 0 && c.origin && jl == 0) {  // H(0) = 0, no move
                q = 0;
                m = 0;
            }
        }
        g.V[cur][r] = q;
        m8[r] = m;
    }
    // traceback bytes of the 8 rows: one 8-byte store per lane, 256 B per warp
    {
        const unsigned lo = (unsigned)m8[0] | (unsigned)m8[1] << 8 | (unsigned)m8[2] << 16 | (unsigned)m8[3] << 24;
        const unsigned hi = (unsigned)m8[4] | (unsigned)m8[5] << 8 | (unsigned)m8[6] << 16 | (unsigned)m8[7] << 24;
        *reinterpret_cast<uint2 *>(c.tbw + (int64_t)t * (c3::W * 32 * c3::R)) = make_uint2(lo, hi);
    }
    // faces: last row of the warp feeds the warp below; last lane feeds CTA (A, B+1)
    if (w + 1 < c3::W) {
        sm.ringi[w + 1][T & (c3::SI - 1)][lane] = g.V[cur][c3::R - 1];
    } else if (T - c3::WR + 1 >= 0) {
        *reinterpret_cast<int2 *>(c.f0dst + (int64_t)(T - c3::WR + 1) * c3::F0W + 2 * lane) =
            make_int2(g.V[cur][c3::R - 1], c.tag);
    }
    if (lane == 31 && T >= 31) {
        int4 *d = reinterpret_cast<int4 *>(c.f1dst + (int64_t)(T - 31) * c3::F1W + 2 * w * c3::R);
        d[0] = make_int4(g.V[cur][0], c.tag, g.V[cur][1], c.tag);
        d[1] = make_int4(g.V[cur][2], c.tag, g.V[cur][3], c.tag);
        d[2] = make_int4(g.V[cur][4], c.tag, g.V[cur][5], c.tag);
        d[3] = make_int4(g.V[cur][6], c.tag, g.V[cur][7], c.tag);
    }
}

template <bool MASK>
__device__ __forceinline__ void c3_chunk(C3Regs &g, C3Smem &sm, const C3Lane &c, int T0) {
#define C3_STEP(s)                                            \
    {                                                         \
        const int T = T0 + (s), t = T - c.w * c3::R;          \
        if (t >= 0 && t < c.TS) c3_step<MASK, (s)>(g, sm, c, T, t); \
        compute_barrier();                                    \
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
    const bool stager = w == c3::W;
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
        if (ld_volatile(&P.istat->status) != 0) continue;  // uniform: every thread reads the same word
        const int lin = (int)(uint32_t)ent;
        const int NB = P.G[1];
        C3Col cc;
        cc.A = lin / NB;
        cc.B = lin - cc.A * NB;
        cc.rho0 = P.rho[0];
        cc.rho1 = P.rho[1];
        cc.rho2 = P.rho[2];
        cc.len2 = P.len[2];
        cc.TS = cc.rho2 + c3::R + 31 + c3::EXTRA;
        cc.nsteps = c3::nsteps(cc.rho2);
        const int nchunks = cc.nsteps / c3::CH;
        cc.f0dst = P.Q + (int64_t)lin * P.face0_stride;
        cc.f1dst = P.aux + (int64_t)lin * P.face1_stride;
        cc.f0src = cc.A > 0 ? P.Q + (int64_t)(lin - NB) * P.face0_stride : nullptr;
        cc.f1src = cc.B > 0 ? P.aux + (int64_t)(lin - 1) * P.face1_stride : nullptr;
        cc.c0src = (cc.A > 0 && cc.B > 0) ? P.aux + (int64_t)(lin - NB - 1) * P.face1_stride : nullptr;
        // a withheld column (test hook) writes faces no reader accepts
        const int tag = (int64_t)ticket == L.withhold ? 0 : L.epoch;

        const int A = P.A;
        // replicated pair table (entry-major, one copy per lane) and axis-2 codes
        const int have = sm.cur_prob;
        __syncthreads();
        if (have != pidx)
            for (int i = tid; i < A * A * 32; i += c3::THREADS) tabr[i] = P.tab[i >> 5];
        if (tid == 0) {
            sm.cur_prob = pidx;
            sm.staged = 0;
            sm.consumed = 0;
            sm.failed = 0;
        }
        for (int i = tid; i < cc.rho2 + 2 * c3::CODEPAD + 32; i += c3::THREADS) {
            const int j = i - c3::CODEPAD;  // position x2 = j consumes residue j - 1
            sc2base[i] = (j >= 1 && j <= cc.len2) ? P.codes[P.cofs[2] + j - 1] : (unsigned char)0;
        }
        // rings start at "no predecessor"
        for (int i = tid; i < c3::S * 32; i += c3::THREADS) (&sm.ring0[0][0])[i] = kNeg;
        for (int i = tid; i < c3::W * c3::SI * 32; i += c3::THREADS) (&sm.ringi[0][0][0])[i] = kNeg;
        for (int i = tid; i < c3::S * c3::WR; i += c3::THREADS) (&sm.f1[0][0])[i] = kNeg;
        for (int i = tid; i < c3::S; i += c3::THREADS) sm.corner0[i] = kNeg;
        __syncthreads();

        if (stager) {
            for (int c = 0; c < nchunks; ++c) {
                // back-pressure: at most AHEAD chunks beyond the compute warps
                const uint64_t t0 = global_ns();
                bool ok = true;
                while (vload(&sm.consumed) <= c - c3::AHEAD) {
                    if (vload(&sm.failed) || ld_volatile(L.err) != 0 ||
                        (int64_t)(global_ns() - t0) > L.spin_ns) {
                        ok = false;
                        break;
                    }
                    __nanosleep(64);
                }
                ok = ok && c3_stage_chunk(sm, cc, c, lane, L.epoch, L);
                if (!ok) {
                    if (lane == 0) {
                        vstore(&sm.failed, 1);
                        atomicCAS(L.err, 0, MSA_ETIMEOUT);
                    }
                    break;
                }
                __syncwarp();
                __threadfence_block();
                if (lane == 0) vstore(&sm.staged, c + 1);
            }
        } else {
            // column constants of this lane
            C3Lane cl;
            cl.lane = lane;
            cl.w = w;
            cl.rho2 = cc.rho2;
            cl.TS = cc.TS;
            cl.tag = tag;
            cl.tabr = tabr;
            cl.f0dst = cc.f0dst;
            cl.f1dst = cc.f1dst;
            const int x1 = cc.B * 32 + lane;
            const int code1 = (x1 >= 1 && x1 <= P.len[1]) ? P.codes[P.cofs[1] + x1 - 1] : 0;
            const int x0b = cc.A * c3::WR + w * c3::R;
#pragma unroll
            for (int r = 0; r < c3::R; ++r) {
                const int x0 = x0b + r;
                const int code0 = (x0 >= 1 && x0 <= P.len[0]) ? P.codes[P.cofs[0] + x0 - 1] : 0;
                cl.rowoff[r] = (code0 * A * 32 + lane) * 4;
                cl.p01[r] = P.tab[code0 * A + code1];
            }
            cl.laneoff = (code1 * A * 32 + lane) * 4;
            // W(x) = x0 + 2 x1 + 4 x2 with x0 = x0b + r, x2 = t - lane - r
            cl.Wb = x0b + 2 * x1 - 4 * lane;
            cl.tbw = P.tb + (int64_t)lin * c3::tb_col_bytes(cc.rho2) + (int64_t)(w * 32 + lane) * c3::R;
            cl.vmring = w == 0 ? &sm.ring0[0][0] : &sm.ringi[w][0][0];
            cl.vmask = w == 0 ? c3::S - 1 : c3::SI - 1;
            cl.sc2 = sc2base + c3::CODEPAD;
            cl.origin = cc.A == 0 && cc.B == 0 && w == 0 && lane == 0;

            C3Regs g;
#pragma unroll
            for (int r = 0; r < c3::R; ++r) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    g.V[k][r] = kNeg;
                    g.U[k][r] = kNeg;
                }
                g.code[r] = 0;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                g.VM[k] = kNeg;
                g.UM[k] = kNeg;
            }

            for (int c = 0; c < nchunks; ++c) {
                if (tid == 0) {
                    const uint64_t t0 = global_ns();
                    int go = 1;
                    while (vload(&sm.staged) <= c) {
                        if (vload(&sm.failed) || (int64_t)(global_ns() - t0) > L.spin_ns) {
                            go = 0;
                            break;
                        }
                        __nanosleep(32);
                    }
                    if (!go) {
                        vstore(&sm.failed, 1);
                        atomicCAS(L.err, 0, MSA_ETIMEOUT);
                    }
                    sm.go = go;
                }
                compute_barrier();
                if (!sm.go) break;
                __threadfence_block();
                const int T0 = c * c3::CH;
                const int t0 = T0 - w * c3::R;
                // interior chunk for this warp: every (lane, row) position inside [1, rho2)
                const bool interior = t0 - 31 - (c3::R - 1) >= 1 && t0 + c3::CH - 1 <= cc.rho2 - 1;
                if (interior)
                    c3_chunk<false>(g, sm, cl, T0);
                else
                    c3_chunk<true>(g, sm, cl, T0);
                if (tid == 0) vstore(&sm.consumed, c + 1);
            }
        }
        __syncthreads();
        if (vload(&sm.failed)) break;
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
