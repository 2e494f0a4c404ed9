// k = 3 column kernel: the fill of section 2 for three sequences, organised as a
// skewed register pipeline instead of independent tiles.
//
// Geometry (see c3:: in internal.h). A CTA owns the column (A, B): CTA rows
// rho = w*R + r (x0 = A*WR + rho) held by warp w in registers, lanes l
// (x1 = 32B + l), and it sweeps axis 2. At CTA time T lane l of warp w computes
// row r's cell at x2 = T - l - rho. Then, for the cell computed at time T+1,
//   e0  (x0-1)          is row rho-1 at time T        (same lane; warp above: ring)
//   e2  (x2-1)          is row rho   at time T        (same lane, same register)
//   e1  (x1-1)          is lane l-1 at time T         (shuffle at time T+1)
//   e01, e12            are lane l-1 at time T-1      (shuffled at time T)
//   e02                 is row rho-1 at time T-1
//   e012                is lane l-1, row rho-1 at time T-2 (shuffled at time T-1)
// so each step first finishes its own cells -- the max of a pre-reduced candidate
// P and the freshly shuffled e1 candidate, then the tie-bit strip -- and then
// prepares P for time T+1 and the e02/e012 pair D for time T+2 from values it
// already holds. Only the shuffle, one max and the strip sit on the step-to-step
// dependency chain.
//
// Communication, all indexed by CTA time T (so every index inside an unrolled
// block of U steps is a compile-time offset):
//   ring[w][T]  row -1 of warp w at time T: (value, tag T) written by warp w-1
//               (its last row), or by the staging warp for w = 0 (the column
//               above, face F0 at its time T + WR). A reader accepts an entry
//               when its tag is T, so warps never wait on a barrier.
//   f1r[T]      lane 0's inputs from the column to the left (its lane 31 at
//               time T + 31) and the corner from the column above-left, copied
//               by the staging warp, which publishes how far it got.
//   F0, F1      global faces of this column, (value, tag) 8-byte entries whose
//               tag carries the launch epoch: no flags and no fences.
// A column runs CTA times -U .. nsteps - 1; the first block computes cells at
// x2 < 0 only, so that the candidates of time 0 and 1 are prepared like any
// other (their e0/e01/e02/e012 predecessors belong to the columns above and to
// the left). Traceback bytes and faces are stored from T = -U on (offset U).
//
// Cells outside the tensor are computed like any other. Positions x2 <= 0 take a
// sentinel code whose pair scores are kSentinelPair, and every value starts at
// kNeg, so such cells stay far below every valid key (the encode kernel's range
// check keeps that margin); the origin's pre-reduced candidate is set to
// H(0) = 0 when time 0 begins.
//
// Cell update with pair scores scaled by 2^3 (packed keys, see internal.h): the
// max over the seven moves gives the key, then m* = (W(x) - max) mod 8 and
// Q(x) = max + m*; m* is the traceback byte. Each lane stores its R bytes of a
// step as one word, 32 * R contiguous bytes per warp step.
#include "api_internal.h"
#include "device_common.cuh"

namespace msadp {

struct C3Smem {
    unsigned long long ring[c3::W][c3::SI][32];  // row -1 of warp w by CTA time: (value, tag)
    int32_t f1r[c3::SF][c3::F1S];                // lane-0 inputs by CTA time: [3 + rho'], rho' = -1 .. WR-1
    int32_t prog[c3::W];                         // compute warp w has finished the steps < prog[w]
    int32_t staged;                              // f1r rows < staged hold this column's values
    int32_t failed;                              // a wait ran out: every warp leaves the column
    int32_t ctl[2];
    int32_t cur_prob;
    int32_t pad[3];
};

int col3_warps_per_cta() { return c3::W + 1; }

namespace {

__device__ __forceinline__ unsigned long long pack_entry(int value, int tag) {
    return (unsigned long long)(unsigned)value | ((unsigned long long)(unsigned)tag << 32);
}
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long lds_u64_volatile(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.volatile.shared.u64 %0, [%1];" : "=l"(v) : "r"(smem_addr(p)));
    return v;
}
__device__ __forceinline__ int ld_acquire_shared(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_shared(int32_t *p, int v) {
    asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ int vload(const int32_t *p) { return *reinterpret_cast<const volatile int32_t *>(p); }
__device__ __forceinline__ void vstore(int32_t *p, int v) { *reinterpret_cast<volatile int32_t *>(p) = v; }
// generic address: a shared ring slot or a global face entry
__device__ __forceinline__ void st_entry(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.u64 [%0], %1;" ::"l"(p), "l"(v));
}
__device__ __forceinline__ void st_global_v2(unsigned long long *p, unsigned long long a, unsigned long long b) {
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b));
}
__device__ __forceinline__ unsigned long long ld_global_relaxed(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ ulonglong2 ld_global_relaxed_v2(const unsigned long long *p) {
    ulonglong2 v;
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ int ldtab(const char *tab, int byte_off) {
    return *reinterpret_cast<const int *>(tab + byte_off);
}

// Mark the column failed (first failure wins the launch status).
__device__ void c3_fail(C3Smem &sm, const LaunchDesc &L) {
    vstore(&sm.failed, 1);
    atomicCAS(L.err, 0, MSA_ETIMEOUT);
}

// Slow path of a ring read: wait (bounded) until every lane's entry carries tag T.
__device__ __noinline__ unsigned long long c3_ring_wait(const unsigned long long *p, int T, C3Smem &sm,
                                                       const LaunchDesc &L) {
    const uint64_t t0 = global_ns();
    unsigned long long e = lds_u64_volatile(p);
    while (__any_sync(kFull, (int)(e >> 32) != T)) {
        if (vload(&sm.failed) || (int64_t)(global_ns() - t0) > L.spin_ns) {
            if ((threadIdx.x & 31) == 0) c3_fail(sm, L);
            return pack_entry(kNeg, T);
        }
        __nanosleep(20);
        e = lds_u64_volatile(p);
    }
    return e;
}

// Registers of one compute lane that change from step to step.
struct C3St {
    int V[c3::R];       // V(T-1, r) on entry to step T, V(T, r) after it
    int P[c3::R];       // max over every candidate of cell (T, r) but e1
    int D[c3::R];       // max of the e02 and e012 candidates of cell (T+1, r)
    int cc[2 * c3::R];  // byte offsets of axis-2 codes: shift register by position
    int pp[2 * c3::R];  // pair scores (x1, x2) of those positions
    int VM;             // V(T-1, -1): the ring entry of the previous step
};

// Constants of one compute lane for a column.
struct C3Ln {
    int p01[c3::R];     // pair score (x0, x1) per row
    int rowb[c3::R];    // byte offset of row r's table row (code of x0) plus 4 * lane
    int laneb;          // byte offset of this lane's table row (code of x1) plus 4 * lane
    int Wl;             // W(x) = Wl + 4T - 3r
    int wR;             // first CTA row of the warp
    int tagout;         // tag base of ring-out entries (0: shared ring, epoch << 16: global face)
    int tagf1;          // tag base of this column's F1 entries
    bool last;          // lane 31 writes the F1 face
    int ctime;          // CTA time at which this lane computes the far corner (else never)
    int crow;           // the corner's row among this lane's R rows
    int32_t *qcorner;   // where the corner's key goes (for the traceback's cross-check)
};

// Per-block addresses (block = U steps starting at CTA time T0).
struct C3Blk {
    const unsigned long long *rin;  // ring[w][T0 mod SI][lane]
    unsigned long long *rout;       // ring[w+1][T0 mod SI][lane] or F0[T0][lane] (generic)
    const int *f1row;               // f1r[T0 mod SF]
    unsigned char *tbp;             // traceback bytes of (T0, w, lane): R bytes
    unsigned long long *f1o;        // F1[T0][wR]
    const uint16_t *c2p;            // code offset of x2 = T0 + 2 - lane - wR
};

template <int s>
__device__ __forceinline__ void c3_step(C3St &g, const C3Ln &c, const char *tab, const C3Blk &b, int T0, int lane,
                                        C3Smem &sm, const LaunchDesc &L) {
    constexpr int M = 2 * c3::R - 1;
    constexpr int R = c3::R;
    static_assert(R == 2 || R == 4, "rows per warp: 2 or 4");
    const int T = T0 + s;
    // U(T, r) from lane l-1 (lane 0: the staged face)
    const int *fr = b.f1row + s * c3::F1S;
    int fv[R];
    if constexpr (R == 4) {
        const int4 f = *reinterpret_cast<const int4 *>(fr + 4 + c.wR);
        fv[0] = f.x, fv[1] = f.y, fv[2] = f.z, fv[3] = f.w;
    } else {
        const int2 f = *reinterpret_cast<const int2 *>(fr + 4 + c.wR);
        fv[0] = f.x, fv[1] = f.y;
    }
    const int fm = fr[3 + c.wR];
    int Un[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int v = __shfl_up_sync(kFull, g.V[r], 1);
        Un[r] = lane == 0 ? fv[r] : v;
    }
    int UMn = __shfl_up_sync(kFull, g.VM, 1);
    if (lane == 0) UMn = fm;
    // the cells of time T
    const int WT = c.Wl + 4 * T;
    unsigned pk = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int acc = max(g.P[r], Un[r]);
        const int m = (WT - 3 * r - acc) & 7;
        g.V[r] = acc + m;
        pk |= (unsigned)m << (8 * r);
    }
    // outputs: last row to the warp below (or face F0), traceback bytes, lane 31 to face F1
    st_entry(b.rout + s * 32, pack_entry(g.V[R - 1], c.tagout + T));
    if constexpr (R == 4)
        *reinterpret_cast<uint32_t *>(b.tbp + s * (c3::W * 32 * R)) = pk;
    else
        *reinterpret_cast<uint16_t *>(b.tbp + s * (c3::W * 32 * R)) = (uint16_t)pk;
    if (c.last) {
        const int tg = c.tagf1 + T;
#pragma unroll
        for (int r = 0; r < R; r += 2)
            st_global_v2(b.f1o + s * c3::WR + r, pack_entry(g.V[r], tg), pack_entry(g.V[r + 1], tg));
    }
    // code of the position x2 = T + 2 - lane - wR (row 0 of time T + 2)
    const int cn = b.c2p[s];
    g.cc[s & M] = cn;
    g.pp[s & M] = ldtab(tab, c.laneb + cn);
    // row -1: V(T, -1) from the ring (written by the warp above at its time T)
    unsigned long long e = lds_u64_volatile(b.rin + s * 32);
    if (__any_sync(kFull, (int)(e >> 32) != T)) e = c3_ring_wait(b.rin + s * 32, T, sm, L);
    const int VMn = (int)(unsigned)e;
    // P of time T + 1 and D of time T + 2
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int vm = r ? g.V[r - 1] : VMn;
        const int um = r ? Un[r - 1] : UMn;
        const int y = um + c.p01[r];
        int pn = max(max(g.D[r], vm), max(g.V[r], y));
        pn = max(pn, Un[r] + g.pp[(s - r - 1) & M]);
        const int p02 = ldtab(tab, c.rowb[r] + g.cc[(s - r) & M]);
        const int p12 = g.pp[(s - r) & M];
        g.D[r] = max(vm + p02, y + p02 + p12);
        g.P[r] = pn;
    }
    g.VM = VMn;
}

// A step of the block that holds the far corner's CTA time (kernels that record
// the corner): the plain step, then the corner's lane stores its row's key.
template <int s>
__device__ __forceinline__ void c3_capture_step(C3St &g, const C3Ln &c, const char *tab, const C3Blk &b, int T0,
                                                int lane, C3Smem &sm, const LaunchDesc &L) {
    c3_step<s>(g, c, tab, b, T0, lane, sm, L);
    if (T0 + s == c.ctime) {
        // a select chain (R is 2 or 4): a loop over r would index the registers dynamically
        const int v = c.crow == 0 ? g.V[0] : c.crow == 1 ? g.V[1] : c.crow == 2 ? g.V[2 % c3::R] : g.V[c3::R - 1];
        __stcg(c.qcorner, v);
    }
}

struct C3Col {
    int A, B, N;
    const unsigned long long *f0up, *f1left, *f1diag;  // producer faces (nullptr: none)
    unsigned long long *f0dst, *f1dst;                  // this column's faces
    int tagbase;                                        // (epoch << 16) of this launch
};

// Staging warp: copy the column's inputs from the producer columns' faces into
// ring[0] and f1r, as soon as their tags show this launch's values, and publish
// the number of CTA-time rows staged. Positions a producer never computes (past
// its last step, or no producer at all) are staged as kNeg. A batch covers SB
// rows: every load of the batch is issued before any tag is checked (one L2 round
// trip per batch). Loads are 16-byte pairs of entries: an F0 row (32 entries) is
// read by half a warp, an F1 row (WR entries) by WR / 2 lanes.
__device__ void c3_stager(C3Smem &sm, const C3Col &cc, int lane, const LaunchDesc &L) {
    constexpr int SB = 8;                        // rows per batch (one block: measured best)
    constexpr int NL0 = SB / 2;                  // F0 loads per lane and batch (2 rows per load)
    constexpr int LPR1 = c3::WR / 2;             // lanes per F1 row
    constexpr int RPI1 = 32 / LPR1;              // F1 rows per load
    constexpr int NL1 = SB / RPI1;               // F1 loads per lane and batch
    static_assert(SB <= c3::SI - c3::U && SB <= c3::SF - c3::U, "staging batch exceeds the rings");
    static_assert(SB % RPI1 == 0 && 32 % LPR1 == 0, "F1 rows per load");
    const int half = lane >> 4, pair0 = 2 * (lane & 15);            // F0: row parity, first entry
    const int sub1 = lane / LPR1, pair1 = 2 * (lane % LPR1);        // F1: row in the load, first entry
    const unsigned rowmask1 = LPR1 == 32 ? 0xffffffffu : ((1u << LPR1) - 1);
    int Ts = -c3::U;
    uint64_t t_progress = global_ns();
    while (Ts < cc.N) {
        // the slots to fill must have been read by the compute warps
        {
            const int need0 = Ts + SB - c3::SI, needall = Ts + SB - c3::SF;
            int ok;
            while (true) {
                const int pw = lane < c3::W ? ld_acquire_shared(&sm.prog[lane]) : (1 << 30);
                const int pmin = __reduce_min_sync(kFull, pw);
                const int p0 = __shfl_sync(kFull, pw, 0);
                ok = p0 >= need0 && pmin >= needall;
                if (ok) break;
                if (vload(&sm.failed) || (int64_t)(global_ns() - t_progress) > L.spin_ns) break;
                __nanosleep(64);
            }
            if (!ok) {
                if (lane == 0 && !vload(&sm.failed)) c3_fail(sm, L);
                return;
            }
        }
        // issue every load of the batch
        ulonglong2 a[NL0], b[NL1];
        unsigned long long d = pack_entry(kNeg, 0);
        const ulonglong2 none = make_ulonglong2(pack_entry(kNeg, 0), pack_entry(kNeg, 0));
#pragma unroll
        for (int i = 0; i < NL0; ++i) {
            const int T = Ts + 2 * i + half;
            a[i] = none;
            if (cc.f0up && T + c3::WR < cc.N)
                a[i] = ld_global_relaxed_v2(cc.f0up + (int64_t)(T + c3::WR + c3::U) * 32 + pair0);
        }
#pragma unroll
        for (int i = 0; i < NL1; ++i) {
            const int T = Ts + RPI1 * i + sub1;
            b[i] = none;
            if (cc.f1left && T + 31 < cc.N)
                b[i] = ld_global_relaxed_v2(cc.f1left + (int64_t)(T + 31 + c3::U) * c3::WR + pair1);
        }
        {
            const int T = Ts + lane;  // lane i fetches the corner of row Ts + i
            if (lane < SB && cc.f1diag && T + 31 + c3::WR < cc.N)
                d = ld_global_relaxed(cc.f1diag + (int64_t)(T + 31 + c3::WR + c3::U) * c3::WR + c3::WR - 1);
        }
        // rows whose entries all carry this launch's tag
        unsigned rows_ok = 0;
#pragma unroll
        for (int i = 0; i < NL0; ++i) {
            const int T = Ts + 2 * i + half;
            bool v = true;
            if (cc.f0up && T + c3::WR < cc.N) {
                const int want = cc.tagbase + T + c3::WR;
                v = (int)(a[i].x >> 32) == want && (int)(a[i].y >> 32) == want;
            }
            const unsigned bal = __ballot_sync(kFull, v);
            rows_ok |= ((bal & 0xffffu) == 0xffffu ? 1u : 0u) << (2 * i);
            rows_ok |= ((bal >> 16) == 0xffffu ? 1u : 0u) << (2 * i + 1);
        }
        unsigned rows_ok1 = 0;
#pragma unroll
        for (int i = 0; i < NL1; ++i) {
            const int T = Ts + RPI1 * i + sub1;
            bool v = true;
            if (cc.f1left && T + 31 < cc.N) {
                const int want = cc.tagbase + T + 31;
                v = (int)(b[i].x >> 32) == want && (int)(b[i].y >> 32) == want;
            }
            const unsigned bal = __ballot_sync(kFull, v);
#pragma unroll
            for (int q = 0; q < RPI1; ++q)
                rows_ok1 |= (((bal >> (q * LPR1)) & rowmask1) == rowmask1 ? 1u : 0u) << (RPI1 * i + q);
        }
        rows_ok &= rows_ok1;
        {
            const int T = Ts + lane;
            const bool v = lane >= SB || !cc.f1diag || T + 31 + c3::WR >= cc.N ||
                           (int)(d >> 32) == cc.tagbase + T + 31 + c3::WR;
            rows_ok &= __ballot_sync(kFull, v) & ((1u << SB) - 1);
        }
        const int n = rows_ok == (1u << SB) - 1 ? SB : __ffs(~rows_ok) - 1;  // rows ready, in order
#pragma unroll
        for (int i = 0; i < NL0; ++i) {
            const int r = 2 * i + half;
            if (r < n) {
                const int T = Ts + r;
                *reinterpret_cast<ulonglong2 *>(&sm.ring[0][T & (c3::SI - 1)][pair0]) =
                    make_ulonglong2(pack_entry((int)(unsigned)a[i].x, T), pack_entry((int)(unsigned)a[i].y, T));
            }
        }
#pragma unroll
        for (int i = 0; i < NL1; ++i) {
            const int r = RPI1 * i + sub1;
            if (r < n) {
                const int T = Ts + r;
                *reinterpret_cast<int2 *>(&sm.f1r[T & (c3::SF - 1)][4 + pair1]) =
                    make_int2((int)(unsigned)b[i].x, (int)(unsigned)b[i].y);
            }
        }
        if (lane < n) sm.f1r[(Ts + lane) & (c3::SF - 1)][3] = (int)(unsigned)d;
        if (n > 0) {
            Ts += n;
            __syncwarp();
            if (lane == 0) st_release_shared(&sm.staged, Ts);
            t_progress = global_ns();
        } else {
            if (vload(&sm.failed) || ld_volatile(L.err) != 0 || (int64_t)(global_ns() - t_progress) > L.spin_ns) {
                if (lane == 0 && !vload(&sm.failed)) c3_fail(sm, L);
                return;
            }
            __nanosleep(64);
        }
    }
}

// Block prologue of a compute warp: publish progress, then wait (bounded) until
// the staged face covers the block and the warp below has freed the ring slots.
__device__ __forceinline__ bool c3_block_wait(C3Smem &sm, int w, int T0, const LaunchDesc &L) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) st_release_shared(&sm.prog[w], T0);
    const int need_st = T0 + c3::U;
    const int need_dn = T0 + c3::U - c3::SI;
    const bool lastw = w == c3::W - 1;
    if (ld_acquire_shared(&sm.staged) >= need_st && (lastw || ld_acquire_shared(&sm.prog[w + 1]) >= need_dn))
        return true;
    const uint64_t t0 = global_ns();
    while (true) {
        __nanosleep(32);
        if (ld_acquire_shared(&sm.staged) >= need_st && (lastw || ld_acquire_shared(&sm.prog[w + 1]) >= need_dn))
            return true;
        if (vload(&sm.failed)) return false;
        if ((int64_t)(global_ns() - t0) > L.spin_ns) {
            if ((threadIdx.x & 31) == 0) c3_fail(sm, L);
            return false;
        }
    }
}

}  // namespace

// CAP: the warp that computes the far corner records its key for the traceback's
// cross-check; the block holding it runs a capturing copy of the steps (which
// costs registers, so plain launches use the kernel without it).
template <bool CAP>
__global__ void __launch_bounds__(c3::THREADS, 1) fill_col3_kernel(const LaunchDesc L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C3Smem &sm = *reinterpret_cast<C3Smem *>(smem_raw);
    int *tabr = reinterpret_cast<int *>(smem_raw + sizeof(C3Smem));
    uint16_t *c2off = reinterpret_cast<uint16_t *>(tabr + L.tab_ints);  // axis-2 code offsets by x2 + CODEPAD

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
        cc.N = c3::nsteps(P.rho[2]);
        const int64_t f0s = P.face0_stride / 2, f1s = P.face1_stride / 2;  // entries per column face
        unsigned long long *F0 = reinterpret_cast<unsigned long long *>(P.Q);
        unsigned long long *F1 = reinterpret_cast<unsigned long long *>(P.aux);
        cc.f0dst = F0 + (int64_t)lin * f0s;
        cc.f1dst = F1 + (int64_t)lin * f1s;
        cc.f0up = cc.A > 0 ? F0 + (int64_t)(lin - NB) * f0s : nullptr;
        cc.f1left = cc.B > 0 ? F1 + (int64_t)(lin - 1) * f1s : nullptr;
        cc.f1diag = (cc.A > 0 && cc.B > 0) ? F1 + (int64_t)(lin - NB - 1) * f1s : nullptr;
        cc.tagbase = L.epoch << 16;
        // a withheld column (test hook) writes faces no reader accepts
        const int tag_faces = (int64_t)ticket == L.withhold ? 0 : cc.tagbase;

        const int A = P.A;
        // replicated pair table (entry-major, one copy per lane) with a sentinel
        // code A for positions x2 <= 0, and the axis-2 code offsets
        const int have = sm.cur_prob;
        __syncthreads();
        if (have != pidx)
            for (int i = tid; i < A * (A + 1) * 32; i += c3::THREADS) {
                const int c0 = i / ((A + 1) * 32), c2 = (i >> 5) % (A + 1);
                tabr[i] = c2 == A ? c3::kSentinelPair : P.tab[c0 * A + c2];
            }
        if (tid == 0) {
            sm.cur_prob = pidx;
            sm.staged = -c3::U;
            sm.failed = 0;
        }
        if (tid < c3::W) sm.prog[tid] = -c3::U;
        const int len2 = P.len[2];
        for (int i = tid; i < P.rho[2] + 2 * c3::CODEPAD + 16; i += c3::THREADS) {
            const int x2 = i - c3::CODEPAD;  // position x2 consumes residue x2 - 1
            const int code = x2 <= 0 ? A : x2 <= len2 ? P.codes[P.cofs[2] + x2 - 1] : 0;
            c2off[i] = (uint16_t)(code * 128);
        }
        // ring entries start with a tag no step uses
        for (int i = tid; i < c3::W * c3::SI * 32; i += c3::THREADS)
            (&sm.ring[0][0][0])[i] = pack_entry(kNeg, 0x7fffffff);
        __syncthreads();

        if (stager) {
            c3_stager(sm, cc, lane, L);
        } else {
            const bool lastw = w == c3::W - 1;
            C3Ln c;
            c.wR = w * c3::R;
            c.last = lane == 31;
            c.tagout = lastw ? tag_faces : 0;
            c.tagf1 = tag_faces;
            const int x1 = cc.B * 32 + lane;
            const int code1 = (x1 >= 1 && x1 <= P.len[1]) ? P.codes[P.cofs[1] + x1 - 1] : 0;
            const int x0b = cc.A * c3::WR + c.wR;
#pragma unroll
            for (int r = 0; r < c3::R; ++r) {
                const int x0 = x0b + r;
                const int code0 = (x0 >= 1 && x0 <= P.len[0]) ? P.codes[P.cofs[0] + x0 - 1] : 0;
                c.rowb[r] = (code0 * (A + 1) * 32 + lane) * 4;
                c.p01[r] = P.tab[code0 * A + code1];
            }
            c.laneb = (code1 * (A + 1) * 32 + lane) * 4;
            c.Wl = cc.A * c3::WR + 64 * cc.B - 2 * lane - 3 * c.wR;
            {  // the far corner (len0, len1, len2): row rho of lane l at CTA time len2 + l + rho
                const int rhoc = P.len[0] - cc.A * c3::WR, lc = P.len[1] - 32 * cc.B;
                const bool mine = rhoc >= c.wR && rhoc < c.wR + c3::R && lc == lane;
                c.ctime = mine ? P.len[2] + lc + rhoc : (int)0x80000000;
                c.crow = rhoc - c.wR;
                c.qcorner = P.qcorner;
            }
            const char *tab = reinterpret_cast<const char *>(tabr);
            const uint16_t *c2lane = c2off + c3::CODEPAD + 2 - lane - c.wR;  // x2 = T + 2 - lane - wR at T

            C3St g;
#pragma unroll
            for (int r = 0; r < c3::R; ++r) {
                g.V[r] = kNeg;
                g.P[r] = kNeg;
                g.D[r] = kNeg;
            }
            const bool origin = cc.A == 0 && cc.B == 0 && w == 0 && lane == 0;
            g.VM = kNeg;
            // shift registers before time -U: positions x2 = 2 - U - lane - wR - j, j = 1 .. 2R-1
#pragma unroll
            for (int j = 1; j < 2 * c3::R; ++j) {
                const int cj = c2lane[-c3::U - j];
                g.cc[(-j) & (2 * c3::R - 1)] = cj;
                g.pp[(-j) & (2 * c3::R - 1)] = ldtab(tab, c.laneb + cj);
            }
            g.cc[0] = g.pp[0] = 0;

            unsigned long long *ringout = lastw ? cc.f0dst + lane : &sm.ring[w + 1][0][lane];
            unsigned char *tbw = P.tb + (int64_t)lin * c3::tb_col_bytes(P.rho[2]) + (w * 32 + lane) * c3::R;
            // the block of the corner's CTA time, the same in every lane of its warp
            int T0c = -2 * c3::U;
            if (CAP) {
                const int ct = __shfl_sync(kFull, c.ctime, (P.len[1] - 32 * cc.B) & 31);
                if (ct != (int)0x80000000) T0c = ct / c3::U * c3::U;
            }
            for (int T0 = -c3::U; T0 < cc.N; T0 += c3::U) {
                if (!c3_block_wait(sm, w, T0, L)) break;
                if (T0 == 0 && origin) g.P[0] = 0;  // H(0) = 0, no move
                C3Blk b;
                b.rin = &sm.ring[w][T0 & (c3::SI - 1)][lane];
                b.rout = lastw ? ringout + (int64_t)(T0 + c3::U) * 32 : ringout + (T0 & (c3::SI - 1)) * 32;
                b.f1row = &sm.f1r[T0 & (c3::SF - 1)][0];
                b.tbp = tbw + (int64_t)(T0 + c3::U) * (c3::W * 32 * c3::R);
                b.f1o = cc.f1dst + (int64_t)(T0 + c3::U) * c3::WR + c.wR;
                b.c2p = c2lane + T0;
                if (!CAP || T0 != T0c) {
                    c3_step<0>(g, c, tab, b, T0, lane, sm, L);
                    c3_step<1>(g, c, tab, b, T0, lane, sm, L);
                    c3_step<2>(g, c, tab, b, T0, lane, sm, L);
                    c3_step<3>(g, c, tab, b, T0, lane, sm, L);
                    c3_step<4>(g, c, tab, b, T0, lane, sm, L);
                    c3_step<5>(g, c, tab, b, T0, lane, sm, L);
                    c3_step<6>(g, c, tab, b, T0, lane, sm, L);
                    c3_step<7>(g, c, tab, b, T0, lane, sm, L);
                } else {
                    c3_capture_step<0>(g, c, tab, b, T0, lane, sm, L);
                    c3_capture_step<1>(g, c, tab, b, T0, lane, sm, L);
                    c3_capture_step<2>(g, c, tab, b, T0, lane, sm, L);
                    c3_capture_step<3>(g, c, tab, b, T0, lane, sm, L);
                    c3_capture_step<4>(g, c, tab, b, T0, lane, sm, L);
                    c3_capture_step<5>(g, c, tab, b, T0, lane, sm, L);
                    c3_capture_step<6>(g, c, tab, b, T0, lane, sm, L);
                    c3_capture_step<7>(g, c, tab, b, T0, lane, sm, L);
                }
            }
            __syncwarp();
            if (lane == 0) st_release_shared(&sm.prog[w], 1 << 30);
        }
        __syncthreads();
        if (vload(&sm.failed)) break;
    }
}

// Dynamic shared memory: rings and staged faces, the replicated pair table with
// its sentinel column (A*(A+1) entries x 32 lanes) and the axis-2 code offsets.
int col3_smem_bytes(int alphabet_size) {
    return (int)sizeof(C3Smem) + alphabet_size * (alphabet_size + 1) * 32 * 4 +
           (c3::MAXRHO2 + 2 * c3::CODEPAD + 16) * 2 + 16;
}

// The attribute allows the largest alphabet's layout; set once per device.
cudaError_t col3_attributes() {
    static DeviceOnce once;
    return once.run([] {
        cudaError_t e = cudaFuncSetAttribute(fill_col3_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             col3_smem_bytes(c3::MAXA));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fill_col3_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     col3_smem_bytes(c3::MAXA));
        return e;
    });
}

int fill_col3_ctas_per_sm(int smem) {
    if (col3_attributes() != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fill_col3_kernel<false>, c3::THREADS, smem) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_fill_col3(const LaunchDesc &L, int grid, int smem, cudaStream_t s) {
    cudaError_t e = col3_attributes();
    if (e != cudaSuccess) return e;
    if (smem > col3_smem_bytes(c3::MAXA)) return cudaErrorInvalidValue;
    if (L.corner)
        fill_col3_kernel<true><<<grid, c3::THREADS, smem, s>>>(L);
    else
        fill_col3_kernel<false><<<grid, c3::THREADS, smem, s>>>(L);
    return cudaGetLastError();
}

}  // namespace msadp
