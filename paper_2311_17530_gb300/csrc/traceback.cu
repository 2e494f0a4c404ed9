// Traceback (section 2): from the far corner follow the stored move of every
// cell back to the origin, then score the path.
//
// One CTA of 256 threads per problem. The walk is a chain of dependent reads
// kept in registers:
//   * column layout (k = 3 column kernel): thread 0 walks alone. A window is one
//     bulk copy (cp.async.bulk, completion on an mbarrier) of whole CTA-time
//     rows of a column -- as many times as a diagonal walk needs to leave the
//     column, within a 112 KB buffer. While it walks one buffer, the other
//     receives the window of the column the walk is predicted to enter next,
//     and the other likely windows (the same column further down, the other
//     neighbouring columns) are prefetched into L2. Every move lowers the CTA
//     time T = x2 + l + (x0 mod WR) by its popcount, so a window holds at least
//     its length / 3 moves unless the walk leaves the column;
//   * row-major layout, k <= 3: boxes [x - D, x] staged by the CTA (rows of the
//     last axis copied in 16-byte granules);
//   * k >= 4 (row-major or tile-major; short paths, large boxes): no staging; warp 0
//     loads the traceback bytes of the current cell and of all its predecessors
//     in one round trip, which fixes two moves.
// The walk records only the masks (last column first). The score is computed
// afterwards by the whole CTA: each thread takes a contiguous run of columns,
// the per-axis move counts are prefix-summed to give each column's position, and
// the column scores u*|m| + sum over moved pairs of (sub - 2 gap) are added up.
// For the generic tile kernel the sum is cross-checked against the corner's
// packed key.
#include "api_internal.h"
#include "device_common.cuh"

namespace msadp {
namespace {

constexpr int kTbThreads = 256;
static_assert(c3::W * 32 * c3::R <= kTracebackSmem, "a traceback window holds at least one CTA time");

__device__ __forceinline__ void cp_async_16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

struct WalkState {
    int x[MSA_MAX_K];
    int ncols;
    int fail;
};

// Validates a move at position x and records it; false ends the walk with a failure.
__device__ __forceinline__ bool take_move(int K, int m, int *x, uint8_t *masks, int len_sum, int &ncols) {
    bool bad = m == 0 || (m >> K) != 0 || ncols >= len_sum;
    for (int i = 0; i < K; ++i)
        if (((m >> i) & 1) && x[i] == 0) bad = true;
    if (bad) return false;
    masks[ncols++] = (uint8_t)m;
    for (int i = 0; i < K; ++i) x[i] -= (m >> i) & 1;
    return true;
}

__device__ __forceinline__ bool at_origin(int K, const int *x) {
    for (int i = 0; i < K; ++i)
        if (x[i] != 0) return false;
    return true;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One bulk copy global -> shared whose bytes complete the barrier's current phase.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads of dst come first
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the completion of phase `parity`; false after about a second.
__device__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15) == 15 && global_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}

__device__ __forceinline__ void prefetch_l2(const void *src, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ int lds_u8(unsigned addr) {
    unsigned v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(addr));
    return (int)v;
}
__device__ __forceinline__ void stg_u8(uint8_t *p, int v) {
    asm volatile("st.global.u8 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Column layout of the k = 3 column kernel: inside column (A, B) the byte of the
// cell with CTA row rho and lane l at CTA time T is at
// (T + U) * kRowB + (rho / R) * 32 R + l * R + rho mod R, so the rows of CTA times
// [t_lo, t_hi] are one contiguous run. The walk only moves to lower rows, lanes
// and times inside a column, so a window is usable from any entry point it holds.
// Two window buffers: while thread 0 walks one, the other receives the window of
// the column the walk is predicted to enter next (a mostly diagonal walk leaves
// through whichever of row and lane is smaller, at a CTA time that follows from
// the entry point); a walk that enters anything else loads its window on demand.
struct ColWindow {
    int a, b, t_lo, t_hi;
};

__device__ void walk_col3(const ProblemDesc &P, const IODesc &io, unsigned char *win, WalkState &ws) {
    static_assert(c3::WR == 32 && c3::R == 4, "index arithmetic below assumes WR = 32, R = 4");
    constexpr int kRowB = c3::W * 32 * c3::R;         // bytes of one CTA time of a column
    static_assert(kRowB == 1024, "the walk steps T by shifting the move count by 10");
    constexpr int kBuf = kTracebackSmem / 2;          // one window buffer
    constexpr int kCap = kBuf / kRowB;                // CTA times per window
    constexpr int kAhead = 8;                         // predicted windows end this far above the entry
    __shared__ __align__(8) uint64_t bar[2];
    if (threadIdx.x != 0) return;
    const int NA = P.G[0], NB = P.G[1];
    const int nT = c3::nsteps(P.rho[2]);
    const int64_t colb = c3::tb_col_bytes(P.rho[2]);
    const unsigned char *tb = P.tb;
    uint8_t *masks = io.masks;
    const int len_sum = P.len_sum;
    int x0 = ws.x[0], x1 = ws.x[1], x2 = ws.x[2];
    int ncols = ws.ncols;
    bool fail = ((uintptr_t)tb & 15) != 0;
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    unsigned phase[2] = {0, 0};
    bool inflight[2] = {false, false};
    ColWindow held[2] = {{-1, -1, 0, -1}, {-1, -1, 0, -1}};
    auto load = [&](int i, ColWindow w) {  // rows [t_lo, t_hi] of column (a, b) into buffer i
        bulk_load(win + i * kBuf, tb + (int64_t)(w.a * NB + w.b) * colb + (int64_t)(w.t_lo + c3::U) * kRowB,
                  (unsigned)(w.t_hi - w.t_lo + 1) * kRowB, &bar[i]);
        held[i] = w;
        inflight[i] = true;
    };
    auto land = [&](int i) {  // bounded wait for buffer i's copy
        if (!inflight[i]) return true;
        inflight[i] = false;
        const bool ok = mbar_wait(&bar[i], phase[i]);
        phase[i] ^= 1;
        if (!ok) mbar_wait(&bar[i], phase[i] ^ 1);  // let it land before the CTA may exit
        return ok;
    };
    auto prefetch = [&](int a, int b, int lo, int hi) {  // L2 prefetch, clipped to the column
        if (a < 0 || b < 0 || a >= NA || b >= NB) return;
        lo = max(lo, 0);
        hi = min(hi, nT - 1);
        if (lo <= hi)
            prefetch_l2(tb + (int64_t)(a * NB + b) * colb + (int64_t)(lo + c3::U) * kRowB,
                        (unsigned)(hi - lo + 1) * kRowB);
    };
    int cur = 0;
    while (!fail && (x0 | x1 | x2) != 0) {
        const int A = x0 >> 5, B = x1 >> 5, rho = x0 & 31, l = x1 & 31;
        const int T = x2 + l + rho;
        // the window holding the entry point: the predicted one, else a demand load
        // of as many CTA times as a diagonal walk needs to leave the column
        const int o = 1 - cur;
        if (held[o].a == A && held[o].b == B && T >= held[o].t_lo && T <= held[o].t_hi)
            cur = o;  // buffer cur's copy is landed: it held the previous window
        else
            load(cur, {A, B, max(0, T - min(kCap, 3 * min(rho, l) + 24) + 1), T});
        // predicted next column, and its CTA time at entry after diagonal moves
        const int d = min(rho, l) + 1;
        int pa = A, pb = B, pt;
        if (rho < l) {
            pa = A - 1;
            pt = x2 - d + (l - d) + 31;
        } else if (l < rho) {
            pb = B - 1;
            pt = x2 - d + 31 + (rho - d);
        } else {
            pa = A - 1;
            pb = B - 1;
            pt = x2 - d + 62;
        }
        const int nxt = 1 - cur;
        if (!land(nxt)) {
            fail = true;
            break;
        }
        if (pa >= 0 && pb >= 0 && x2 - d >= 0) {
            const int hi = min(pt + kAhead, nT - 1);
            load(nxt, {pa, pb, max(0, hi - kCap + 1), hi});
        } else {
            held[nxt] = {-1, -1, 0, -1};
        }
        // the other candidates only into L2: further down this column, the other neighbours
        prefetch(A, B, held[cur].t_lo - 48, held[cur].t_lo - 1);
        if (!(pa == A - 1 && pb == B)) prefetch(A - 1, B, pt - 64, pt + kAhead);
        if (!(pa == A && pb == B - 1)) prefetch(A, B - 1, pt - 64, pt + kAhead);
        if (!land(cur)) {
            fail = true;
            break;
        }
        const int t_lo = held[cur].t_lo;
        const unsigned wlo = smem_u32(win + cur * kBuf);
        const unsigned wbase = wlo - (unsigned)(t_lo * kRowB);
        const int before = ncols;
        // The next cell's byte is loaded before this move's checks branch, so the
        // branches resolve under the load's latency; an address below the window
        // is clamped to its first byte (in bounds, unused: the walk leaves).
        unsigned a = wbase + (unsigned)(T * kRowB + (rho >> 2) * (32 * c3::R) + l * c3::R + (rho & 3));
        int m = lds_u8(a);
        while (true) {
            // next address: every moved axis lowers T (kRowB bytes); axis 0 also
            // lowers the row (1 byte, or 125 when it crosses a warp block of R
            // rows), axis 1 the lane (R bytes). The part below kRowB is a byte
            // table indexed by the mask (selected by the row's position in its block).
            const int mm = m & 7;
            const unsigned small = __byte_perm((x0 & 3) ? 0x05040100u : 0x81047d00u,
                                               (x0 & 3) ? 0x05040100u : 0x81047d00u, (unsigned)mm);
            const unsigned an = (unsigned)max((int)a - (__popc(mm) << 10) - (int)small, (int)wlo);
            const int mn = lds_u8(an);
            const int zero = (x0 == 0) | ((x1 == 0) << 1) | ((x2 == 0) << 2);
            const bool bad = ((unsigned)(m - 1) > 6u) | ((m & zero) != 0) | (ncols >= len_sum);
            const int y0 = x0 - (m & 1), y1 = x1 - ((m >> 1) & 1), y2 = x2 - (m >> 2);
            const bool in = ((y0 >> 5) == A) & ((y1 >> 5) == B) & (y2 + (y1 & 31) + (y0 & 31) >= t_lo) &
                            ((y0 | y1 | y2) != 0);
            if (bad) {
                fail = true;
                break;
            }
            stg_u8(masks + ncols, m);
            ++ncols;
            x0 = y0;
            x1 = y1;
            x2 = y2;
            if (!in) break;
            m = mn;
            a = an;
        }
        if (ncols == before) fail = true;  // a window must advance the walk
    }
    land(0);
    land(1);
    ws.x[0] = x0;
    ws.x[1] = x1;
    ws.x[2] = x2;
    ws.ncols = ncols;
    if (fail) ws.fail = 1;
}

// Row-major layout, boxes [x - D, x] (k <= 3).
template <int K>
__device__ void walk_boxes(const ProblemDesc &P, const IODesc &io, unsigned char *box, WalkState &ws) {
    const int tid = threadIdx.x;
    const int D = traceback_box(K);
    constexpr int G = 16;
    int64_t ts[K];
    for (int i = 0; i < K; ++i) ts[i] = P.tbstride[i];
    const int len_sum = P.len_sum;
    while (true) {
        __syncthreads();
        if (ws.fail || at_origin(K, ws.x)) break;
        int lo[K], ext[K];
        int64_t bs[K];
        for (int i = 0; i < K; ++i) lo[i] = max(0, ws.x[i] - D);
        const int a = lo[K - 1] & ~(G - 1);
        const int rowb = round_up(ws.x[K - 1] - a + 1, G);
        const int cpr = rowb / G;
        bs[K - 1] = 1;
        int64_t stride = rowb;
        int rows = 1;
        for (int i = K - 2; i >= 0; --i) {
            bs[i] = stride;
            ext[i] = ws.x[i] - lo[i] + 1;
            stride *= ext[i];
            rows *= ext[i];
        }
        for (int idx = tid; idx < rows * cpr; idx += kTbThreads) {
            int r = idx / cpr;
            const int c = idx - r * cpr;
            const int row = r;
            int64_t g = a;
            for (int i = K - 2; i >= 0; --i) {
                const int ci = r % ext[i];
                r /= ext[i];
                g += (int64_t)(lo[i] + ci) * ts[i];
            }
            cp_async_16(box + (int64_t)row * rowb + 16 * c, P.tb + g + 16 * c);
        }
        cp_async_wait_all();
        __syncthreads();
        if (tid == 0) {
            int x[K];  // registers, not shared memory, on the dependent chain
            for (int i = 0; i < K; ++i) x[i] = ws.x[i];
            int ncols = ws.ncols;
            const int before = ncols;
            bool fail = false;
            const unsigned bbase = smem_u32(box);
            int li = x[K - 1] - a;
            for (int i = 0; i < K - 1; ++i) li += (x[i] - lo[i]) * (int)bs[i];
            // as in the column walk: the next byte is loaded before this move's
            // checks branch; a next cell outside the box reads byte 0 (unused)
            int m = lds_u8(bbase + li);
            while (true) {
                int zero = 0, y[K], lj = li;
                bool out = false, at0 = true;
                for (int i = 0; i < K; ++i) {
                    const int b = (m >> i) & 1;
                    zero |= (x[i] == 0) << i;
                    y[i] = x[i] - b;
                    lj -= b * (int)bs[i];
                    out |= y[i] < lo[i];
                    at0 &= y[i] == 0;
                }
                const bool bad = (m == 0) | ((m >> K) != 0) | ((m & zero) != 0) | (ncols >= len_sum);
                const bool in = !out & !at0;
                const int mn = lds_u8(bbase + (in ? lj : 0));
                if (bad) {
                    fail = true;
                    break;
                }
                stg_u8(io.masks + ncols, m);
                ++ncols;
                for (int i = 0; i < K; ++i) x[i] = y[i];
                li = lj;
                if (!in) break;
                m = mn;
            }
            if (ncols == before && !at_origin(K, x)) fail = true;  // a box must advance the walk
            for (int i = 0; i < K; ++i) ws.x[i] = x[i];
            ws.ncols = ncols;
            if (fail) ws.fail = 1;
        }
    }
}

// Byte offset of cell x in the traceback tensor: row-major (tbstride), or
// tile-major (layouts 2 and 3: tile t = sum (x_i / E_i) gstride_i holds a block
// of tb_block bytes, the cell at sum_i (x_i mod E_i) * lst_i inside it; layout 2
// is local row-major, layout 3 the line kernel's skewed rows).
__device__ __forceinline__ int64_t tb_cell(const ProblemDesc &P, const int *x) {
    int64_t g = 0;
    if (P.tb_layout == 2 || P.tb_layout == 3) {
        int64_t t = 0, loc = 0;
        for (int i = 0; i < P.k; ++i) {
            const int e = P.E[i], q = x[i] / e;
            t += (int64_t)q * P.gstride[i];
            loc += (int64_t)(x[i] - q * e) * P.lst[i];
        }
        g = t * P.tb_block + loc;
    } else {
        for (int i = 0; i < P.k; ++i) g += (int64_t)x[i] * P.tbstride[i];
    }
    return g;
}

// k >= 4 (row-major or tile-major): the current cell and all its predecessors per round trip.
__device__ void walk_direct(const ProblemDesc &P, const IODesc &io, unsigned char *pred, WalkState &ws) {
    const int tid = threadIdx.x;
    const int K = P.k;
    const int NM = (1 << K) - 1;
    if (tid >= 32) return;
    int x[MSA_MAX_K];
    for (int i = 0; i < K; ++i) x[i] = ws.x[i];
    int ncols = 0, fail = 0;
    while (!fail && !at_origin(K, x)) {
        // slot 0: the cell itself; slot m: its predecessor x - e_m (if inside)
        for (int m = tid; m <= NM; m += 32) {
            int c[MSA_MAX_K];
            bool in = true;
            for (int i = 0; i < K; ++i) {
                c[i] = x[i] - ((m >> i) & 1);
                in = in && c[i] >= 0;
            }
            pred[m] = in ? __ldcg(P.tb + tb_cell(P, c)) : (unsigned char)0;
        }
        __syncwarp();
        if (tid == 0) {
            const int m1 = pred[0];
            if (!take_move(K, m1, x, io.masks, P.len_sum, ncols)) {
                fail = 1;
            } else if (!at_origin(K, x) && !take_move(K, pred[m1], x, io.masks, P.len_sum, ncols)) {
                fail = 1;
            }
        }
        __syncwarp();
        for (int i = 0; i < K; ++i) x[i] = __shfl_sync(kFull, x[i], 0);
        fail = __shfl_sync(kFull, fail, 0);
        ncols = __shfl_sync(kFull, ncols, 0);
    }
    if (tid == 0) {
        for (int i = 0; i < K; ++i) ws.x[i] = x[i];
        ws.ncols = ncols;
        ws.fail = fail;
    }
}

// Tile-major layouts (k >= 4): the CTA stages the blocks of the tiles
// [q - span + 1, q] per axis around the current cell's tile q (span 4, 3 or 2:
// the largest whose blocks fit the window memory), one 16-byte-aligned copy of
// each block, and thread 0 walks them in registers -- local coordinates, the
// offset inside the tile and the tile's slot updated per move -- until the walk
// leaves the staged tiles (at least (span - 1) E moves along every axis).
template <int K>
__device__ void walk_tiles(const ProblemDesc &P, const IODesc &io, unsigned char *smem, WalkState &ws) {
    const int tid = threadIdx.x;
    int E[K], lst[K];
    for (int i = 0; i < K; ++i) {
        E[i] = P.E[i];
        lst[i] = P.lst[i];
    }
    const int vol = P.tb_block;                // bytes of one tile's block
    const int slot = round_up(vol + 15, 16);  // a block copied from the 16-byte boundary below it
    const int cps = slot / 16;
    int span = 0, nslot = 0;
    for (int sp = 4; sp >= 2 && !span; --sp) {
        int n = 1;
        for (int i = 0; i < K; ++i) n *= sp;
        if ((int64_t)n * (slot + 12) <= kTracebackSmem) {
            span = sp;
            nslot = n;
        }
    }
    if (!span || cps > kTbThreads) {
        walk_direct(P, io, smem, ws);
        return;
    }
    int64_t *sstart = reinterpret_cast<int64_t *>(smem + (size_t)nslot * slot);  // per slot: block's global offset
    unsigned *sbase = reinterpret_cast<unsigned *>(sstart + nslot);             // per slot: shared address of its byte 0
    const int len_sum = P.len_sum;
    while (true) {
        __syncthreads();
        if (ws.fail || at_origin(K, ws.x)) break;
        int qlo[K], sst[K];
        int n = 1;
        for (int i = K - 1; i >= 0; --i) {
            qlo[i] = max(0, ws.x[i] / E[i] - span + 1);
            sst[i] = n;
            n *= ws.x[i] / E[i] - qlo[i] + 1;
        }
        for (int sl = tid; sl < n; sl += kTbThreads) {  // each staged tile's block
            int r = sl;
            int64_t t = 0;
            for (int i = 0; i < K; ++i) {
                const int d = r / sst[i];
                r -= d * sst[i];
                t += (int64_t)(qlo[i] + d) * P.gstride[i];
            }
            const int64_t start = t * vol;
            sstart[sl] = start & ~(int64_t)15;
            sbase[sl] = smem_u32(smem + (size_t)sl * slot) + (unsigned)(start & 15);
        }
        __syncthreads();
        {  // thread tid copies chunk tid % cps of every (kTbThreads / cps)-th block,
           // where the block reaches it (never past the block's last 16-byte run)
            const int ch = tid % cps, step = kTbThreads / cps;
            for (int sl = tid / cps; sl < n && tid < step * cps; sl += step)
                if (16 * ch < (int)(sbase[sl] & 15) + vol)
                    cp_async_16(smem + (size_t)sl * slot + 16 * ch, P.tb + sstart[sl] + 16 * ch);
        }
        cp_async_wait_all();
        __syncthreads();
        if (tid == 0) {
            int x[K], c[K], q[K];
            int loc = 0, sl = 0;
            for (int i = 0; i < K; ++i) {
                x[i] = ws.x[i];
                q[i] = x[i] / E[i];
                c[i] = x[i] - q[i] * E[i];
                loc += c[i] * lst[i];
                sl += (q[i] - qlo[i]) * sst[i];
            }
            unsigned base = sbase[sl];
            int ncols = ws.ncols;
            const int before = ncols;
            bool fail = false;
            while (!at_origin(K, x)) {
                const int m = lds_u8(base + (unsigned)loc);
                int zero = 0;
                for (int i = 0; i < K; ++i) zero |= (x[i] == 0) << i;
                if (m == 0 || (m >> K) != 0 || (m & zero) != 0 || ncols >= len_sum) {
                    fail = true;
                    break;
                }
                stg_u8(io.masks + ncols, m);
                ++ncols;
                bool out = false, cross = false;
                for (int i = 0; i < K; ++i)
                    if ((m >> i) & 1) {
                        --x[i];
                        if (c[i] > 0) {
                            --c[i];
                            loc -= lst[i];
                        } else {  // into the tile below along axis i
                            c[i] = E[i] - 1;
                            loc += (E[i] - 1) * lst[i];
                            --q[i];
                            sl -= sst[i];
                            cross = true;
                            out = out || q[i] < qlo[i];
                        }
                    }
                if (out) break;
                if (cross) base = sbase[sl];
            }
            if (ncols == before && !at_origin(K, x)) fail = true;  // a region must advance the walk
            for (int i = 0; i < K; ++i) ws.x[i] = x[i];
            ws.ncols = ncols;
            if (fail) ws.fail = 1;
        }
    }
}

// Line tiles spanning the whole last axis (layout 3 with one segment: the line
// kernels' tiles of 32 lines over the first k - 1 axes, each a block of rows of
// 32 bytes, cell (c, z) in row z + sum c_i at the lane of its line): a block is
// too large to stage whole, so the CTA stages a window of rows of every tile
// within a span below the current cell's tile along each line axis. A cell's
// row never exceeds the current cell's z plus the block's largest skew and only
// falls along a path, so the window holds rows [rhi - RW + 1, rhi] with rhi the
// current z plus that skew, and thread 0 walks until a move leaves the staged
// tiles or falls below the window. The spans grow the axis the walk would leave
// soonest ((span - 1) x extent moves), within a staging volume that keeps a
// re-stage short.
constexpr int kLineWindowMinBlock = 2048;  // smaller line tiles are staged whole (walk_tiles)
template <int K>
__device__ void walk_lines(const ProblemDesc &P, const IODesc &io, unsigned char *smem, WalkState &ws) {
    constexpr int NA = K - 1;
    constexpr int RW = 40, RB = RW * 32;                // rows per window, bytes per staged tile
    constexpr int kBudget = (24 * 1024) / RB;           // staged tiles (measured: 24 KB beats 48, 96, 192)
    const int tid = threadIdx.x;
    int E[NA], lst[NA], span[NA];
    int skew = 0;
    for (int i = 0; i < NA; ++i) {
        E[i] = P.E[i];
        lst[i] = P.lst[i];
        span[i] = 1;
        skew += E[i] - 1;
    }
    for (int guard = 0; guard < 64; ++guard) {
        int n = 1, best = -1;
        for (int i = 0; i < NA; ++i) n *= span[i];
        for (int i = 0; i < NA; ++i)
            if (n / span[i] * (span[i] + 1) <= kBudget && (best < 0 || span[i] * E[i] < span[best] * E[best]))
                best = i;
        if (best < 0) break;
        ++span[best];
    }
    const int len_sum = P.len_sum;
    while (true) {
        __syncthreads();
        if (ws.fail || at_origin(K, ws.x)) break;
        int qlo[NA], sst[NA];
        int n = 1;
        for (int i = NA - 1; i >= 0; --i) {
            const int q = ws.x[i] / E[i];
            qlo[i] = max(0, q - span[i] + 1);
            sst[i] = n;
            n *= q - qlo[i] + 1;
        }
        const int rhi = ws.x[NA] + skew;
        const int rlo = max(0, rhi - RW + 1);
        const int nch = (rhi - rlo + 1) * 2;  // 16-byte chunks of a tile's window
        for (int w = tid; w < n * nch; w += kTbThreads) {
            const int sl = w / nch, ch = w - sl * nch;
            int r = sl;
            int64_t t = 0;
            for (int i = 0; i < NA; ++i) {
                const int d = r / sst[i];
                r -= d * sst[i];
                t += (int64_t)(qlo[i] + d) * P.gstride[i];
            }
            cp_async_16(smem + (size_t)sl * RB + 16 * ch, P.tb + t * P.tb_block + 32 * (int64_t)rlo + 16 * ch);
        }
        cp_async_wait_all();
        __syncthreads();
        if (tid == 0) {
            int x[K], c[NA], q[NA];
            int sl = 0, loc = 32 * (ws.x[NA] - rlo);  // byte offset in the window: 32 (row - rlo) + lane
            for (int i = 0; i < K; ++i) x[i] = ws.x[i];
            for (int i = 0; i < NA; ++i) {
                q[i] = x[i] / E[i];
                c[i] = x[i] - q[i] * E[i];
                loc += c[i] * lst[i];
                sl += (q[i] - qlo[i]) * sst[i];
            }
            unsigned base = smem_u32(smem + (size_t)sl * RB);
            int ncols = ws.ncols;
            const int before = ncols;
            bool fail = false;
            while (!at_origin(K, x)) {
                const int m = lds_u8(base + (unsigned)loc);
                int zero = 0;
                for (int i = 0; i < K; ++i) zero |= (x[i] == 0) << i;
                if (m == 0 || (m >> K) != 0 || (m & zero) != 0 || ncols >= len_sum) {
                    fail = true;
                    break;
                }
                stg_u8(io.masks + ncols, m);
                ++ncols;
                bool out = false, cross = false;
                if ((m >> NA) & 1) {
                    --x[NA];
                    loc -= 32;
                }
                for (int i = 0; i < NA; ++i)
                    if ((m >> i) & 1) {
                        --x[i];
                        if (c[i] > 0) {
                            --c[i];
                            loc -= lst[i];
                        } else {  // into the tile below along axis i
                            c[i] = E[i] - 1;
                            loc += (E[i] - 1) * lst[i];
                            --q[i];
                            sl -= sst[i];
                            cross = true;
                            out = out || q[i] < qlo[i];
                        }
                    }
                if (out || loc < 0) break;  // left the staged tiles, or below the window's rows
                if (cross) base = smem_u32(smem + (size_t)sl * RB);
            }
            if (ncols == before && !at_origin(K, x)) fail = true;  // a window must advance the walk
            for (int i = 0; i < K; ++i) ws.x[i] = x[i];
            ws.ncols = ncols;
            if (fail) ws.fail = 1;
        }
    }
}

// Score of the recorded path, by the whole CTA: sum over columns of
// u*|m| + sum over moved pairs (sub - 2 gap), each column at the position the
// suffix of later moves (earlier in the record) gives it.
__device__ int score_path(const ProblemDesc &P, const IODesc &io, int ncols, int *scan) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = P.k, B = P.B, A = P.A;
    const int u = io.gap * (K - 1);
    const int per = (ncols + kTbThreads - 1) / kTbThreads;
    const int j0 = min(ncols, tid * per), j1 = min(ncols, j0 + per);
    // moves per axis in this thread's run, then an exclusive scan over threads
    int cnt[MSA_MAX_K] = {};
    for (int j = j0; j < j1; ++j) {
        const int m = io.masks[j];
        for (int i = 0; i < K; ++i) cnt[i] += (m >> i) & 1;
    }
    int off[MSA_MAX_K];
    for (int i = 0; i < K; ++i) {
        int v = cnt[i];
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(kFull, v, d);
            if (lane >= d) v += y;
        }
        if (lane == 31) scan[i * 8 + warp] = v;
        off[i] = v - cnt[i];
    }
    __syncthreads();
    for (int i = 0; i < K; ++i)
        for (int w2 = 0; w2 < warp; ++w2) off[i] += scan[i * 8 + w2];
    int x[MSA_MAX_K];
    for (int i = 0; i < K; ++i) x[i] = P.len[i] - off[i];
    int s = 0;
    for (int j = j0; j < j1; ++j) {
        const int m = io.masks[j];
        int c[MSA_MAX_K], nm = 0;
        for (int i = 0; i < K; ++i)
            if ((m >> i) & 1) c[nm++] = P.codes[P.cofs[i] + x[i] - 1];
        int col = u * nm;
        for (int a = 0; a < nm; ++a)
            for (int b = a + 1; b < nm; ++b) col += P.tab[c[a] * A + c[b]] >> B;
        s += col;
        for (int i = 0; i < K; ++i) x[i] -= (m >> i) & 1;
    }
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(kFull, s, d);
    __syncthreads();
    if (lane == 0) scan[64 + warp] = s;
    __syncthreads();
    int total = 0;
    for (int w2 = 0; w2 < kTbThreads / 32; ++w2) total += scan[64 + w2];
    return total;
}

__global__ void __launch_bounds__(kTbThreads) traceback_kernel(const ProblemDesc *probs, const int32_t *err,
                                                               const IODesc *io_arr, IODesc io1) {
    const int p = blockIdx.x;
    const ProblemDesc &P = probs[p];
    const IODesc io = io_arr ? io_arr[p] : io1;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ WalkState ws;
    __shared__ int scan[64 + kTbThreads / 32];
    const int tid = threadIdx.x;
    int status = ld_volatile(&P.istat->status);
    if (status == 0 && err) status = ld_volatile(err);
    if (status != 0) {
        if (tid == 0) {
            io.result->status = status;
            io.result->score = 0;
            io.result->ncols = 0;
        }
        return;
    }
    const int K = P.k;
    if (tid == 0) {
        for (int i = 0; i < K; ++i) ws.x[i] = P.len[i];
        ws.ncols = 0;
        ws.fail = 0;
    }
    __syncthreads();
    if (P.tb_layout == 1)
        walk_col3(P, io, smem, ws);
    else if (K == 2)
        walk_boxes<2>(P, io, smem, ws);
    else if (K == 3)
        walk_boxes<3>(P, io, smem, ws);
    else if (P.tb_layout == 3 && P.G[K - 1] == 1 && P.tb_block > kLineWindowMinBlock && K == 4)
        walk_lines<4>(P, io, smem, ws);
    else if (P.tb_layout == 3 && P.G[K - 1] == 1 && P.tb_block > kLineWindowMinBlock && K == 5)
        walk_lines<5>(P, io, smem, ws);
    else if (P.tb_layout == 3 && P.G[K - 1] == 1 && P.tb_block > kLineWindowMinBlock && K == 6)
        walk_lines<6>(P, io, smem, ws);
    else if (P.tb_layout >= 2 && K == 4)
        walk_tiles<4>(P, io, smem, ws);
    else if (P.tb_layout >= 2 && K == 5)
        walk_tiles<5>(P, io, smem, ws);
    else if (P.tb_layout >= 2 && K == 6)
        walk_tiles<6>(P, io, smem, ws);
    else if (P.tb_layout >= 2 && K == 7)
        walk_tiles<7>(P, io, smem, ws);
    else if (P.tb_layout >= 2 && K == 8)
        walk_tiles<8>(P, io, smem, ws);
    else
        walk_direct(P, io, smem, ws);
    __syncthreads();
    const int ncols = ws.ncols;
    int fail = ws.fail;
    const int score = fail ? 0 : score_path(P, io, ncols, scan);
    if (tid == 0) {
        if (!fail && P.has_qcorner) {
            // cross-check against the fill's own corner value: q = H' * 2^B + W(corner)
            const int q = *P.qcorner;
            const int h = ((q - P.w_corner) >> P.B) + io.gap * (K - 1) * P.len_sum;
            if (h != score) fail = 1;
        }
        io.result->score = score;
        io.result->ncols = ncols;
        io.result->status = fail ? MSA_ECUDA : MSA_OK;
    }
}

}  // namespace

cudaError_t traceback_attributes() {
    static DeviceOnce once;  // attribute set once per device, never inside a stream capture
    return once.run([] {
        return cudaFuncSetAttribute(traceback_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTracebackSmem);
    });
}

cudaError_t launch_traceback(const ProblemDesc *d_probs, int nprob, const int32_t *err,
                             const IODesc *io_array, IODesc io_single, cudaStream_t s) {
    cudaError_t e = traceback_attributes();
    if (e != cudaSuccess) return e;
    traceback_kernel<<<nprob, kTbThreads, kTracebackSmem, s>>>(d_probs, err, io_array, io_single);
    return cudaGetLastError();
}

}  // namespace msadp
