// Traceback (section 2): from the far corner follow the stored move of every
// cell back to the origin, then score the path.
//
// One CTA of 256 threads per problem. The walk is a chain of dependent reads, so
// thread 0 walks; the rest of the CTA stages the data it reads:
//   * column layout (k = 3 column kernel): windows of one column, as many CTA
//     times as fit in shared memory of the warp blocks and lanes the walk can
//     still reach (cp.async by all threads), for about as many CTA times as a
//     diagonal walk needs to leave the column; every move lowers the CTA time
//     T = x2 + l + (x0 mod WR) by its popcount, so a window of n times holds at
//     least n / 3 moves unless the walk leaves the column;
//   * row-major layout, k <= 3: boxes [x - D, x] (rows of the last axis copied in
//     16-byte granules);
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
__device__ __forceinline__ bool take_move(int K, int m, int *x, const ProblemDesc &P, const IODesc &io, int &ncols) {
    bool bad = m == 0 || (m >> K) != 0 || ncols >= P.len_sum;
    for (int i = 0; i < K; ++i)
        if (((m >> i) & 1) && x[i] == 0) bad = true;
    if (bad) return false;
    io.masks[ncols++] = (uint8_t)m;
    for (int i = 0; i < K; ++i) x[i] -= (m >> i) & 1;
    return true;
}

__device__ __forceinline__ bool at_origin(int K, const int *x) {
    for (int i = 0; i < K; ++i)
        if (x[i] != 0) return false;
    return true;
}

// Column layout of the k = 3 column kernel.
__device__ void walk_col3(const ProblemDesc &P, const IODesc &io, unsigned char *win, WalkState &ws) {
    const int tid = threadIdx.x;
    const int NB = P.G[1];
    const int rho2 = P.rho[2];
    const int64_t colb = c3::tb_col_bytes(rho2);
    const int nT = c3::nsteps(rho2);
    while (true) {
        __syncthreads();
        if (ws.fail || at_origin(3, ws.x)) break;
        const int x0 = ws.x[0], x1 = ws.x[1], x2 = ws.x[2];
        const int cA = x0 / c3::WR, cB = x1 >> 5;
        const unsigned char *col = P.tb + (int64_t)(cA * NB + cB) * colb;
        // window: the walk only moves to lower rows and lanes, so only warp blocks
        // 0 .. w and lanes 0 .. l are staged (16-byte runs from the start of each
        // warp block's 32 * R bytes), for as many CTA times as the shared memory
        // holds (up to 255): [t_hi - nt + 1, t_hi]
        constexpr int kRowB = 32 * c3::R;                              // bytes per (time, warp block)
        const int nw = x0 % c3::WR / c3::R + 1;                        // warp blocks staged
        const int ncp = ((x1 & 31) * c3::R + c3::R + 15) / 16;         // 16-byte runs per warp block
        const int per_t = nw * ncp;                                    // runs per CTA time
        // mostly diagonal paths leave the column after about min(row, lane) moves
        // of three CTA times each: stage that much (plus slack), within the memory
        const int nt = min(min(255, kTracebackSmem / (16 * per_t)), 3 * min(x0 % c3::WR, x1 & 31) + 24);
        const int t_hi = x2 + (x1 & 31) + x0 % c3::WR;
        const int t_lo = t_hi - nt + 1;
        for (int i = tid; i < nt * per_t; i += kTbThreads) {
            const int row = i / per_t, rem = i - row * per_t;
            const int w = rem / ncp, part = rem - w * ncp;
            const int tt = t_lo + row;
            if (tt >= 0 && tt < nT)
                cp_async_16(win + 16 * i, col + (int64_t)(tt + c3::U) * (c3::W * kRowB) + w * kRowB + 16 * part);
        }
        cp_async_wait_all();
        __syncthreads();
        if (tid == 0) {
            int *x = ws.x;
            const int before = ws.ncols;
            while (!at_origin(3, x)) {
                const int rho = x[0] % c3::WR, l = x[1] & 31;
                const int tt = x[2] + l + rho;
                if (x[0] / c3::WR != cA || (x[1] >> 5) != cB || tt < t_lo) break;
                const int byte = l * c3::R + rho % c3::R;  // < ncp * 16: l and rho only decrease in a column
                const int m = win[((tt - t_lo) * nw + rho / c3::R) * (16 * ncp) + byte];
                if (!take_move(3, m, x, P, io, ws.ncols)) {
                    ws.fail = 1;
                    break;
                }
            }
            if (ws.ncols == before && !at_origin(3, x)) ws.fail = 1;  // a window must advance the walk
        }
    }
}

// Row-major layout, boxes [x - D, x] (k <= 3).
__device__ void walk_boxes(const ProblemDesc &P, const IODesc &io, unsigned char *box, WalkState &ws) {
    const int tid = threadIdx.x;
    const int K = P.k;
    const int D = traceback_box(K);
    constexpr int G = 16;
    int64_t ts[MSA_MAX_K];
    for (int i = 0; i < K; ++i) ts[i] = P.tbstride[i];
    while (true) {
        __syncthreads();
        if (ws.fail || at_origin(K, ws.x)) break;
        int lo[MSA_MAX_K], ext[MSA_MAX_K];
        int64_t bs[MSA_MAX_K];
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
            int *x = ws.x;
            const int before = ws.ncols;
            int64_t li = x[K - 1] - a;
            for (int i = 0; i < K - 1; ++i) li += (int64_t)(x[i] - lo[i]) * bs[i];
            while (!at_origin(K, x)) {
                const int m = box[li];
                if (!take_move(K, m, x, P, io, ws.ncols)) {
                    ws.fail = 1;
                    break;
                }
                bool out = false;
                for (int i = 0; i < K; ++i)
                    if ((m >> i) & 1) {
                        li -= bs[i];
                        if (x[i] < lo[i]) out = true;
                    }
                if (out) break;
            }
            if (ws.ncols == before && !at_origin(K, x)) ws.fail = 1;  // a box must advance the walk
        }
    }
}

// Byte offset of cell x in the traceback tensor: row-major (tbstride), or
// tile-major (layout 2: tile t = sum (x_i / E_i) gstride_i holds a block of
// prod E_i bytes in local row-major order).
__device__ __forceinline__ int64_t tb_cell(const ProblemDesc &P, const int *x, int64_t vol) {
    int64_t g = 0;
    if (P.tb_layout == 2) {
        int64_t t = 0, loc = 0;
        for (int i = 0; i < P.k; ++i) {
            const int e = P.E[i], q = x[i] / e;
            t += (int64_t)q * P.gstride[i];
            loc = loc * e + (x[i] - q * e);
        }
        g = t * vol + loc;
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
    int64_t vol = 1;
    for (int i = 0; i < K; ++i) vol *= P.E[i];
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
            pred[m] = in ? __ldcg(P.tb + tb_cell(P, c, vol)) : (unsigned char)0;
        }
        __syncwarp();
        if (tid == 0) {
            const int m1 = pred[0];
            if (!take_move(K, m1, x, P, io, ncols)) {
                fail = 1;
            } else if (!at_origin(K, x) && !take_move(K, pred[m1], x, P, io, ncols)) {
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
    else if (K <= 3)
        walk_boxes(P, io, smem, ws);
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
