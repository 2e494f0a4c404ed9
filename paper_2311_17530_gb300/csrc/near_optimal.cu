// Optimal and near-optimal alignments on the device (section 6 proposes
// retrieving further solutions by forking at equally ranked paths, or within a
// threshold the user sets): every alignment scoring at least OPT - delta,
// enumerated from the far corner by a depth-first walk over the kept score
// tensor, the moves of each column tried in increasing mask order (so the
// alignments come in increasing lexicographic order of their reversed column
// sequence, the first being the single-alignment traceback's for delta = 0).
//
// A move m from cell x to p = x - e_m is followed when
//     H(p) + SP(m at x) + (score of the columns already fixed) >= OPT - delta,
// H being the forward tensor: H(p) is the best any completion through p can add,
// so every qualifying alignment is reached and no other one is produced.
//
// The fill is the generic tile kernel, which keeps the packed key of every cell:
// Q(x) = H'(x) 2^k + W(x) with H'(x) = H(x) - gap (k - 1) |x|_1 and
// W(x) = sum_i 2^i x_i, so H(x) = (Q(x) - W(x)) / 2^k + gap (k - 1) |x|_1
// exactly. One warp walks: at each depth its 32 lanes judge 32 consecutive
// masks at once and a ballot picks the lowest one that qualifies.
#include "device_common.cuh"

namespace msadp {

// Element offset of cell x in the tile kernel's score tensor: row-major
// (qstride) for k <= 3, tile-major (the traceback's layout 2) for k >= 4.
__device__ __forceinline__ int64_t score_cell(const ProblemDesc &P, const int *x) {
    int64_t g = 0;
    if (P.tb_layout == 2) {
        int64_t t = 0, loc = 0;
        for (int i = 0; i < P.k; ++i) {
            const int e = P.E[i], q = x[i] / e;
            t += (int64_t)q * P.gstride[i];
            loc += (int64_t)(x[i] - q * e) * P.lst[i];
        }
        g = t * P.tb_block + loc;
    } else {
        for (int i = 0; i < P.k; ++i) g += (int64_t)x[i] * P.qstride[i];
    }
    return g;
}

__device__ __forceinline__ int64_t forward_score(const ProblemDesc &P, const int *x, int64_t u) {
    int64_t w = 0, s = 0;
    for (int i = 0; i < P.k; ++i) {
        w += (int64_t)x[i] << i;
        s += x[i];
    }
    return (((int64_t)P.Q[score_cell(P, x)] - w) >> P.k) + u * s;
}

__global__ void __launch_bounds__(32) near_optimal_kernel(const ProblemDesc *probs, IODesc io, int64_t delta,
                                                          int32_t max_count, NearOut o) {
    const ProblemDesc &P = probs[0];
    const int lane = threadIdx.x;
    const int k = P.k, A = P.A, total = P.len_sum, nm = (1 << k) - 1;
    if (ld_volatile(&P.istat->status) != 0) {  // the fill did not complete: nothing to enumerate
        if (lane == 0) {
            o.count_more[0] = 0;
            o.count_more[1] = 0;
        }
        return;
    }
    const int64_t u = (int64_t)io.gap * (k - 1);
    int x[MSA_MAX_K];
    for (int i = 0; i < k; ++i) x[i] = P.len[i];
    const int64_t thr = forward_score(P, x, u) - delta;  // OPT - delta
    int d = 0, count = 0, more = 0;
    int64_t acc = 0;  // score of the columns fixed so far (depth d)
    int nxt = 1;      // next mask to try at depth d
    // Every move followed leads to at least one qualifying alignment (H(p) is
    // reached by some path), so the walk takes at most 2 (total + 1) steps per
    // alignment it stores, plus one; the bound below only guards that argument.
    const int64_t limit = 2 * ((int64_t)total + 1) * ((int64_t)max_count + 1) + 2;
    for (int64_t it = 0; d >= 0; ++it) {
        if (it > limit) {
            more = 2;  // reported as an inconsistent tensor
            break;
        }
        bool origin = true;
        for (int i = 0; i < k; ++i) origin = origin && x[i] == 0;
        int mstar = 0;
        int64_t spstar = 0;
        if (origin) {
            if (count == max_count) {
                more = 1;
                break;
            }
            uint8_t *dst = o.masks + (int64_t)count * total;
            for (int c = lane; c < d; c += 32) dst[c] = o.path[d - 1 - c];
            if (lane == 0) {
                o.ncols[count] = d;
                o.scores[count] = acc;
            }
            ++count;
        } else {
            // residues at x (the column a move consumes)
            int code[MSA_MAX_K];
            for (int i = 0; i < k; ++i) code[i] = x[i] >= 1 ? P.codes[P.cofs[i] + x[i] - 1] : 0;
            for (int base = nxt; base <= nm && !mstar; base += 32) {
                const int m = base + lane;
                bool ok = m <= nm;
                int64_t sp = 0;
                if (ok) {
                    int y[MSA_MAX_K];
                    for (int i = 0; i < k; ++i) {
                        const int b = (m >> i) & 1;
                        ok = ok && (!b || x[i] >= 1);
                        y[i] = x[i] - b;
                    }
                    if (ok) {
                        for (int i = 0; i < k; ++i)
                            for (int j = i + 1; j < k; ++j) {
                                const int bi = (m >> i) & 1, bj = (m >> j) & 1;
                                if (bi && bj)
                                    sp += io.subst[code[i] * A + code[j]];
                                else if (bi || bj)
                                    sp += io.gap;
                            }
                        ok = forward_score(P, y, u) + sp + acc >= thr;
                    }
                }
                const unsigned hit = __ballot_sync(kFull, ok);
                if (hit) {
                    const int src = __ffs(hit) - 1;
                    mstar = base + src;
                    spstar = __shfl_sync(kFull, sp, src);
                }
            }
        }
        __syncwarp();
        if (mstar) {  // descend
            if (lane == 0) {
                o.path[d] = (uint8_t)mstar;
                o.next[d] = mstar + 1;
                o.acc[d] = acc;
            }
            for (int i = 0; i < k; ++i) x[i] -= (mstar >> i) & 1;
            acc += spstar;
            nxt = 1;
            ++d;
        } else {  // back to the previous depth (its move undone, its next mask resumed)
            --d;
            if (d >= 0) {
                __syncwarp();
                const int m = o.path[d];
                for (int i = 0; i < k; ++i) x[i] += (m >> i) & 1;
                acc = o.acc[d];
                nxt = o.next[d];
            }
        }
        __syncwarp();
    }
    if (lane == 0) {
        o.count_more[0] = count;
        o.count_more[1] = more;
    }
}

cudaError_t launch_near_optimal(const ProblemDesc *d_prob, IODesc io, int64_t delta, int32_t max_count, NearOut o,
                                cudaStream_t s) {
    near_optimal_kernel<<<1, 32, 0, s>>>(d_prob, io, delta, max_count, o);
    return cudaGetLastError();
}

}  // namespace msadp
