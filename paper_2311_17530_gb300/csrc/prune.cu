// Exact search-space pruning on the device, the restriction of the search space
// the paper leaves for future work (section 6: search only the partitions where
// an optimal alignment can lie), by the bound of Carrillo and Lipman. An
// alignment's sum-of-pairs score is the sum of the scores of its pairwise
// projections (gap against gap scores 0, section 5.2), and the projection of an
// alignment through cell x passes through (x_i, x_j), so no alignment through x
// scores above
//     U(x) = sum_{i<j} fwd_ij[x_i][x_j] + bwd_ij[x_i][x_j],
// fwd_ij / bwd_ij being the optimal pairwise scores of the prefixes / suffixes
// (Eq. 1 on each pair). A tile's bound is the sum over pairs of the largest
// fwd + bwd over the tile's rectangle of the (i, j) plane, never below U(x) of
// any cell inside; a tile whose bound is below a lower bound L on the optimum
// (the score of any feasible alignment) holds no cell of any optimal alignment,
// nor any optimal predecessor of such a cell, so the fill may leave it out and
// the optimal alignment (with its tie-break) is unchanged.
//
// Kernels, in stream order after the encode step:
//   pair_tables_kernel   fwd and bwd of every pair, by anti-diagonals (one CTA
//                        per pair and direction, three diagonals in shared memory)
//   block_max_kernel     per pair, the largest fwd + bwd of every tile rectangle
//   greedy_bound_kernel  L: the score of the alignment built from the origin by
//                        taking, at every cell, the move to the neighbour with the
//                        largest U (ties: lowest mask) -- a feasible alignment
//   tile_bounds_kernel   per tile, the sum of its rectangles' maxima; the tiles
//                        below L are flagged for the fill and counted
#include "device_common.cuh"

namespace msadp {

constexpr int kPruneThreads = 1024;

__global__ void __launch_bounds__(kPruneThreads) pair_tables_kernel(const PruneDesc D) {
    const int pr = blockIdx.x, dir = blockIdx.y;  // dir 0: prefixes (fwd), 1: suffixes (bwd)
    const int i = D.pi[pr], j = D.pj[pr];
    const int na = D.len[i], nb = D.len[j], A = D.A, gap = D.gap;
    const uint8_t *a = D.codes + D.cofs[i], *b = D.codes + D.cofs[j];
    const int64_t W = (int64_t)nb + 1;
    int32_t *T = D.tables + D.toff[pr] + (dir ? ((int64_t)na + 1) * W : 0);
    extern __shared__ int32_t dg[];  // three anti-diagonals, indexed by p
    int32_t *d0 = dg, *d1 = dg + (na + 1), *d2 = dg + 2 * (na + 1);
    // For the suffixes the same recurrence runs on the reversed sequences:
    // bwd[p][q] is the value at reversed coordinates (na - p, nb - q).
    for (int d = 0; d <= na + nb; ++d) {
        const int plo = d - nb > 0 ? d - nb : 0, phi = d < na ? d : na;
        for (int p = plo + (int)threadIdx.x; p <= phi; p += blockDim.x) {
            const int q = d - p;
            int v = 0;
            if (d > 0) {
                int best = INT32_MIN / 2;
                if (p > 0) best = max(best, d1[p - 1] + gap);
                if (q > 0) best = max(best, d1[p] + gap);
                if (p > 0 && q > 0) {
                    const int ca = dir ? a[na - p] : a[p - 1], cb = dir ? b[nb - q] : b[q - 1];
                    best = max(best, d2[p - 1] + D.sub[ca * A + cb]);
                }
                v = best;
            }
            d0[p] = v;
            if (dir)
                T[(int64_t)(na - p) * W + (nb - q)] = v;
            else
                T[(int64_t)p * W + q] = v;
        }
        __syncthreads();
        int32_t *t = d2;
        d2 = d1;
        d1 = d0;
        d0 = t;
    }
}

__device__ __forceinline__ int64_t pair_fb(const PruneDesc &D, int pr, int p, int q) {
    const int nb = D.len[D.pj[pr]];
    const int64_t W = (int64_t)nb + 1, n = ((int64_t)D.len[D.pi[pr]] + 1) * W;
    const int32_t *T = D.tables + D.toff[pr];
    return (int64_t)T[(int64_t)p * W + q] + T[n + (int64_t)p * W + q];
}

__global__ void block_max_kernel(const PruneDesc D) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < D.nblocks; g += (int64_t)gridDim.x * blockDim.x) {
        int pr = 0;
        while (pr + 1 < D.npairs && D.boff[pr + 1] <= g) ++pr;
        const int i = D.pi[pr], j = D.pj[pr];
        const int64_t r = g - D.boff[pr];
        const int bi = (int)(r / D.G[j]), bj = (int)(r - (int64_t)bi * D.G[j]);
        const int p0 = bi * D.E[i], p1 = min(p0 + D.E[i], D.len[i] + 1);
        const int q0 = bj * D.E[j], q1 = min(q0 + D.E[j], D.len[j] + 1);
        int64_t best = INT64_MIN / 4;
        for (int p = p0; p < p1; ++p)
            for (int q = q0; q < q1; ++q) best = max(best, pair_fb(D, pr, p, q));
        D.blk[g] = best;
    }
}

// One warp. Lanes judge 32 masks at a time; the warp keeps the best (largest U,
// then lowest mask) and moves there, adding the column's SP score.
__global__ void __launch_bounds__(32) greedy_bound_kernel(const PruneDesc D) {
    const int lane = threadIdx.x, k = D.k, nm = (1 << k) - 1;
    int x[MSA_MAX_K];
    for (int i = 0; i < k; ++i) x[i] = 0;
    int64_t score = 0;
    int steps = 0;
    while (steps <= D.len_sum) {
        bool at_corner = true;
        for (int i = 0; i < k; ++i) at_corner = at_corner && x[i] == D.len[i];
        if (at_corner) break;
        int64_t bu = INT64_MIN;
        int bm = 0;
        for (int base = 1; base <= nm; base += 32) {
            const int m = base + lane;
            bool ok = m <= nm;
            int y[MSA_MAX_K];
            for (int i = 0; i < k; ++i) {
                const int bit = (m >> i) & 1;
                ok = ok && (!bit || x[i] < D.len[i]);
                y[i] = x[i] + bit;
            }
            if (ok) {
                int64_t u = 0;
                for (int pr = 0; pr < D.npairs; ++pr) u += pair_fb(D, pr, y[D.pi[pr]], y[D.pj[pr]]);
                if (u > bu) {  // masks rise with the chunk: strict > keeps the lowest
                    bu = u;
                    bm = m;
                }
            }
        }
        // warp arg-max: largest U, then lowest mask
        for (int off = 16; off; off >>= 1) {
            const int64_t ou = __shfl_xor_sync(kFull, bu, off);
            const int om = __shfl_xor_sync(kFull, bm, off);
            if (om != 0 && (bm == 0 || ou > bu || (ou == bu && om < bm))) {
                bu = ou;
                bm = om;
            }
        }
        // the column of move bm, consumed at y = x + e_bm
        int64_t sp = 0;
        for (int i = 0; i < k; ++i) x[i] += (bm >> i) & 1;
        for (int i = 0; i < k; ++i)
            for (int j = i + 1; j < k; ++j) {
                const int bi = (bm >> i) & 1, bj = (bm >> j) & 1;
                if (bi && bj)
                    sp += D.sub[D.codes[D.cofs[i] + x[i] - 1] * D.A + D.codes[D.cofs[j] + x[j] - 1]];
                else if (bi || bj)
                    sp += D.gap;
            }
        score += sp;
        ++steps;
    }
    if (lane == 0) *D.lower = score;
}

__global__ void tile_bounds_kernel(const PruneDesc D) {
    const int64_t L = D.skip ? *D.lower : 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < D.ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        int c[MSA_MAX_K];
        int64_t rem = t, cells = 1;
        for (int i = 0; i < D.k; ++i) {
            c[i] = (int)(rem / D.gstride[i]);
            rem -= (int64_t)c[i] * D.gstride[i];
            cells *= min(D.E[i], D.len[i] + 1 - c[i] * D.E[i]);
        }
        int64_t bound = 0;
        for (int pr = 0; pr < D.npairs; ++pr) bound += D.blk[D.boff[pr] + (int64_t)c[D.pi[pr]] * D.G[D.pj[pr]] + c[D.pj[pr]]];
        if (D.bound) D.bound[t] = bound;
        if (D.skip) {
            const bool out = bound < L;
            D.skip[t] = out;
            if (out) {
                atomicAdd(reinterpret_cast<unsigned long long *>(D.stats), 1ull);
                atomicAdd(reinterpret_cast<unsigned long long *>(D.stats + 1), (unsigned long long)cells);
            }
        }
    }
}

cudaError_t launch_prune(const PruneDesc &D, bool greedy, cudaStream_t s) {
    int maxa = 0;
    for (int pr = 0; pr < D.npairs; ++pr) maxa = max(maxa, D.len[D.pi[pr]] + 1);
    const int smem = 3 * maxa * 4;
    cudaError_t e = cudaFuncSetAttribute(pair_tables_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    pair_tables_kernel<<<dim3(D.npairs, 2), kPruneThreads, smem, s>>>(D);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nbb = (D.nblocks + 255) / 256;
    block_max_kernel<<<(int)(nbb < 4096 ? (nbb < 1 ? 1 : nbb) : 4096), 256, 0, s>>>(D);
    e = cudaGetLastError();
    if (e == cudaSuccess && greedy) {
        greedy_bound_kernel<<<1, 32, 0, s>>>(D);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int64_t nt = (D.ntiles + 255) / 256;
        tile_bounds_kernel<<<(int)(nt < 4096 ? (nt < 1 ? 1 : nt) : 4096), 256, 0, s>>>(D);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace msadp
