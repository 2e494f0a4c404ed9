// Encode + table kernel (hot-path step a1) and the single-warp traceback kernel
// (step a4), plus the per-k dispatch of the generic tile fill.
#include "device_common.cuh"

namespace msadp {

// Residues -> alphabet codes; pair table scaled for the packed-key fill:
// tab[a][b] = (sub[a][b] - 2 gap) << k. Rejects residues outside the alphabet
// and non-symmetric tables (MSA_EINVAL), and any table whose keys could leave
// the exact int32 range (MSA_ETOOBIG), by writing the problem's status word.
__global__ void encode_kernel(const ProblemDesc *probs, const IODesc *io_arr, IODesc io1) {
    const int p = blockIdx.y;
    const ProblemDesc &P = probs[p];
    const IODesc io = io_arr ? io_arr[p] : io1;
    msa_device_result *st = P.istat;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.ncode; i += gridDim.x * blockDim.x) {
        const uint8_t c = P.amap[(uint8_t)io.residues[i]];
        if (c == 0xFF) atomicCAS(&st->status, 0, MSA_EINVAL);
        P.codes[i] = (c == 0xFF) ? (uint8_t)0 : c;
    }
    if (blockIdx.x != 0) return;
    __shared__ int smax, sbad;
    if (threadIdx.x == 0) {
        smax = 0;
        sbad = 0;
    }
    __syncthreads();
    const int A = P.A, B = P.B;
    int lmax = 0, lbad = 0, lbig = 0;
    for (int i = threadIdx.x; i < A * A; i += blockDim.x) {
        const int a = i / A, b = i - a * A;
        const int64_t v = io.subst[i];
        if (v != (int64_t)io.subst[b * A + a]) lbad = 1;
        const int64_t pp = v - 2 * (int64_t)io.gap;  // pair score with the gap terms folded in
        const int64_t ap = pp < 0 ? -pp : pp;
        if ((ap << B) >= kKeyLimit) {
            lbig = 1;
            P.tab[i] = 0;
        } else {
            lmax = max(lmax, (int)ap);
            P.tab[i] = (int32_t)(pp * ((int64_t)1 << B));
        }
    }
    atomicMax(&smax, lmax);
    if (lbad) atomicOr(&sbad, 1);
    if (lbig) atomicOr(&sbad, 2);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sbad & 1) atomicCAS(&st->status, 0, MSA_EINVAL);
        // |H'| <= maxp * sum_{i<j} min(len_i, len_j); a candidate adds at most
        // C(k,2) * maxp; keys carry the factor 2^B and the potential W <= W(len).
        // The margin 4 * (len_sum + 64) keeps the k = 3 column kernel's skew cells
        // (x2 < 0, seeded at kNeg, tie bits adding at most 7 per cell along a path
        // of at most len_sum + 63 cells) strictly below every valid key.
        const int64_t npairs = (int64_t)P.k * (P.k - 1) / 2;
        const int64_t key_bound = (int64_t)smax * (P.pair_min_sum + npairs) * ((int64_t)1 << B) + P.w_corner +
                                  4 * ((int64_t)P.len_sum + 64);
        const int64_t g = io.gap < 0 ? -(int64_t)io.gap : (int64_t)io.gap;
        const int64_t score_bound = (int64_t)smax * P.pair_min_sum + g * (P.k - 1) * P.len_sum;
        if ((sbad & 2) || key_bound >= kKeyLimit || score_bound >= ((int64_t)1 << 31) - 1)
            atomicCAS(&st->status, 0, MSA_ETOOBIG);
    }
}

cudaError_t launch_encode(const ProblemDesc *d_probs, int nprob, int max_ncode,
                          const IODesc *io_array, IODesc io_single, cudaStream_t s) {
    int bx = (max_ncode + 255) / 256;
    if (bx < 1) bx = 1;
    if (bx > 64) bx = 64;
    encode_kernel<<<dim3(bx, nprob), 256, 0, s>>>(d_probs, io_array, io_single);
    return cudaGetLastError();
}

// Traceback (section 2): from the far corner follow the stored move of every
// cell back to the origin. One warp per problem: the warp stages the box
// [x - D, x] of the traceback tensor into shared memory with asynchronous
// global->shared copies (all issued, then one wait), lane 0 walks the path inside
// the box until it leaves through a lower face, and the next box is staged
// around the new position. Boxes are aligned to the copy granule along the last
// axis. The masks are written last column first; the score is decoded from the
// corner's packed key.
__device__ __forceinline__ void cp_async_16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Traceback over the k = 3 column kernel's layout. The walk stays inside one
// column (A, B) as long as it can; the warp stages a window of that column --
// CTA times [T - 24, T + 7], every warp block w, lanes [l0, l0 + 16) -- as
// 16-byte runs per (time, w), and lane 0 walks inside it. Every move lowers the
// CTA time T = x2 + l + (x0 mod WR) of the walk by its number of moved sequences.
constexpr int kTbcSteps = 32;                          // steps per window
constexpr int kTbcLanes = 16;                          // lanes per window
constexpr int kTbcRow = kTbcLanes * c3::R;             // bytes per (step, warp block) in a window
constexpr int kTbcParts = kTbcRow / 16;                // 16-byte copies per (step, warp block)
constexpr int kTbcAlign = 16 / c3::R;                  // window start lane: 16-byte aligned
constexpr int kTbcBytes = kTbcSteps * c3::W * kTbcRow;
static_assert(kTbcBytes <= kTracebackSmem, "traceback window exceeds its shared memory");

__device__ void traceback_col3(const ProblemDesc &P, const IODesc &io, unsigned char *box, int lane) {
    const int nsym = P.A, bits = P.B;  // alphabet size, tie bits
    const int u = io.gap * 2;  // gap * (k - 1)
    const int NB = P.G[1];
    const int rho2 = P.rho[2];
    const int64_t colb = c3::tb_col_bytes(rho2);
    int x0 = P.len[0], x1 = P.len[1], x2 = P.len[2];
    int score = 0, ncols = 0, fail = 0;
    while ((x0 | x1 | x2) != 0 && !fail) {
        const int cA = x0 / c3::WR, cB = x1 >> 5;
        const int l = x1 & 31;
        const int t_lo = x2 + l + x0 % c3::WR - (kTbcSteps - 8);
        const int l0 = max(0, l - (kTbcLanes - kTbcAlign)) & ~(kTbcAlign - 1);  // l0 <= l < l0 + 16
        const unsigned char *col = P.tb + (int64_t)(cA * NB + cB) * colb;
        // rows of the window: (step, w) pairs, 8 x 16 B each
        for (int i = lane; i < kTbcSteps * c3::W * kTbcParts; i += 32) {
            const int part = i % kTbcParts, row = i / kTbcParts;
            const int tt = t_lo + row / c3::W, w = row % c3::W;
            if (tt >= 0 && tt < c3::nsteps(rho2))
                cp_async_16(box + row * kTbcRow + part * 16,
                            col + ((int64_t)((tt + c3::U) * c3::W + w) * 32 + l0) * c3::R + part * 16);
        }
        cp_async_wait_all();
        __syncwarp();
        if (lane == 0) {
            const int before = ncols;
            while ((x0 | x1 | x2) != 0) {
                const int ca = x0 / c3::WR, cb = x1 >> 5;
                const int ll = x1 & 31, rr = x0 & (c3::R - 1), ww = (x0 % c3::WR) / c3::R;
                const int tt = x2 + ll + x0 % c3::WR;
                if (ca != cA || cb != cB || ll < l0 || ll >= l0 + kTbcLanes || tt < t_lo || tt >= t_lo + kTbcSteps)
                    break;
                const int m = box[((tt - t_lo) * c3::W + ww) * kTbcRow + (ll - l0) * c3::R + rr];
                if (m == 0 || m > 7 || ((m & 1) && x0 == 0) || ((m & 2) && x1 == 0) || ((m & 4) && x2 == 0) ||
                    ncols >= P.len_sum) {
                    fail = 1;
                    break;
                }
                io.masks[ncols++] = (uint8_t)m;
                // column score: u per residue plus the pair terms among moved sequences
                int c[3], nm = 0;
                if (m & 1) c[nm++] = P.codes[P.cofs[0] + x0 - 1];
                if (m & 2) c[nm++] = P.codes[P.cofs[1] + x1 - 1];
                if (m & 4) c[nm++] = P.codes[P.cofs[2] + x2 - 1];
                int col_score = u * nm;
                for (int i = 0; i < nm; ++i)
                    for (int j = i + 1; j < nm; ++j) col_score += P.tab[c[i] * nsym + c[j]] >> bits;
                score += col_score;
                x0 -= m & 1;
                x1 -= (m >> 1) & 1;
                x2 -= (m >> 2) & 1;
            }
            if (ncols == before && (x0 | x1 | x2) != 0) fail = 1;  // a window must advance the walk
        }
        x0 = __shfl_sync(kFull, x0, 0);
        x1 = __shfl_sync(kFull, x1, 0);
        x2 = __shfl_sync(kFull, x2, 0);
        ncols = __shfl_sync(kFull, ncols, 0);
        fail = __shfl_sync(kFull, fail, 0);
        __syncwarp();
    }
    if (lane == 0) {
        io.result->score = score;
        io.result->ncols = ncols;
        io.result->status = fail ? MSA_ECUDA : MSA_OK;
    }
}

__global__ void __launch_bounds__(32) traceback_kernel(const ProblemDesc *probs, const int32_t *err,
                                                       const IODesc *io_arr, IODesc io1) {
    const int p = blockIdx.x;
    const ProblemDesc &P = probs[p];
    const IODesc io = io_arr ? io_arr[p] : io1;
    extern __shared__ __align__(16) unsigned char box[];
    const int lane = threadIdx.x;
    int status = ld_volatile(&P.istat->status);
    if (status == 0 && err) status = ld_volatile(err);
    if (status != 0) {
        if (lane == 0) {
            io.result->status = status;
            io.result->score = 0;
            io.result->ncols = 0;
        }
        return;
    }
    if (P.tb_layout == 1) {
        traceback_col3(P, io, box, lane);
        return;
    }
    const int K = P.k, B = P.B;
    const int D = traceback_box(K);
    const int G = traceback_granule(K);  // bytes per copy: 16 (k <= 4) or 4
    const int A = P.A;
    int x[MSA_MAX_K], lo[MSA_MAX_K], ext[MSA_MAX_K];
    int64_t bs[MSA_MAX_K], ts[MSA_MAX_K];
    for (int i = 0; i < K; ++i) {
        x[i] = P.len[i];
        ts[i] = P.tbstride[i];
    }
    // The score is the sum of the traced columns' SP scores: with the gap terms
    // folded in, a column of move m scores u*|m| + sum_{i<j in m} (sub - 2 gap),
    // u = gap * (k - 1), and tab holds (sub - 2 gap) << k.
    const int u = io.gap * (K - 1);
    int score = 0;
    int ncols = 0;
    int fail = 0;
    while (true) {
        bool any = false;
        for (int i = 0; i < K; ++i) any = any || x[i] > 0;
        if (!any || fail) break;
        for (int i = 0; i < K; ++i) lo[i] = max(0, x[i] - D);
        const int a = lo[K - 1] & ~(G - 1);
        const int rowb = round_up(x[K - 1] - a + 1, G);
        const int cpr = rowb / G;  // copies per row
        bs[K - 1] = 1;
        int64_t stride = rowb;
        int rows = 1;
        for (int i = K - 2; i >= 0; --i) {
            bs[i] = stride;
            ext[i] = x[i] - lo[i] + 1;
            stride *= ext[i];
            rows *= ext[i];
        }
        for (int row = lane; row < rows; row += 32) {
            int r = row;
            int64_t g = a;
            for (int i = K - 2; i >= 0; --i) {
                const int ci = r % ext[i];
                r /= ext[i];
                g += (int64_t)(lo[i] + ci) * ts[i];
            }
            unsigned char *dst = box + (int64_t)row * rowb;
            const uint8_t *src = P.tb + g;
            if (G == 16)
                for (int c = 0; c < cpr; ++c) cp_async_16(dst + 16 * c, src + 16 * c);
            else
                for (int c = 0; c < cpr; ++c) cp_async_4(dst + 4 * c, src + 4 * c);
        }
        cp_async_wait_all();
        __syncwarp();
        if (lane == 0) {
            const int before = ncols;
            int64_t li = x[K - 1] - a;
            for (int i = 0; i < K - 1; ++i) li += (int64_t)(x[i] - lo[i]) * bs[i];
            while (true) {
                bool any2 = false;
                for (int i = 0; i < K; ++i) any2 = any2 || x[i] > 0;
                if (!any2) break;
                const int m = box[li];
                bool bad = (m == 0) || (m >> K) != 0 || ncols >= P.len_sum;
                for (int i = 0; i < K; ++i)
                    if (((m >> i) & 1) && x[i] == 0) bad = true;
                if (bad) {
                    fail = 1;
                    break;
                }
                io.masks[ncols++] = (uint8_t)m;
                // column score: residues entering x (position x_i - 1 of each moved sequence)
                int c[MSA_MAX_K];
                int nm = 0;
                for (int i = 0; i < K; ++i)
                    if ((m >> i) & 1) {
                        c[nm++] = P.codes[P.cofs[i] + x[i] - 1];
                    }
                int col = u * nm;
                for (int i = 0; i < nm; ++i)
                    for (int j = i + 1; j < nm; ++j) col += P.tab[c[i] * A + c[j]] >> B;
                score += col;
                bool out = false;
                for (int i = 0; i < K; ++i)
                    if ((m >> i) & 1) {
                        x[i] -= 1;
                        li -= bs[i];
                        if (x[i] < lo[i]) out = true;
                    }
                if (out) break;
            }
            bool left = false;
            for (int i = 0; i < K; ++i) left = left || x[i] > 0;
            if (ncols == before && left) fail = 1;  // a box must advance the walk
        }
        for (int i = 0; i < K; ++i) x[i] = __shfl_sync(kFull, x[i], 0);
        ncols = __shfl_sync(kFull, ncols, 0);
        fail = __shfl_sync(kFull, fail, 0);
        __syncwarp();
    }
    if (lane == 0) {
        if (!fail && P.has_qcorner) {
            // cross-check against the fill's own corner value: q = H' * 2^B + W(corner)
            const int q = *P.qcorner;
            const int h = ((q - P.w_corner) >> B) + u * P.len_sum;
            if (h != score) fail = 1;
        }
        io.result->score = score;
        io.result->ncols = ncols;
        io.result->status = fail ? MSA_ECUDA : MSA_OK;
    }
}

static cudaError_t traceback_attributes() {
    static DeviceOnce once;  // attribute set once per device, never inside a stream capture
    return once.run([] {
        return cudaFuncSetAttribute(traceback_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTracebackSmem);
    });
}

cudaError_t launch_traceback(const ProblemDesc *d_probs, int nprob, const int32_t *err,
                             const IODesc *io_array, IODesc io_single, cudaStream_t s) {
    cudaError_t e = traceback_attributes();
    if (e != cudaSuccess) return e;
    traceback_kernel<<<nprob, 32, kTracebackSmem, s>>>(d_probs, err, io_array, io_single);
    return cudaGetLastError();
}

#define MSADP_TILES_K(k)                                                                      \
    cudaError_t launch_fill_tiles_k##k(int edge, const LaunchDesc &L, int grid, cudaStream_t s); \
    int fill_tiles_ctas_k##k(int edge);                                                          \
    int fill_tiles_warps_k##k(int edge);
MSADP_TILES_K(2)
MSADP_TILES_K(3)
MSADP_TILES_K(4)
MSADP_TILES_K(5)
MSADP_TILES_K(6)
MSADP_TILES_K(7)
MSADP_TILES_K(8)
#undef MSADP_TILES_K

cudaError_t launch_fill_tiles(int k, int edge, const LaunchDesc &L, int grid, cudaStream_t s) {
    switch (k) {
        case 2: return launch_fill_tiles_k2(edge, L, grid, s);
        case 3: return launch_fill_tiles_k3(edge, L, grid, s);
        case 4: return launch_fill_tiles_k4(edge, L, grid, s);
        case 5: return launch_fill_tiles_k5(edge, L, grid, s);
        case 6: return launch_fill_tiles_k6(edge, L, grid, s);
        case 7: return launch_fill_tiles_k7(edge, L, grid, s);
        case 8: return launch_fill_tiles_k8(edge, L, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int fill_tiles_ctas_per_sm(int k, int edge) {
    switch (k) {
        case 2: return fill_tiles_ctas_k2(edge);
        case 3: return fill_tiles_ctas_k3(edge);
        case 4: return fill_tiles_ctas_k4(edge);
        case 5: return fill_tiles_ctas_k5(edge);
        case 6: return fill_tiles_ctas_k6(edge);
        case 7: return fill_tiles_ctas_k7(edge);
        case 8: return fill_tiles_ctas_k8(edge);
        default: return 0;
    }
}

int fill_tiles_warps_per_cta(int k, int edge) {
    switch (k) {
        case 2: return fill_tiles_warps_k2(edge);
        case 3: return fill_tiles_warps_k3(edge);
        case 4: return fill_tiles_warps_k4(edge);
        case 5: return fill_tiles_warps_k5(edge);
        case 6: return fill_tiles_warps_k6(edge);
        case 7: return fill_tiles_warps_k7(edge);
        case 8: return fill_tiles_warps_k8(edge);
        default: return 0;
    }
}

cudaError_t col3_attributes();

// Every kernel attribute the launch wrappers need on the current device, so that
// a later stream capture contains launches only.
cudaError_t prepare_kernel_attributes() {
    cudaError_t e = traceback_attributes();
    if (e == cudaSuccess) e = col3_attributes();
    for (int k = 2; k <= MSA_MAX_K && e == cudaSuccess; ++k)
        for (int i = 0; i < kMaxTileEdges && e == cudaSuccess; ++i)
            if (tile_edge_candidate(k, i) > 0 && fill_tiles_ctas_per_sm(k, tile_edge_candidate(k, i)) <= 0)
                e = cudaErrorInvalidValue;
    return e;
}

}  // namespace msadp
