// Encode + table kernel (hot-path step a1), plus the per-k dispatch of the
// generic tile fill and of the line-sweep fill.
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
    if (P.clear_faces) {
        // Column-kernel faces in a reused region: tag 0 everywhere, so that no
        // stale word can pass for an entry of this launch (the fill runs after this
        // kernel on the same stream). Face sizes are multiples of 64 ints.
        const int64_t n0 = P.face0_stride * P.ntiles / 4, n1 = P.face1_stride * P.ntiles / 4;
        const int4 z = make_int4(0, 0, 0, 0);
        for (int64_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n0; i += (int64_t)gridDim.x * blockDim.x)
            reinterpret_cast<int4 *>(P.Q)[i] = z;
        for (int64_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += (int64_t)gridDim.x * blockDim.x)
            reinterpret_cast<int4 *>(P.aux)[i] = z;
    }
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
                          const IODesc *io_array, IODesc io_single, cudaStream_t s, int min_blocks) {
    int bx = (max_ncode + 255) / 256;
    if (bx < min_blocks) bx = min_blocks;
    if (bx < 1) bx = 1;
    if (bx > 64) bx = 64;
    encode_kernel<<<dim3(bx, nprob), 256, 0, s>>>(d_probs, io_array, io_single);
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

#define MSADP_LINES_K(k)                                                                      \
    cudaError_t launch_fill_lines_k##k(int z, const LaunchDesc &L, int grid, cudaStream_t s); \
    int fill_lines_ctas_k##k(int z);                                                          \
    int fill_lines_warps_k##k(int z);
MSADP_LINES_K(4)
MSADP_LINES_K(5)
MSADP_LINES_K(6)
#undef MSADP_LINES_K

cudaError_t launch_fill_lines(int k, int z, const LaunchDesc &L, int grid, cudaStream_t s) {
    switch (k) {
        case 4: return launch_fill_lines_k4(z, L, grid, s);
        case 5: return launch_fill_lines_k5(z, L, grid, s);
        case 6: return launch_fill_lines_k6(z, L, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int fill_lines_ctas_per_sm(int k, int z) {
    switch (k) {
        case 4: return fill_lines_ctas_k4(z);
        case 5: return fill_lines_ctas_k5(z);
        case 6: return fill_lines_ctas_k6(z);
        default: return 0;
    }
}

int fill_lines_warps_per_cta(int k, int z) {
    switch (k) {
        case 4: return fill_lines_warps_k4(z);
        case 5: return fill_lines_warps_k5(z);
        case 6: return fill_lines_warps_k6(z);
        default: return 0;
    }
}

cudaError_t launch_fill_stream_k4(const LaunchDesc &L, int grid, cudaStream_t s);
cudaError_t launch_fill_stream_k5(const LaunchDesc &L, int grid, cudaStream_t s);
cudaError_t launch_fill_stream_k6(const LaunchDesc &L, int grid, cudaStream_t s, int rho_s);
int fill_stream_ctas_k4();
int fill_stream_ctas_k5();
int fill_stream_ctas_k6();

cudaError_t launch_fill_stream(int k, const LaunchDesc &L, int grid, cudaStream_t s, int rho_s) {
    return k == 4   ? launch_fill_stream_k4(L, grid, s)
           : k == 5 ? launch_fill_stream_k5(L, grid, s)
           : k == 6 ? launch_fill_stream_k6(L, grid, s, rho_s)
                    : cudaErrorInvalidValue;
}

int fill_stream_ctas_per_sm(int k) {
    return k == 4 ? fill_stream_ctas_k4() : k == 5 ? fill_stream_ctas_k5() : k == 6 ? fill_stream_ctas_k6() : 0;
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
    for (int k = kLinesMinK; k <= kLinesMaxK && e == cudaSuccess; ++k)
        for (int i = 0; i < kMaxLineSegments && e == cudaSuccess; ++i)
            if (line_z_candidate(k, i) > 0 && fill_lines_ctas_per_sm(k, line_z_candidate(k, i)) <= 0)
                e = cudaErrorInvalidValue;
    for (int k = kStreamMinK; k <= kStreamMaxK && e == cudaSuccess; ++k)
        if (fill_stream_ctas_per_sm(k) <= 0) e = cudaErrorInvalidValue;
    return e;
}

}  // namespace msadp
