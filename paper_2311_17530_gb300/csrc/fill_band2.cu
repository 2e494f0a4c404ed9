// k = 2 band kernel: the pairwise DP (Eq. 1, section 2's 2^k - 1 = 3 neighbours
// for k = 2) as a skewed wavefront along warp lanes.
//
// A band is 32 consecutive rows x0 of one problem; one warp fills it, lane l
// owning row 32 b + l and sweeping the columns x1 with a skew of one column per
// lane: at warp step t lane l computes column j = t - l. Then the cell above
// (x0 - 1, j) was computed by lane l - 1 at step t - 1 and the diagonal cell
// (x0 - 1, j - 1) at step t - 2, so both arrive by one shuffle per step; the left
// cell is the lane's own previous value. Lane 0 takes the cells above from the
// band above, whose lane 31 writes its row to a face in global memory and
// publishes how many 32-column blocks of it are complete (release store); the
// band below waits (bounded acquire) for a block before its lane 0 reaches it and
// loads it with one coalesced 32-entry read. Bands are handed out by an atomic
// ticket in order, band above first, so a band only waits for a band already
// running.
//
// Values are the packed keys of every fill kernel: Q = (H - gap |x|) * 4 + W(x),
// W(x) = x0 + 2 x1, single-sequence moves cost 0 and the diagonal move the
// pair table entry ((sub - 2 gap) << 2); one max gives the best value and, in its
// low two bits, the lowest move mask among ties. Traceback bytes are written
// row-major, four columns per 4-byte store; the lane that computes the far corner
// records its key, which the traceback compares with the rescored path.
#include "api_internal.h"
#include "device_common.cuh"

namespace msadp {
namespace {

constexpr int kBandWarps = 8;  // warps per CTA, one band each

__global__ void __launch_bounds__(kBandWarps * 32) fill_band2_kernel(const LaunchDesc L) {
    const int lane = threadIdx.x & 31;
    // per warp: each lane's row of the pair table, transposed (entry b of lane l
    // at b * 32 + l, so a step's 32 lookups hit 32 banks)
    __shared__ int tabT[kBandWarps][MSA_MAX_ALPHABET * 32];
    int *trow = tabT[threadIdx.x >> 5];
    while (true) {
        int t = 0, err = 0;
        if (lane == 0) {
            t = atomicAdd(L.ticket, 1);
            err = ld_volatile(L.err);
        }
        t = __shfl_sync(kFull, t, 0);
        err = __shfl_sync(kFull, err, 0);
        if ((int64_t)t >= L.ntickets || err != 0) break;
        const uint64_t ent = L.order[t];
        const ProblemDesc &P = L.probs[(int)(ent >> 32)];
        const int band = (int)(uint32_t)ent;
        const int rho0 = P.rho[0], rho1 = P.rho[1];
        const int nblocks = (rho1 + 31) >> 5;
        const int64_t fstride = P.face0_stride;
        int32_t *prog_out = &L.done[P.tile_base + band];
        const int32_t *prog_in = band > 0 ? &L.done[P.tile_base + band - 1] : nullptr;
        const int32_t *face_in = band > 0 ? P.Q + (int64_t)(band - 1) * fstride : nullptr;
        int32_t *face_out = P.Q + (int64_t)band * fstride;
        int st = 0;
        if (lane == 0) st = ld_volatile(&P.istat->status);
        st = __shfl_sync(kFull, st, 0);
        if (st != 0) {  // a failed problem: no work, but let the band below pass
            if (lane == 31 && (int64_t)t != L.withhold) st_release(prog_out, nblocks);
            continue;
        }
        const int i = band * 32 + lane;  // this lane's row x0
        const bool row_ok = i < rho0;
        const uint8_t *c1 = P.codes + P.cofs[1];
        const int arow = (row_ok && i >= 1) ? (int)P.codes[P.cofs[0] + i - 1] * P.A : 0;
        __syncwarp();
        for (int b = 0; b < P.A; ++b) trow[b * 32 + lane] = __ldg(P.tab + arow + b);
        __syncwarp();
        uint8_t *tbrow = P.tb + (int64_t)(row_ok ? i : 0) * P.tbstride[0];
        const bool publish = lane == 31 && (int64_t)t != L.withhold;
        int V = kNeg;        // this lane's value at its previous column
        int up_prev = kNeg;  // the cell above one column back: the diagonal predecessor
        int fblk = kNeg;     // lane q holds the band above's face at column 32 * block + q
        int cblk = 0;        // lane q holds the residue code consumed at column 32 * block + q
        int bj = 0;          // the code consumed at this lane's column (shifted along the lanes)
        unsigned pk = 0;     // traceback bytes of the current 4-column group
        bool ok = true;
        for (int s = 0; s < rho1 + 31; ++s) {
            if ((s & 31) == 0 && s < rho1) {  // lane 0 enters block s / 32: stage its codes and face
                const int col = s + lane;
                cblk = (col >= 1 && col < rho1) ? (int)c1[col - 1] : 0;
                if (band > 0) {
                    const int need = (s >> 5) + 1;
                    bool w = true;
                    if (lane == 0) w = wait_at_least(prog_in, need, L.err, L.spin_ns);
                    ok = __shfl_sync(kFull, w, 0);
                    if (!ok) break;
                    __syncwarp();
                    fblk = col < rho1 ? __ldcg(face_in + col) : kNeg;
                }
            }
            {  // lane l's column s - l consumes the code lane l - 1 held a step ago
                const int b0 = __shfl_sync(kFull, cblk, s & 31);
                const int b = __shfl_up_sync(kFull, bj, 1);
                bj = lane == 0 ? b0 : b;
            }
            const int from_face = __shfl_sync(kFull, fblk, s & 31);
            int up = __shfl_up_sync(kFull, V, 1);
            if (lane == 0) up = (band > 0 && s < rho1) ? from_face : kNeg;
            const int diag = up_prev;
            up_prev = up;
            const int j = s - lane;
            int Vn = kNeg;
            if (row_ok && j >= 0 && j < rho1) {
                int m = 0;
                if (i == 0 && j == 0) {
                    Vn = 0;  // H(0) = 0, no move
                } else {
                    int acc = max(up, V);
                    if (i >= 1 && j >= 1) acc = __viaddmax_s32(diag, trow[bj * 32 + lane], acc);
                    m = (i + 2 * j - acc) & 3;
                    Vn = acc + m;
                }
                pk |= (unsigned)m << (8 * (j & 3));
                if ((j & 3) == 3 || j == rho1 - 1) {
                    *reinterpret_cast<uint32_t *>(tbrow + (j & ~3)) = pk;
                    pk = 0;
                    // the far corner's key, for the traceback's cross-check
                    if (j == rho1 - 1 && i == rho0 - 1) *P.qcorner = Vn;
                }
                if (lane == 31) {
                    face_out[j] = Vn;
                    if (publish && ((j & 31) == 31 || j == rho1 - 1)) st_release(prog_out, (j >> 5) + 1);
                }
            }
            V = Vn;
        }
        if (!ok) {
            if (lane == 0) atomicCAS(L.err, 0, MSA_ETIMEOUT);
            break;
        }
        // rows past the tensor (a partial last band) never reach the publishing lane
        if (publish && !row_ok) st_release(prog_out, nblocks);
    }
}

}  // namespace

cudaError_t launch_fill_band2(const LaunchDesc &L, int grid, cudaStream_t s) {
    fill_band2_kernel<<<grid, kBandWarps * 32, 0, s>>>(L);
    return cudaGetLastError();
}

int fill_band2_ctas_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fill_band2_kernel, kBandWarps * 32, 0) != cudaSuccess) return 0;
    return n;
}

int fill_band2_warps_per_cta() { return kBandWarps; }

}  // namespace msadp
