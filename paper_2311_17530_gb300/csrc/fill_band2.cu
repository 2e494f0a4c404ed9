// k = 2 band kernel: the pairwise DP (Eq. 1, section 2's 2^k - 1 = 3 neighbours
// for k = 2) as a skewed wavefront along warp lanes.
//
// A band is 32 R consecutive rows x0 of one problem; one warp fills it, lane l
// owning rows 32 R b + R l .. + R - 1 and sweeping the columns x1 with a skew of
// one column per lane: at warp step t lane l fills column j = t - l of its R rows,
// top to bottom. The cell above its first row, (x0 - 1, j), was filled by lane
// l - 1 at step t - 1 and the diagonal cell (x0 - 1, j - 1) at step t - 2, so both
// arrive by one shuffle per step; within a lane the cells above and on the
// diagonal are the row filled just before and its previous column, and the left
// cell is the row's own previous value. Shuffles, the code shift along the lanes
// and the loop are paid once per R cells.
//
// Lane 0 takes the cells above from the band above: its lane 31 writes its last
// row to a face in global memory as (value, tag) 8-byte entries, the tag being the
// launch's epoch; the band below loads a block of 32 entries when its lane 0
// reaches it and accepts it once every entry carries the epoch (a bounded wait),
// so no fence or release/acquire pair is needed: an aligned 8-byte entry is
// written by one store and read whole, and entries of earlier launches carry
// smaller epochs (the plan clears the faces before the first launch and when
// epochs wrap; serving clears them in the encode step). Bands are handed out by
// an atomic ticket in order, band above first, so a band only waits for a band
// already running.
//
// The sweep runs in three loops -- the skew ramp (some lanes left of column 0),
// the interior (every lane on a column), the ramp out (some lanes past the last
// column) -- so interior steps carry no bounds checks. A lane off the tensor
// keeps its values (no cell there: the initial "no cell" keys on the way in, the
// last column's keys on the way out).
//
// Values are the packed keys of every fill kernel: Q = (H - gap |x|) * 4 + W(x),
// W(x) = x0 + 2 x1, single-sequence moves cost 0 and the diagonal move the
// pair table entry ((sub - 2 gap) << 2); one max gives the best value and, in its
// low two bits, the lowest move mask among ties. Traceback bytes are written
// row-major, four columns per 4-byte store; the lane holding the far corner
// records its key, which the traceback compares with the rescored path.
#include "api_internal.h"
#include "device_common.cuh"

#include <type_traits>

namespace msadp {
namespace {

constexpr int kBandR = kBand2RowsPerLane;
constexpr int kBandWarps = kBandR <= 2 ? 4 : 2;  // warps per CTA, one band each (the tables take 32 KB)

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long face_entry(int value, int tag) {
    return (unsigned long long)(unsigned)value | ((unsigned long long)(unsigned)tag << 32);
}

template <int R>
__global__ void __launch_bounds__(kBandWarps * 32) fill_band2_kernel(const LaunchDesc L) {
    const int lane = threadIdx.x & 31;
    // per warp: the pair-table rows of each lane's R residues, transposed (entry b
    // of row q of lane l at (b R + q) 32 + l, so a step's 32 lookups hit 32 banks)
    __shared__ int tabT[kBandWarps][MSA_MAX_ALPHABET * R * 32];
    int *trow = tabT[threadIdx.x >> 5];
    const int epoch = L.epoch;
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
        int st = 0;
        if (lane == 0) st = ld_volatile(&P.istat->status);
        // a failed problem: none of its bands works, so none waits for this one
        if (__shfl_sync(kFull, st, 0) != 0) continue;
        const int rho0 = P.rho[0], rho1 = P.rho[1];
        const int tagout = (int64_t)t == L.withhold ? 0 : epoch;  // a withheld band publishes nothing valid
        const int64_t fstride = P.face0_stride / 2;                // 8-byte entries per face
        unsigned long long *Fq = reinterpret_cast<unsigned long long *>(P.Q);
        const unsigned long long *face_in = band > 0 ? Fq + (int64_t)(band - 1) * fstride : nullptr;
        unsigned long long *face_out = Fq + (int64_t)band * fstride;
        const int i0 = band * 32 * R + lane * R;  // this lane's first row x0
        const uint8_t *c1 = P.codes + P.cofs[1];
        const int A = P.A;
        __syncwarp();
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = i0 + q;
            const int arow = (i >= 1 && i < rho0) ? (int)P.codes[P.cofs[0] + i - 1] * A : 0;
            for (int b = 0; b < A; ++b) trow[(b * R + q) * 32 + lane] = __ldg(P.tab + arow + b);
        }
        __syncwarp();
        const int64_t tbs = P.tbstride[0];
        uint8_t *tbrow = P.tb + (int64_t)(i0 < rho0 ? i0 : 0) * tbs;  // row i0 + q at tbrow + q tbs
        const bool origin_lane = band == 0 && lane == 0;

        int prev[R];      // this lane's rows at its previous column
        unsigned pk[R];   // traceback bytes of the current 4-column group, per row
#pragma unroll
        for (int q = 0; q < R; ++q) {
            prev[q] = kNeg;
            pk[q] = 0;
        }
        int up_prev = kNeg;  // the cell above one column back: the diagonal predecessor
        int fblk = kNeg;     // lane c holds the band above's face at column 32 * block + c
        int cblk = 0;        // lane c holds the residue code consumed at column 32 * block + c
        int bj = 0;          // the code consumed at this lane's column (shifted along the lanes)
        bool ok = true;
        // the next block's codes, loaded a block ahead (the face is loaded when the
        // block starts: loading it earlier, while the band above still writes it,
        // measured slower)
        int cnext = (lane >= 1 && lane < rho1) ? (int)c1[lane - 1] : 0;

        // One step; CHECK: some lane may be off the columns [0, rho1).
        auto step = [&](int s, auto check) {
            constexpr bool CHECK = decltype(check)::value;
            if ((s & 31) == 0 && s < rho1) {  // lane 0 enters block s / 32: stage its codes and face
                const int col = s + lane;
                cblk = cnext;
                cnext = (col + 32 < rho1) ? (int)c1[col + 31] : 0;
                if (band > 0) {
                    uint64_t t0 = 0;
                    unsigned long long e = 0;
                    if (col < rho1) e = ld_relaxed_u64(face_in + col);
                    for (int polls = 0;; ++polls) {
                        const bool good = col >= rho1 || (int)(e >> 32) == epoch;
                        fblk = col < rho1 ? (int)(unsigned)e : kNeg;
                        if (__all_sync(kFull, good)) break;
                        int expired = 0;
                        if (lane == 0) {
                            if (t0 == 0) t0 = global_ns();
                            expired = ld_volatile(L.err) != 0 || (int64_t)(global_ns() - t0) > L.spin_ns;
                        }
                        if (__shfl_sync(kFull, expired, 0)) {
                            ok = false;
                            return;
                        }
                        __nanosleep(polls < 16 ? 32 : 256);
                        if (col < rho1) e = ld_relaxed_u64(face_in + col);
                    }
                }
            }
            {  // lane l's column s - l consumes the code lane l - 1 held a step ago
                const int b0 = __shfl_sync(kFull, cblk, s & 31);
                const int b = __shfl_up_sync(kFull, bj, 1);
                bj = lane == 0 ? b0 : b;
            }
            const int from_face = __shfl_sync(kFull, fblk, s & 31);
            int up = __shfl_up_sync(kFull, prev[R - 1], 1);
            if (lane == 0) up = (band > 0 && s < rho1) ? from_face : kNeg;
            int diag = up_prev;
            up_prev = up;
            const int j = s - lane;
            const bool valid = !CHECK || (unsigned)j < (unsigned)rho1;
            const int w = i0 + 2 * j;  // W(x) of row i0
            const int *tr = trow + bj * R * 32 + lane;
            // the left and diagonal candidates do not depend on the row above: only
            // the max with the cell above, and forming the key, are chained over q
            int x[R];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                x[q] = __viaddmax_s32(diag, tr[q * 32], prev[q]);
                diag = prev[q];
            }
            unsigned m4[R];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int acc = max(up, x[q]);
                int m = (w + q - acc) & 3;
                int v = acc + m;
                if (CHECK && origin_lane && q == 0 && j == 0) {  // H(0) = 0: no move
                    v = 0;
                    m = 0;
                }
                m4[q] = (unsigned)m;
                up = v;
                if (valid) prev[q] = v;
            }
            if (valid) {
                const int sh = 8 * (j & 3);
                const bool flush = (j & 3) == 3 || j == rho1 - 1;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    pk[q] |= m4[q] << sh;
                    if (flush) {
                        if (i0 + q < rho0) *reinterpret_cast<uint32_t *>(tbrow + q * tbs + (j & ~3)) = pk[q];
                        pk[q] = 0;
                    }
                }
                if (lane == 31) st_relaxed_u64(face_out + j, face_entry(prev[R - 1], tagout));
            }
        };
        const int s_in = rho1 < 31 ? rho1 : 31;  // first step with every lane on a column (if any)
        int s = 0;
        for (; s < s_in && ok; ++s) step(s, std::true_type{});
        for (; s < rho1 && ok; ++s) step(s, std::false_type{});
        for (; s < rho1 + 31 && ok; ++s) step(s, std::true_type{});
        if (!ok) {
            if (lane == 0) atomicCAS(L.err, 0, MSA_ETIMEOUT);
            break;
        }
        // the far corner's key (the lane keeps its last column's keys), for the traceback's cross-check
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (i0 + q == rho0 - 1) *P.qcorner = prev[q];
    }
}

}  // namespace

cudaError_t launch_fill_band2(const LaunchDesc &L, int grid, cudaStream_t s) {
    fill_band2_kernel<kBandR><<<grid, kBandWarps * 32, 0, s>>>(L);
    return cudaGetLastError();
}

int fill_band2_ctas_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fill_band2_kernel<kBandR>, kBandWarps * 32, 0) !=
        cudaSuccess)
        return 0;
    return n;
}

int fill_band2_warps_per_cta() { return kBandWarps; }

}  // namespace msadp
