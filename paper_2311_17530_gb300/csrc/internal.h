// Internal structures shared by the host planner, the C-ABI and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "../../include/msadp.h"

namespace msadp {

// Score sentinel for predecessors outside the tensor. Every admissible packed
// key lies in (-2^29, 2^29) (checked on the device before the fill), so
// kNeg + any scaled pair sum stays below every valid key and cannot overflow.
constexpr int32_t kNeg = -(1 << 30);
constexpr int32_t kKeyLimit = 1 << 29;

// One problem of a launch. The fill works on packed keys
//   Q(x) = H'(x) * 2^B + W(x),  H'(x) = H(x) - u * |x|_1,  u = gap * (k - 1),
//   W(x) = sum_i 2^i x_i,  B = k.
// A move m emits one column whose SP score is
//   sum_{i<j in m} sub + gap * |m| * (k - |m|)
//     = u * |m| + sum_{i<j in m} (sub - 2 gap)          (|m|(k-|m|) = (k-1)|m| - 2 C(|m|,2)),
// and since |x|_1 - |x - e_m|_1 = |m| the u-term cancels against the potential:
//   H'(x) = max_m [ H'(x - e_m) + sum_{i<j in m} (sub_ij - 2 gap) ].
// With W(x) - W(x - e_m) = m the candidate key Q(x - e_m) + 2^B * pairs equals
// 2^B * value + W(x) - m, so one integer max picks the best value and, among
// equal values, the lowest mask; then m* = (W(x) - max) mod 2^B and
// Q(x) = max + m*.
struct ProblemDesc {
    int32_t k;
    int32_t A;           // alphabet size
    int32_t B;           // tie bits = k
    int32_t ncode;       // total residues
    int32_t rho[MSA_MAX_K];      // extents len_i + 1
    int32_t len[MSA_MAX_K];
    int32_t cofs[MSA_MAX_K];     // offset of sequence i in codes
    int32_t G[MSA_MAX_K];        // tile grid
    int32_t E[MSA_MAX_K];        // tile extents used by the kernel
    int64_t gstride[MSA_MAX_K];  // tile-grid row-major strides
    int64_t sgstride[MSA_MAX_K]; // streamed line kernel: strides of the grid of super-blocks (its tickets)
    int64_t qstride[MSA_MAX_K];  // score scratch strides (int32 elements)
    int64_t tbstride[MSA_MAX_K]; // traceback tensor strides (bytes)
    int64_t tile_base;           // first index of this problem in done[]
    int64_t ntiles;
    int32_t pair_min_sum;        // sum_{i<j} min(len_i, len_j): bound on pair moves
    int32_t w_corner;            // W(len)
    int32_t len_sum;
    int32_t has_qcorner;         // the fill records the corner's packed key (cross-check)
    int32_t lzq;                 // line kernels: entries per line in a tile's (column's) face block
    int32_t tb_block;            // tile-major layouts: traceback bytes per tile
    int32_t lst[MSA_MAX_K];      // tile-major layouts: byte stride of axis i inside a tile's block
    int64_t face0_stride;        // column kernel: ints per column in Q (axis-0 faces)
    int64_t face1_stride;        // column kernel: ints per column in aux (axis-1 faces)
    int32_t face0_rows;          // column kernel: skewed rows per axis-0 face
    int32_t face1_rows;          // column kernel: skewed rows per axis-1 face
    int32_t tb_layout;           // 0: row-major (tbstride); 1: column-blocked (column kernel);
                                 // 2, 3: tile-major (generic tile kernel, line kernel)
    int32_t clear_faces;         // the encode step zeroes the column kernel's faces first (serving:
                                 // the arena region may hold stale words of other requests)
    const uint8_t *amap;         // device 256-entry char -> code map (0xFF: invalid)
    uint8_t *codes;              // device codes
    int32_t *tab;                // device scaled pair table ((sub - 2 gap) << B)
    int32_t *Q;                  // score scratch (full tensor for the tile kernel,
                                 // faces for the column kernel)
    int32_t *aux;                // column kernel: second face array
    uint8_t *tb;                 // traceback tensor
    int32_t *qcorner;            // packed key of the far corner
    msa_device_result *istat;    // internal status block (reset before every run)
    const uint8_t *skip;         // generic tile kernel: per tile, nonzero = left out by the
                                 // pruning bound (nullptr: every tile is filled)
};

// Per-execution inputs and outputs of one problem.
struct IODesc {
    const char *residues;        // device, the k sequences concatenated
    const int32_t *subst;        // device, A*A table
    msa_device_result *result;   // device, caller's result block
    uint8_t *masks;              // device, caller's mask buffer (last column first)
    int32_t gap;
    int32_t pad;
};

// One persistent launch over the tiles of one or more problems of equal k.
struct LaunchDesc {
    const ProblemDesc *probs;
    const uint64_t *order;   // ticket -> (problem << 32) | tile linear index, in wave order
    int64_t ntickets;
    int32_t *done;           // per tile completion flags (or progress counters)
    int32_t *ticket;         // ticket counter
    int32_t *err;            // launch status (MSA_ETIMEOUT on a wait that ran out)
    int64_t spin_ns;         // limit of one dependency wait
    int64_t withhold;        // test hook: this ticket never publishes (-1: off)
    int32_t nprob;
    int32_t tab_ints;        // column kernel: shared-memory ints of the replicated table
    int32_t epoch;           // column and streamed line kernels: tag of this launch's face entries (>= 1)
    int32_t corner;          // column kernel: record the far corner's key (the traceback checks it)
};

// Tile shapes of the generic kernel. A shape is named by its edge E: the tile
// spans E cells on every axis, except k = 2 where it spans E x 2E. Each k has a
// few compiled shapes (the autotuner picks among them; kTileEdgeDefault is used
// until it has); the kernel is instantiated per (k, E).
__host__ __device__ constexpr int tile_ext(int k, int edge, int i) { return k == 2 && i == 1 ? 2 * edge : edge; }
constexpr int kMaxTileEdges = 3;
// From this k on the generic kernel keeps its score scratch and traceback bytes
// tile-major (each tile one contiguous block), so halo reads and write-back are
// block transfers.
constexpr int kTileMajorMinK = 4;
// candidate edges per k (0 = unused slot)
__host__ __device__ constexpr int tile_edge_candidate(int k, int idx) {
    return k == 2 ? (idx == 0 ? 16 : idx == 1 ? 32 : 64)
         : k == 3 ? (idx == 0 ? 8 : idx == 1 ? 12 : 16)
         : k == 4 ? (idx == 0 ? 4 : idx == 1 ? 5 : 6)
         : k == 5 ? (idx == 0 ? 3 : idx == 1 ? 4 : 5)
         : k == 6 ? (idx == 0 ? 2 : idx == 1 ? 3 : 4)
         : k == 7 ? (idx == 0 ? 2 : idx == 1 ? 3 : 0)
         : (idx == 0 ? 2 : 0);
}
__host__ __device__ constexpr int tile_edge_default(int k) {
    return k == 2 ? 32 : k == 3 ? 12 : k == 4 ? 6 : k == 5 ? 4 : k == 6 ? 3 : 2;
}
__host__ __device__ constexpr bool tile_edge_valid(int k, int edge) {
    return edge > 0 && (tile_edge_candidate(k, 0) == edge || tile_edge_candidate(k, 1) == edge ||
                        tile_edge_candidate(k, 2) == edge);
}

// Line-sweep kernel geometry shared by the planner and the kernel (k = 4 .. 6;
// see fill_lines.cuh). A tile is a block of 32 lines over the first k - 1 axes
// (extents line_ext) times a segment of the last axis of at most Z positions
// (the compiled candidates below); lane l owns the line whose local coordinates
// are the mixed-radix digits of l (last line axis fastest) and is skewed by
// their sum.
constexpr int kLinesMinK = 4, kLinesMaxK = 6;
__host__ __device__ constexpr int line_ext(int K, int i) {
    return K == 4 ? (i == 0 ? 2 : 4)   // 2 x 4 x 4
         : K == 5 ? (i == 3 ? 4 : 2)   // 2 x 2 x 2 x 4
                  : 2;                 // k = 6: 2^5
}
constexpr int kMaxLineSegments = 3;
__host__ __device__ constexpr int line_z_candidate(int k, int idx) {
    return k == 4 ? (idx == 0 ? 8 : idx == 1 ? 16 : idx == 2 ? 32 : 0)
         : k == 5 ? (idx == 0 ? 16 : idx == 1 ? 32 : 0)
         : k == 6 ? (idx == 0 ? 16 : idx == 1 ? 25 : 0)
                  : 0;
}
__host__ __device__ constexpr int line_z_default(int k) { return k == 4 ? 32 : k == 5 ? 32 : 25; }
__host__ __device__ constexpr bool line_z_valid(int k, int z) {
    return z > 0 && k >= kLinesMinK && k <= kLinesMaxK &&
           (line_z_candidate(k, 0) == z || line_z_candidate(k, 1) == z || line_z_candidate(k, 2) == z);
}
__host__ __device__ constexpr int line_lstride(int K, int i) {  // lane stride of line axis i
    int s = 1;
    for (int j = K - 2; j > i; --j) s *= line_ext(K, j);
    return s;
}
__host__ __device__ constexpr int line_skew_max(int K) {
    int s = 0;
    for (int i = 0; i < K - 1; ++i) s += line_ext(K, i) - 1;
    return s;
}

// Streamed line kernel (fill_lines_stream.cuh): a CTA of stream_warps(k) warps
// sweeps a super-block of line blocks (each warp one 32-line block of the line
// kernel, extents line_ext; the warps form a grid of extents stream_wg) over the
// whole last axis in lockstep, in blocks of stream_block(k) steps; super-blocks
// exchange faces as (value, epoch) entries indexed by time.
constexpr int kStreamMinK = 4, kStreamMaxK = 6;
__host__ __device__ constexpr int stream_block(int K) { return K == 6 ? 4 : 8; }  // steps per block = times per face chunk
// k = 6: the streamed kernel's whole-column form (fill_lines_wide.cuh) holds a
// last axis of at most kWideZ positions; longer ones take the pipelined form.
constexpr int kWideZ = 25;
__host__ __device__ constexpr int stream_wg(int K, int i) {  // warps along line axis i
    return K == 4 ? 2 : (i < 2 ? 2 : 1);  // k = 4: 2 x 2 x 2; k = 5: 2 x 2 x 1 x 1; k = 6: 2 x 2 x 1 x 1 x 1
}
__host__ __device__ constexpr int stream_warps(int K) {
    int w = 1;
    for (int i = 0; i < K - 1; ++i) w *= stream_wg(K, i);
    return w;
}
__host__ __device__ constexpr int stream_sb(int K, int i) { return stream_wg(K, i) * line_ext(K, i); }
__host__ __device__ constexpr int stream_skew_max(int K) {  // largest sum of local coordinates in a super-block
    int s = 0;
    for (int i = 0; i < K - 1; ++i) s += stream_sb(K, i) - 1;
    return s;
}
__host__ __device__ constexpr int stream_face_lines(int K) {  // lines of a super-block with some c_i = SB_i - 1
    int all = 1, inner = 1;
    for (int i = 0; i < K - 1; ++i) {
        all *= stream_sb(K, i);
        inner *= stream_sb(K, i) - 1;
    }
    return all - inner;
}

// k = 2 band kernel: rows per lane (a band is 32 of them per lane, 32 lanes).
constexpr int kBand2RowsPerLane = 4;

// k = 3 column kernel geometry (shared by the planner and the kernel).
//
// A CTA owns a column: rows x0 in [A*WR, A*WR + WR) (warp w holds rows
// w*R .. w*R + R - 1 in registers), lanes x1 in [32B, 32B + 32), and sweeps axis
// 2. All of its warps share one clock, the CTA time T: at time T lane l of warp
// w computes, for each of its rows r, the cell with CTA row rho = w*R + r at
// x2 = T - l - rho. Every predecessor of that cell is then produced at time T-1
// or T-2 (same lane, lane l-1, or row rho-1), so rings indexed by T connect the
// warps of a CTA and faces indexed by T connect neighbouring columns.
namespace c3 {
constexpr int R = 4;          // rows per warp (registers)
constexpr int W = 8;          // compute warps per CTA
constexpr int WR = R * W;     // rows per CTA
constexpr int U = 8;          // steps per block (the unrolled loop body), a multiple of 2R
constexpr int SI = 32;        // depth of the rings into each warp (CTA-time entries), multiple of U
constexpr int SF = 64;        // depth of the staged axis-1 face ring, multiple of U
constexpr int F1S = WR + 4;   // ints per staged axis-1 face row: [3] row -1, [4 + rho] row rho
constexpr int THREADS = 32 * (W + 1);  // compute warps + one staging warp
constexpr int MAXA = 24;      // largest alphabet (replicated pair table)
constexpr int MAXRHO2 = 4096; // largest axis-2 extent (staged codes)
constexpr int CODEPAD = 96;   // axis-2 code staging pad on both sides
constexpr int kSentinelPair = -(1 << 27);  // pair score of a move into x2 <= 0 (no residue)
static_assert(U % (2 * R) == 0 && SI % U == 0 && SF % U == 0 && (WR == 16 || WR == 32), "column geometry");
// CTA-time steps of one column: the last cell x2 = rho2 - 1 of lane 31, row
// WR - 1 is computed at T = rho2 + WR + 29; rounded up to whole blocks. A column
// runs T = -U .. nsteps - 1: the first block only fills the pipeline (its cells
// lie at x2 < 0) so that time 0 starts with every candidate prepared.
__host__ __device__ constexpr int nsteps(int rho2) { return (rho2 + WR + 30 + U - 1) / U * U; }
// Faces between columns hold (value, tag) pairs, one 8-byte entry each, stored
// from T = -U on (row T + U):
//   F0[T][l]    row WR - 1 of the column at CTA time T, lane l (read by the column below)
//   F1[T][rho]  lane 31 of the column at CTA time T, row rho (read by the columns to the
//               right and, for rho = WR - 1, diagonally below-right)
constexpr int F0W = 32 * 2;   // ints per F0 row
constexpr int F1W = WR * 2;   // ints per F1 row
__host__ __device__ constexpr int face0_rows(int rho2) { return nsteps(rho2) + U; }
__host__ __device__ constexpr int face1_rows(int rho2) { return nsteps(rho2) + U; }
// Traceback bytes are stored column-blocked and skewed: column (A, B) owns
// (nsteps(rho2) + U) * W * 32 * R bytes, and the move of cell (x0 = A*WR + w*R + r,
// x1 = 32B + l, x2) sits at (((T + U)*W + w)*32 + l)*R + r with
// T = x2 + l + w*R + r, so each warp step stores one contiguous run of 32 lanes x
// R bytes.
__host__ __device__ constexpr int64_t tb_col_bytes(int rho2) { return (int64_t)(nsteps(rho2) + U) * W * 32 * R; }
}  // namespace c3

// Traceback box edge D for the row-major layout with k <= 3 (the box [x-D, x] is
// staged in shared memory, rows along the last axis in 16-byte granules, so a
// staged row holds at most round_up(D + 16, 16) bytes); larger k reads cells
// directly.
__host__ __device__ constexpr int traceback_box(int k) { return k == 2 ? 192 : 28; }
constexpr int kTracebackSmem = 224 * 1024;  // two 112 KB windows (column layout)
// The traceback tensor's last axis is padded to this many bytes (16-byte rows).
constexpr int kTbRowAlign = 16;

// Runs a host action once per device (the current device when called), e.g. a
// kernel attribute, so that launch wrappers make no such call while a stream is
// being captured into a graph after the first use.
class DeviceOnce {
  public:
    template <class F>
    cudaError_t run(F f) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return f();
        const unsigned long long bit = 1ull << dev;
        if (done_.load(std::memory_order_acquire) & bit) return cudaSuccess;
        std::lock_guard<std::mutex> g(mu_);
        if (done_.load(std::memory_order_relaxed) & bit) return cudaSuccess;
        e = f();
        if (e == cudaSuccess) done_.fetch_or(bit, std::memory_order_release);
        return e;
    }

  private:
    std::atomic<unsigned long long> done_{0};
    std::mutex mu_;
};

// Kernel entry points (host wrappers), defined in the .cu files.
// A kernel reads its per-problem IODesc from io_array[p] when io_array is set,
// else from io_single (single-problem executions pass it by value).
cudaError_t launch_encode(const ProblemDesc *d_probs, int nprob, int max_ncode,
                          const IODesc *io_array, IODesc io_single, cudaStream_t s, int min_blocks = 1);
cudaError_t launch_fill_tiles(int k, int edge, const LaunchDesc &L, int grid, cudaStream_t s);
cudaError_t prepare_kernel_attributes();
cudaError_t traceback_attributes();
int fill_tiles_ctas_per_sm(int k, int edge);
int fill_tiles_warps_per_cta(int k, int edge);
cudaError_t launch_fill_col3(const LaunchDesc &L, int grid, int smem, cudaStream_t s);
int fill_col3_ctas_per_sm(int smem);
cudaError_t launch_fill_band2(const LaunchDesc &L, int grid, cudaStream_t s);
cudaError_t launch_fill_lines(int k, int z, const LaunchDesc &L, int grid, cudaStream_t s);
int fill_lines_ctas_per_sm(int k, int z);
int fill_lines_warps_per_cta(int k, int z);
cudaError_t launch_fill_stream(int k, const LaunchDesc &L, int grid, cudaStream_t s, int rho_s);  // rho_s: last axis
int fill_stream_ctas_per_sm(int k);
int fill_band2_ctas_per_sm();
int fill_band2_warps_per_cta();
int col3_smem_bytes(int alphabet_size);
// Outputs and stack of the near-optimal enumeration (near_optimal.cu), device memory:
// masks max_count x len_sum (first column first), ncols and scores per alignment,
// count_more[2] = {alignments stored, 1 when more were left (2: walk inconsistent)},
// and per depth (len_sum + 1 entries) the move taken, the score so far and the next mask.
struct NearOut {
    uint8_t *masks;
    int32_t *ncols;
    int64_t *scores;
    int32_t *count_more;
    uint8_t *path;
    int64_t *acc;
    int32_t *next;
};
cudaError_t launch_near_optimal(const ProblemDesc *d_prob, IODesc io, int64_t delta, int32_t max_count, NearOut o,
                                cudaStream_t s);

// Exact pruning (prune.cu): the pairwise tables of every pair i < j, the largest
// fwd + bwd of every tile rectangle, the tiles' bounds and, against a lower
// bound L on the optimum, the tiles the fill leaves out. Device pointers:
// tables (for pair pr at toff[pr]: fwd then bwd, (len_i + 1) x (len_j + 1) int32
// each, row-major), blk (for pair pr at boff[pr]: G_i x G_j rectangle maxima),
// bound (ntiles, optional), skip (ntiles flags, optional), lower (L: written by
// the greedy walk, or set by the caller), stats ({tiles left out, their cells}).
constexpr int kMaxPairs = MSA_MAX_K * (MSA_MAX_K - 1) / 2;
struct PruneDesc {
    int32_t k, A, gap, npairs, len_sum;
    int32_t greedy;  // 1: L from the greedy walk; 0: *lower set by the caller
    int32_t len[MSA_MAX_K], cofs[MSA_MAX_K], E[MSA_MAX_K], G[MSA_MAX_K];
    int64_t gstride[MSA_MAX_K];
    int32_t pi[kMaxPairs], pj[kMaxPairs];
    int64_t toff[kMaxPairs], boff[kMaxPairs];
    int64_t ntiles, nblocks, table_elems;
    const uint8_t *codes;
    const int32_t *sub;
    int32_t *tables;
    int64_t *blk;
    int64_t *bound;
    uint8_t *skip;
    int64_t *lower;
    int64_t *stats;
};
cudaError_t launch_prune(const PruneDesc &D, bool greedy, cudaStream_t s);
cudaError_t launch_traceback(const ProblemDesc *d_probs, int nprob, const int32_t *err,
                             const IODesc *io_array, IODesc io_single, cudaStream_t s);

}  // namespace msadp
