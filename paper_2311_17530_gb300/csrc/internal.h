// Internal structures shared by the host planner, the C-ABI and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
    int64_t qstride[MSA_MAX_K];  // score scratch strides (int32 elements)
    int64_t tbstride[MSA_MAX_K]; // traceback tensor strides (bytes)
    int64_t tile_base;           // first index of this problem in done[]
    int64_t ntiles;
    int32_t pair_min_sum;        // sum_{i<j} min(len_i, len_j): bound on pair moves
    int32_t w_corner;            // W(len)
    int32_t len_sum;
    int32_t pad0;
    const uint8_t *amap;         // device 256-entry char -> code map (0xFF: invalid)
    uint8_t *codes;              // device codes
    int32_t *tab;                // device scaled pair table ((sub - 2 gap) << B)
    int32_t *Q;                  // score scratch (full tensor for the tile kernel,
                                 // faces for the column kernel)
    int32_t *aux;                // column kernel: second face array
    uint8_t *tb;                 // traceback tensor
    int32_t *qcorner;            // packed key of the far corner
    msa_device_result *istat;    // internal status block (reset before every run)
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
    int32_t pad;
};

// Tile extents of the generic kernel, per k (compile-time in the kernel).
__host__ __device__ constexpr int tile_extent(int k, int i) {
    return k == 2 ? (i == 0 ? 32 : 64)
         : k == 3 ? 12
         : k == 4 ? 6
         : k == 5 ? 4
         : k == 6 ? 3
         : 2;
}

// Traceback box edge per k (box of (D+1)^k cells staged in shared memory).
__host__ __device__ constexpr int traceback_box(int k) {
    return k == 2 ? 200 : k == 3 ? 32 : k == 4 ? 12 : k == 5 ? 7 : k == 6 ? 4 : k == 7 ? 3 : 2;
}
constexpr int kTracebackSmem = 48 * 1024;

// Kernel entry points (host wrappers), defined in the .cu files.
// A kernel reads its per-problem IODesc from io_array[p] when io_array is set,
// else from io_single (single-problem executions pass it by value).
cudaError_t launch_encode(const ProblemDesc *d_probs, int nprob, int max_ncode,
                          const IODesc *io_array, IODesc io_single, cudaStream_t s);
cudaError_t launch_fill_tiles(int k, const LaunchDesc &L, int grid, cudaStream_t s);
int fill_tiles_ctas_per_sm(int k);
cudaError_t launch_fill_col3(const LaunchDesc &L, int grid, cudaStream_t s);
int fill_col3_ctas_per_sm();
cudaError_t launch_traceback(const ProblemDesc *d_probs, int nprob, const int32_t *err,
                             const IODesc *io_array, IODesc io_single, cudaStream_t s);

}  // namespace msadp
