// Host planner: tensor shape, mixed-radix strides, tile grid and wave order.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "internal.h"

namespace msadp {

enum FillKernel {
    kKernelAuto = 0,
    kKernelTiles = 1,
    kKernelCol3 = 2,
    kKernelBand2 = 3,
    kKernelLines = 4,
    kKernelStream = 5,
    kKernelCount = 6
};

// Kernels whose faces carry (value, epoch) entries: the plan clears them before
// the first launch and gives every launch a new epoch.
inline bool tagged_faces(int kernel) { return kernel == kKernelCol3 || kernel == kKernelStream || kernel == kKernelBand2; }

struct HostPlan {
    int k = 0;
    int A = 0;
    int kernel = kKernelTiles;
    int32_t lens[MSA_MAX_K] = {};
    int32_t rho[MSA_MAX_K] = {};
    int64_t cells = 0;
    int32_t E[MSA_MAX_K] = {};     // tile extents
    int32_t G[MSA_MAX_K] = {};     // tile grid
    int64_t gstride[MSA_MAX_K] = {};
    int64_t ntiles = 0;            // tiles (columns for the k=3 kernel)
    int64_t nunits = 0;            // tickets: ntiles, or super-blocks for the streamed line kernel
    int32_t SG[MSA_MAX_K] = {};    // streamed line kernel: grid of super-blocks
    int64_t sgstride[MSA_MAX_K] = {};
    int32_t waves = 0;
    int64_t qstride[MSA_MAX_K] = {};
    int64_t qelems = 0;            // score scratch elements
    int64_t aux_elems = 0;         // second scratch array (column kernel)
    int64_t face0_stride = 0;      // column kernel face layout
    int64_t face1_stride = 0;
    int32_t face0_rows = 0;
    int32_t face1_rows = 0;
    int64_t tbstride[MSA_MAX_K] = {};  // row-major strides (the layout msa_plan_read_tb returns)
    int64_t tbbytes = 0;               // row-major size
    int32_t tb_layout = 0;             // device layout: 0 row-major, 1 column-blocked, 2, 3 tile-major
    int64_t tb_dev_bytes = 0;          // device size of the traceback tensor
    int32_t tb_block = 0;              // tile-major layouts: bytes per tile
    int32_t lst[MSA_MAX_K] = {};       // tile-major layouts: byte stride of each axis inside a tile
    int32_t lzq = 0;                   // line kernels: entries per line in a tile's (column's) face block
    int32_t edge = 0;              // tile edge of the generic kernel (tile_ext); longest segment of the
                                   // line kernel; 0 for the column and band kernels
    int32_t check_corner = 1;      // the fill records the far corner's key and the traceback checks it
                                   // (always, but optional for the column kernel: msa_config "verify_corner")
    int32_t pair_min_sum = 0;
    int32_t w_corner = 0;
    int32_t len_sum = 0;
    std::vector<uint64_t> order;   // ticket -> tile linear index (problem bits added by callers)
    std::vector<int64_t> wave_start;  // order[wave_start[w] .. wave_start[w + 1]) is wave w (tile index sum)
};

// Tile (or column) extents the planner uses for these lengths, kernel and edge.
void tile_extents(int k, const int32_t *lens, int kernel, int edge, int32_t *E);

// Tuned choices per k (process-wide, thread-safe): the generic kernel's tile
// edge (0 restores the default) and, for k = 3 (k = 2), whether the automatic
// choice prefers the generic kernel over the column (band) kernel.
int tile_edge_for(int k);
int set_tile_edge(int k, int edge);
bool prefer_tiles_k3();
void set_prefer_tiles_k3(bool v);
// k = 2: whether the automatic choice prefers the generic kernel over the band kernel
bool prefer_tiles_k2();
void set_prefer_tiles_k2(bool v);
// k = 4 .. 6: the line kernel's longest segment (0 restores the default) and
// whether the automatic choice prefers the generic tile kernel over it.
int line_z_for(int k);
int set_line_z(int k, int z);
bool prefer_tiles_lines(int k);
void set_prefer_tiles_lines(int k, bool v);
// k = 4, 5: whether the automatic choice of the line kernel takes its streamed
// form (one column per warp over the whole last axis); reset restores the default.
bool prefer_stream(int k);
void set_prefer_stream(int k, bool v);
void reset_prefer_stream(int k);
// Whether the streamed line kernel can take these lengths (32-bit face offsets).
bool stream_fits(int k, const int32_t *lens);

// Score scratch and traceback layouts from k, rho, the kernel, tile extents and
// tile count (row-major, or tile-major for the generic kernel at k >= 4).
// False when the scratch would need offsets beyond 32 bits.
bool score_and_traceback_layout(HostPlan &hp);

// Shape, limits, tile grid and layouts of one problem without the ticket order:
// everything of make_plan that needs no heap memory. Returns MSA_OK or an MSA_E*
// code with `err` set; edge < 0 takes the current tuned edge for k.
// allow_stream = false keeps the automatic choice off the streamed line kernel
// (serving, whose arena regions are reused without clearing faces).
int plan_shape(int k, const int32_t *lens, int A, int kernel_choice, HostPlan &hp, std::string &err, int edge = -1,
               bool allow_stream = true);

// Fill `hp` for one problem: plan_shape and the ticket order. Returns MSA_OK or
// an MSA_E* code with `err` set. edge < 0 takes the current tuned edge for k.
int make_plan(int k, const int32_t *lens, int A, int kernel_choice, HostPlan &hp, std::string &err,
              int edge = -1, bool allow_stream = true);

// Units on each wave of a grid (tiles whose coordinates sum to w), w = 0, 1, ...
void wave_sizes(int k, const int32_t *grid, std::vector<int64_t> &out);

// Which fill kernel runs for this shape when the caller leaves the choice open.
int choose_kernel(int k, const int32_t *lens, int A, int requested, bool allow_stream = true);

}  // namespace msadp
