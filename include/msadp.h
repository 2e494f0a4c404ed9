/*
 * libmsadp -- optimal multiple sequence alignment by dynamic programming on one
 * NVIDIA GB300 GPU (sm_103a).
 *
 * The method (Helal, El-Gindy, Mullin, Gaeta, "Parallelizing Optimal Multiple
 * Sequence Alignment by Dynamic Programming"):
 *   - k sequences span a k-dimensional scoring tensor of shape rho_i = len_i + 1
 *     (section 3.2: the initial gap character), N = prod rho_i cells (section 2);
 *   - every cell x != 0 takes the maximum, over its 2^k - 1 lower neighbours
 *     x - e_m (section 2; Eq. 1 is the k = 2 case), of the neighbour's score plus
 *     the sum-of-pairs (SP) score of the column the move emits (section 5.2:
 *     table score for residue/residue, `gap` for residue/gap, 0 for gap/gap);
 *     the origin scores 0 (section 4);
 *   - the optimal alignment is traced back from the far corner (section 2).
 *
 * Conventions fixed by this library where the paper is silent:
 *   - global alignment: traceback starts at (len_0, ..., len_{k-1});
 *   - move mask m: bit i set means sequence i consumes a residue in that column;
 *   - ties: the lowest move mask wins at every cell, so the returned alignment is
 *     the optimal one whose reversed column sequence is lexicographically smallest;
 *   - the substitution table must be symmetric; arithmetic is exact int32.
 *
 * All functions return MSA_OK (0) or a negative MSA_E* code; msa_poll may also
 * return MSA_PENDING. No function aborts the process. A thread-local message for
 * the last failure is available from msa_last_error().
 */
#ifndef MSADP_H
#define MSADP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MSA_OK 0
#define MSA_PENDING 1
#define MSA_EINVAL (-1)      /* bad argument: k outside [2,8], NULL pointer, negative length,
                                residue not in the alphabet, alphabet size outside [1,32] or
                                with repeated characters, non-symmetric table */
#define MSA_ETOOBIG (-2)     /* scores could leave the exact int32 range, or the problem
                                needs more device memory than the configured budget */
#define MSA_ENOMEM (-3)      /* a device or host allocation failed */
#define MSA_ECUDA (-4)       /* a CUDA call failed (message in msa_last_error) */
#define MSA_ETIMEOUT (-5)    /* a device-side dependency wait exceeded its time limit;
                                the kernel stopped cleanly and the context stays usable */
#define MSA_EBADHANDLE (-6)  /* unknown, already-consumed or cancelled request handle */

#define MSA_MAX_K 8
#define MSA_MAX_ALPHABET 32

/* ------------------------------------------------------------------------ */
/* One alignment, host buffers, synchronous.                                 */
/* ------------------------------------------------------------------------ */

/*
 * Optimal global SP alignment of k sequences (section 2; section 4; section 5.2).
 *
 * k              number of sequences, 2 <= k <= 8
 * seqs           k pointers to residue strings (not necessarily NUL-terminated)
 * lens           k lengths, each >= 0 (0 allowed: that row is all gaps)
 * alphabet       NUL-terminated string of the |S| distinct residue characters
 *                (case-sensitive), 1 <= |S| <= 32
 * subst          |S| x |S| int32 substitution scores, row-major, symmetric,
 *                indexed in alphabet order
 * gap            score of one residue against a gap (gap against gap scores 0)
 * out_score      receives the optimal SP score
 * out_alignment  caller-owned, k * (sum(lens) + 1) bytes: row i starts at
 *                i * (sum(lens) + 1), holds ncols characters ('-' for gaps) and a
 *                terminating NUL; every row has the same ncols
 *
 * All inputs are read before the call returns; the caller keeps ownership of
 * every buffer. Work runs on the stream set by msa_set_stream (default: a stream
 * owned by the library). Thread-safe (calls are serialised internally).
 */
int msa_align(int k, const char *const *seqs, const int32_t *lens, const char *alphabet,
              const int32_t *subst, int32_t gap, int32_t *out_score, char *out_alignment);

/*
 * Every alignment scoring at least OPT - delta (delta >= 0; delta = 0: every
 * optimal alignment), the further optimal and near-optimal solutions the paper
 * proposes to retrieve by forking at equally ranked paths or within a user
 * threshold (section 6). The fill keeps every cell's score (the generic tile
 * kernel); a walk on the device from the far corner follows a move only when the
 * best completion through its predecessor still reaches OPT - delta, trying the
 * moves of each column in increasing mask order, so alignments come in
 * increasing lexicographic order of their reversed column sequence (for
 * delta = 0 the first is msa_align's).
 *
 *   k, seqs, lens, alphabet, subst, gap   as for msa_align
 *   delta       score threshold below the optimum
 *   max_count   alignments to store, >= 1
 *   out_masks   max_count x sum(lens) bytes: alignment a's move masks, first column
 *               first, at a * sum(lens) (bit i set: sequence i consumes a residue)
 *   out_ncols   max_count: alignment a's column count
 *   out_scores  max_count: alignment a's SP score
 *   out_count   alignments stored
 *   out_more    1 when the walk stopped at max_count with more alignments left
 *
 * Host buffers; allocates device memory for the call and frees it; synchronous.
 * Errors as msa_align; MSA_EINVAL also for delta < 0, max_count < 1 or NULL
 * outputs.
 */
int msa_near_optimal(int k, const char *const *seqs, const int32_t *lens, const char *alphabet,
                     const int32_t *subst, int32_t gap, int64_t delta, int32_t max_count, uint8_t *out_masks,
                     int32_t *out_ncols, int64_t *out_scores, int32_t *out_count, int32_t *out_more);

/*
 * Exact search-space pruning (section 6 proposes searching only the partitions
 * where an optimal alignment can lie). Any alignment through cell x scores at
 * most U(x) = sum over pairs i < j of fwd_ij(x_i, x_j) + bwd_ij(x_i, x_j), the
 * optimal pairwise scores of the prefixes and suffixes (Eq. 1 on each pair; gap
 * against gap scores 0, section 5.2). The fill is the generic tile kernel; a
 * tile whose bound -- the sum over pairs of the largest fwd + bwd over the tile's
 * rectangle -- is below a lower bound L on the optimum holds no cell of an
 * optimal alignment and is left out. The score and alignment equal msa_align's
 * (the same tie rule) whenever L does not exceed the optimum.
 *
 *   have_lower_bound  0: L is the score of a feasible alignment the device builds
 *                     from the origin, taking at each cell the move to the
 *                     neighbour with the largest U (ties: lowest mask);
 *                     1: L = lower_bound (e.g. the score of a heuristic alignment)
 *   out_score, out_alignment  as for msa_align
 *   out_stats         (may be NULL) the bound used and what was left out
 *
 * Sequences of at most 16383 residues. Host buffers; allocates device memory for
 * the call; synchronous. MSA_EINVAL also when a given lower bound exceeds the
 * optimum (detected after the fill).
 */
typedef struct msa_prune_stats {
    int64_t lower_bound;   /* L */
    int64_t tiles;         /* tiles of the fill */
    int64_t tiles_skipped; /* tiles left out */
    int64_t cells_skipped; /* cells of the tensor in them */
    int64_t cells;         /* cells of the tensor */
} msa_prune_stats;
int msa_align_pruned(int k, const char *const *seqs, const int32_t *lens, const char *alphabet,
                     const int32_t *subst, int32_t gap, int32_t have_lower_bound, int64_t lower_bound,
                     int32_t *out_score, char *out_alignment, msa_prune_stats *out_stats);

/*
 * The pruning bound of every tile of extents `extents` (k entries >= 1; tile grid
 * G_i = ceil((len_i + 1) / extents_i), tiles numbered row-major, last axis
 * fastest), computed on the device as msa_align_pruned does:
 * out_bounds[t] = sum over pairs i < j of the largest fwd_ij + bwd_ij over the
 * tile's range of axis i times its range of axis j. out_bounds holds prod G_i
 * entries. Sequences of at most 16383 residues; host buffers; synchronous.
 */
int msa_tile_bounds(int k, const char *const *seqs, const int32_t *lens, const char *alphabet,
                    const int32_t *subst, int32_t gap, const int32_t *extents, int64_t *out_bounds);

/* Thread-local description of the last failure in this thread ("" if none). */
const char *msa_last_error(void);

/* Stream (a cudaStream_t, may be NULL for the legacy default stream) that
   msa_align and msa_autotune launch on from now on, in every thread (default: a
   non-blocking stream the library creates). The serving loop keeps its own
   streams; plans take a stream per msa_plan_execute. */
int msa_set_stream(void *stream);

/*
 * Runtime settings (integer values):
 *   "spin_timeout_ms"   device dependency-wait limit per wait (default 5000)
 *   "device_budget_mb"  device memory the serving loop may hold (default 16384)
 *   "max_batch"         problems per batched launch in the serving loop (default 64)
 *   "use_graphs"        1: the serving loop replays captured CUDA graphs (default 1)
 *   "batching"          1: serve by continuous batching; 0: one plain launch per
 *                       request, in arrival order (default 1)
 *   "fill_kernel"       0: automatic; 1: generic tile kernel; 2: k=3 column kernel;
 *                       3: k=2 band kernel; 4: k=4..6 line kernel (segments of the
 *                       last axis); 5: k=4..6 streamed line kernel (a CTA sweeps a
 *                       super-block of 32-line blocks over the whole last axis; at
 *                       k=6 the whole-column form when the last axis holds at most
 *                       25 positions, the pipelined form otherwise). The automatic
 *                       choice is 5 at k=4,5 and at k=6 for a last axis of at most 25
 *                       positions, else 4 (until msa_autotune picks otherwise); the
 *                       serving loop runs 4 where 5 would be chosen or asked for
 *   "timing"            1: msa_plan_execute records per-stage CUDA events (default 0)
 *   "verify_corner"     1: later plans and requests on the k=3 column kernel record the
 *                       far corner's score during the fill, and the traceback reports
 *                       MSA_ECUDA when the rescored alignment disagrees with it (about
 *                       3 % slower); the other fill kernels always do (default 0)
 *   "test_withhold_tile" test hook: the tile with this ticket never publishes its
 *                       completion, so its dependants time out (default -1: off)
 *   "test_poison_tb"    test hook: 1 makes msa_plan_execute fill the plan's traceback
 *                       tensor with 0xFF before the fill, so a cell the fill never
 *                       writes keeps a value no move has for k < 8 (default 0)
 *   "test_shuffle_waves" test hook: a nonzero seed makes later plans permute the
 *                       tickets inside every wave (another topological order of
 *                       the same tiles); 0 keeps the canonical order (default 0)
 */
int msa_config(const char *key, int64_t value);

/* ------------------------------------------------------------------------ */
/* Plans: device-resident inputs and outputs, asynchronous.                  */
/* ------------------------------------------------------------------------ */

typedef struct msa_plan msa_plan;

/* Everything a plan fixed, for callers and tests. */
typedef struct msa_plan_info {
    int32_t k;
    int32_t alphabet_size;
    int64_t cells;              /* prod(len_i + 1) */
    int64_t tb_strides[MSA_MAX_K]; /* bytes; traceback tensor index = sum x_i * tb_strides[i]
                                      (row-major, last axis padded) */
    int64_t tb_bytes;
    int64_t workspace_bytes;    /* device bytes the plan owns */
    int32_t tile_grid[MSA_MAX_K];
    int32_t tile_extent[MSA_MAX_K];
    int64_t tiles;
    int32_t waves;              /* tile hyperplanes (section 3.1, Eq. 2) */
    int32_t fill_kernel;        /* 1 generic tile kernel, 2 k=3 column kernel, 3 k=2 band kernel,
                                   4 k=4..6 line kernel, 5 k=4..6 streamed line kernel */
    void   *d_tb;               /* device pointer of the uint8 traceback tensor: row-major with
                                   tb_strides for the tile kernel (k <= 3) and the band kernel;
                                   tile-major for the tile kernel at k >= 4 and for the line
                                   kernels; for the k=3 column kernel a column-blocked layout
                                   (msa_plan_read_tb returns row-major) */
} msa_plan_info;

/* Result block written on the device by msa_plan_execute. */
typedef struct msa_device_result {
    int32_t score;   /* optimal SP score */
    int32_t ncols;   /* alignment columns */
    int32_t status;  /* MSA_OK; MSA_EINVAL (bad residue / asymmetric table), MSA_ETOOBIG (keys
                        could leave the int32 range), MSA_ETIMEOUT (a dependency wait ran
                        out), or another negative value if the traceback met an
                        inconsistent tensor (reported as MSA_ECUDA by msa_align) */
    int32_t pad;
} msa_device_result;

/*
 * Fix the shape of a problem (k, lens, alphabet) and allocate its device
 * workspace: residue codes, the scaled pair table, the traceback tensor
 * (1 byte per cell), the score scratch and the tile schedule (section 3.2:
 * tiles grouped into waves of equal index sum). Host work plus cudaMalloc.
 */
int msa_plan_create(int k, const int32_t *lens, const char *alphabet, msa_plan **out_plan);

/*
 * Run the whole hot path for one problem on `stream`, without host copies:
 * encode residues and scale the pair table, fill the tensor, trace back.
 *
 * d_residues  device, sum(lens) bytes: the k sequences concatenated in order
 * d_subst     device, |S|*|S| int32 symmetric table (checked on the device)
 * gap         residue/gap score
 * d_result    device msa_device_result
 * d_masks     device, >= sum(lens) bytes: move mask of every column, LAST column
 *             first (reverse order), d_result->ncols of them
 * stream      cudaStream_t or NULL
 * Returns after launching (MSA_ECUDA if a launch fails). Data errors and
 * timeouts appear in d_result->status once the stream reaches that point.
 * A plan runs one execution at a time: launches on one stream serialise.
 */
int msa_plan_execute(msa_plan *plan, const char *d_residues, const int32_t *d_subst, int32_t gap,
                     msa_device_result *d_result, uint8_t *d_masks, void *stream);

int msa_plan_get_info(const msa_plan *plan, msa_plan_info *out_info);
int msa_plan_destroy(msa_plan *plan);

/*
 * Copy the traceback tensor of the last execution to host memory, row-major
 * (info.tb_bytes bytes, layout given by info.tb_strides; the move mask of every
 * cell, 0 at the origin), converting from the device layout if needed.
 * Synchronises the plan's last stream. Diagnostic use.
 */
int msa_plan_read_tb(msa_plan *plan, void *host_dst, int64_t bytes);

/*
 * With msa_config("timing", 1), msa_plan_execute records CUDA events around its
 * three stages on the execution stream (no synchronisation). This returns the
 * mean stage durations, in milliseconds, over the executions recorded since the
 * previous call (the last 256 at most): out_ms[0] encode + tables, out_ms[1]
 * fill, out_ms[2] traceback. Synchronises on the recorded events.
 */
int msa_plan_timings(msa_plan *plan, float out_ms[3]);

/*
 * One alignment without any memory allocation (no counterpart in the paper; a
 * library facility). For callers that must not call cudaMalloc: code running
 * while another allocator owns the GPU's memory, latency-critical loops where an
 * allocation would stall, callers that cannot recover from an allocation failure
 * mid-request. Inputs, outputs and asynchrony are those of msa_plan_execute
 * (d_residues, d_subst, d_result, d_masks are the caller's device buffers; the
 * call only enqueues work on the stream and reads no host memory after it
 * returns); all
 * working memory is a fixed array of MSA_NOALLOC_SCRATCH_BYTES compiled into the
 * library, held by every GPU that loads it until the process exits. Problems
 * whose working set exceeds it (about 6 million cells) return MSA_ETOOBIG with
 * the size they would need. The first call on each device looks up the array's
 * device address; make that first call before any stream capture. Every call
 * reuses the same array: calls whose GPU work overlaps (different streams or
 * threads) race on it and must be serialised by the caller. Always uses the
 * generic tile fill.
 */
#define MSA_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int msa_align_noalloc(int k, const int32_t *lens, const char *alphabet, const char *d_residues,
                      const int32_t *d_subst, int32_t gap, msa_device_result *d_result, uint8_t *d_masks,
                      void *stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of independent requests.                     */
/* ------------------------------------------------------------------------ */

typedef struct msa_request {
    int32_t k;
    const char *const *seqs;
    const int32_t *lens;
    const char *alphabet;
    const int32_t *subst;
    int32_t gap;
} msa_request;

/*
 * Queue one alignment (same fields and rules as msa_align). Inputs are copied
 * before returning. The serving loop admits queued requests into batched
 * persistent launches while request slots and the device-memory budget allow
 * (footprint = prod(len_i + 1) traceback bytes plus score scratch), keeps
 * their tensors on the device, and overlaps new launches with running ones.
 */
int msa_submit(const msa_request *req, uint64_t *out_handle);

/*
 * MSA_PENDING while the request is queued or running; otherwise its final
 * status, with out_score / out_alignment filled as msa_align does on MSA_OK.
 * The first call that returns something other than MSA_PENDING releases the
 * handle. out_alignment needs k * (sum(lens) + 1) bytes.
 */
int msa_poll(uint64_t handle, int32_t *out_score, char *out_alignment);

/* Drop a request that has not been polled to completion. */
int msa_cancel(uint64_t handle);

/* Block until every submitted request has finished (results stay pollable). */
int msa_drain(void);

/*
 * Completion queue: wait up to timeout_us microseconds for a request to finish
 * and return MSA_OK with its handle in *out_handle (every finished request is
 * reported once, in completion order; handles already released by msa_poll or
 * msa_cancel are skipped), or MSA_PENDING when none finished in time. The
 * reported handle is then read with msa_poll. Thread-safe.
 */
int msa_wait_any(int64_t timeout_us, uint64_t *out_handle);

/* ------------------------------------------------------------------------ */
/* Host-only planner queries (no CUDA calls; usable without a GPU).         */
/* ------------------------------------------------------------------------ */

/*
 * Number of tiles on each wave of a tile grid with extents grid[0..k-1]
 * (section 3.1 Eq. 2 gives the wave count sum(grid) - k + 1; Eq. 3 the tile count
 * prod(grid); Tables 1 and 2 list these sizes). out_sizes receives
 * min(max_waves, waves) values; out_waves the total wave count.
 */
int msa_wave_sizes(int k, const int32_t *grid, int64_t *out_sizes, int32_t max_waves,
                   int32_t *out_waves);

/* The tile extents and tile grid the planner uses for these lengths. */
int msa_tile_shape(int k, const int32_t *lens, int32_t *out_extent, int32_t *out_grid);

/*
 * Tile edge of the generic kernel for k (the paper's partition size S, section
 * 3.2): the tile spans `edge` cells on every axis (k = 2: edge x 2*edge). Only
 * compiled edges are accepted (k=2: 16 32 64; k=3: 8 12 16; k=4: 4 5 6; k=5: 3 4
 * 5; k=6: 2 3 4; k=7: 2 3; k=8: 2); 0 restores the default (for k = 3 also the
 * automatic choice of the column kernel where it fits, for k = 2 of the band
 * kernel). Later plans and serving batches use the setting. Host-only,
 * thread-safe.
 */
int msa_set_tile_edge(int k, int32_t edge);
int msa_get_tile_edge(int k, int32_t *out_edge);

/*
 * Longest segment of the last axis that one tile of the line kernel (k = 4..6)
 * sweeps; the planner cuts the axis into equal segments no longer than this.
 * Only compiled lengths are accepted (k=4: 8 16 32; k=5: 16 32; k=6: 16 25); 0
 * restores the default (32, 32, 25) and the automatic choice of the line kernel
 * for k = 4..6 (its streamed form at k = 4, 5, and at k = 6 for a last axis of at
 * most 25 positions). Later plans and serving batches
 * use the setting (the streamed form has no segments). Host-only, thread-safe;
 * MSA_EINVAL for other k or lengths.
 */
int msa_set_line_segment(int k, int32_t z);
int msa_get_line_segment(int k, int32_t *out_z);

/* ------------------------------------------------------------------------ */
/* Autotuner (no counterpart in the paper, which fixes S by hand).          */
/* ------------------------------------------------------------------------ */

#define MSA_MAX_TUNING_CANDIDATES 8

typedef struct msa_tuning {
    int32_t k;
    int32_t ncand;                                   /* candidates timed */
    int32_t cand_kernel[MSA_MAX_TUNING_CANDIDATES];  /* 1 generic tiles, 2 k=3 column, 3 k=2 band, 4 lines,
                                                        5 streamed lines */
    int32_t cand_edge[MSA_MAX_TUNING_CANDIDATES];    /* tile edge; line segment for the line kernel;
                                                        0 for the column and band kernels */
    float cand_ms[MSA_MAX_TUNING_CANDIDATES];        /* mean ms of one execution (encode+fill+traceback) */
    int32_t best;                                    /* index of the chosen candidate */
} msa_tuning;

/*
 * Time every compiled tile edge for k (and the column kernel for k = 3, the band
 * kernel for k = 2, each compiled line segment for k = 4..6 and the streamed line
 * kernel for k = 4..6) on a synthetic problem with these lengths over an alphabet
 * of alphabet_size letters: one warm-up and `repeats` executions each, on the
 * library stream. The fastest becomes the choice for k (msa_set_tile_edge or
 * msa_set_line_segment, and whether the automatic kernel choice takes the band,
 * column, line or streamed line kernel).
 * Allocates device memory; synchronous.
 */
int msa_autotune(int k, const int32_t *lens, int alphabet_size, int32_t repeats, msa_tuning *out);

/* Library version string. */
const char *msa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MSADP_H */
