/*
 * ORACLE for optimal sum-of-pairs multiple sequence alignment by dynamic
 * programming (Helal et al., "Parallelizing Optimal Multiple Sequence Alignment
 * by Dynamic Programming").
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or run this code. The
 * product path (libmsadp and its CUDA kernels) shares nothing with it.
 *
 * This is the plain definition, deliberately slow and unblocked:
 *   - the k-dimensional scoring tensor has rho_i = len_i + 1 cells per axis
 *     (the initial gap character, section 3.2), N = prod rho_i cells (section 2);
 *   - every cell x != 0 is the max over its 2^k-1 lower neighbours x - e_m
 *     (section 2 counts 2^k-1 of them per cell, generalising Eq. 1), m a
 *     non-empty subset of the sequences, bit i of m meaning that sequence i
 *     consumes its residue x_i - 1 in this column and a clear bit a gap in row i;
 *   - the score of a move is the sum of pairs over the column (section 5.2):
 *     sub(a, b) for two residues, the gap value for a residue against a gap,
 *     0 for two gaps; pair scores are evaluated directly, O(k^2) per move
 *     (section 4 scores every pair of residues of a column);
 *   - H(0) = 0 (section 4 initialises the origin cell);
 *   - ties go to the lowest move mask: a candidate replaces the best only when
 *     strictly greater while masks are visited in increasing order;
 *   - traceback starts at the far corner (global alignment) and follows the
 *     stored moves back to the origin (section 2).
 *
 * Cells are visited in increasing row-major linear index (last axis fastest),
 * which is a topological order: every predecessor has a smaller index.
 * Arithmetic is int64, so no overflow is possible for any admissible input.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAXK 8

/*
 * k        number of sequences, 1 <= k <= 8
 * lens     k lengths (>= 0)
 * codes    concatenated residue codes, sequence i at offset sum_{j<i} lens[j],
 *          each code in [0, A)
 * A        alphabet size
 * sub      A*A substitution scores, row-major: sub[a*A + b] is the score of
 *          residue a (from the lower-numbered sequence) against residue b
 * gap      score of a residue against a gap (gap against gap scores 0)
 * out_score  optimal global SP score
 * out_tb   optional (may be NULL): N bytes, the chosen move mask of every cell
 *          in row-major order (0 at the origin)
 * out_H    optional (may be NULL): N int64 cell scores
 * out_masks  >= sum(lens) bytes: the move mask of every alignment column, in
 *          column order (first column first)
 * out_ncols  number of columns
 * returns 0, -1 on bad arguments, -2 when memory cannot be allocated.
 */
int oracle_msa(int k, const int32_t *lens, const uint8_t *codes, int A,
               const int32_t *sub, int32_t gap, int64_t *out_score,
               uint8_t *out_tb, int64_t *out_H, uint8_t *out_masks,
               int32_t *out_ncols)
{
    if (k < 1 || k > ORACLE_MAXK || !lens || !sub || A < 1 || !out_score ||
        !out_masks || !out_ncols)
        return -1;

    int64_t rho[ORACLE_MAXK], stride[ORACLE_MAXK];
    const uint8_t *seq[ORACLE_MAXK];
    int64_t total_len = 0;
    for (int i = 0; i < k; ++i) {
        if (lens[i] < 0)
            return -1;
        rho[i] = (int64_t)lens[i] + 1;
        seq[i] = codes + total_len;
        total_len += lens[i];
    }
    if (total_len > 0 && !codes)
        return -1;
    for (int64_t t = 0; t < total_len; ++t)
        if (codes[t] >= A)
            return -1;

    int64_t N = 1;
    for (int i = k - 1; i >= 0; --i) {
        stride[i] = N;
        N *= rho[i];
    }

    int64_t *H = out_H ? out_H : (int64_t *)malloc((size_t)N * sizeof(int64_t));
    uint8_t *TB = out_tb ? out_tb : (uint8_t *)malloc((size_t)N);
    if (!H || !TB) {
        if (!out_H) free(H);
        if (!out_tb) free(TB);
        return -2;
    }

    const int nmoves = (1 << k) - 1;
    int64_t x[ORACLE_MAXK];
    for (int64_t l = 0; l < N; ++l) {
        /* decode the cell coordinates from the linear index */
        int64_t rem = l;
        for (int i = 0; i < k; ++i) {
            x[i] = rem / stride[i];
            rem -= x[i] * stride[i];
        }
        if (l == 0) {
            H[0] = 0;
            TB[0] = 0;
            continue;
        }
        int64_t best = 0;
        int have = 0;
        int best_m = 0;
        for (int m = 1; m <= nmoves; ++m) {
            int valid = 1;
            int64_t pred = l;
            for (int i = 0; i < k; ++i) {
                if ((m >> i) & 1) {
                    if (x[i] < 1) {
                        valid = 0;
                        break;
                    }
                    pred -= stride[i];
                }
            }
            if (!valid)
                continue;
            /* sum-of-pairs score of the column this move emits */
            int64_t sp = 0;
            for (int i = 0; i < k; ++i) {
                int in_i = (m >> i) & 1;
                for (int j = i + 1; j < k; ++j) {
                    int in_j = (m >> j) & 1;
                    if (in_i && in_j) {
                        int a = seq[i][x[i] - 1];
                        int b = seq[j][x[j] - 1];
                        sp += sub[a * A + b];
                    } else if (in_i || in_j) {
                        sp += gap;
                    }
                }
            }
            int64_t cand = H[pred] + sp;
            if (!have || cand > best) {
                best = cand;
                best_m = m;
                have = 1;
            }
        }
        H[l] = best;
        TB[l] = (uint8_t)best_m;
    }

    *out_score = H[N - 1];

    /* traceback from the far corner to the origin */
    int32_t ncols = 0;
    int64_t l = N - 1;
    while (l != 0) {
        int m = TB[l];
        out_masks[ncols++] = (uint8_t)m;
        for (int i = 0; i < k; ++i)
            if ((m >> i) & 1)
                l -= stride[i];
    }
    /* columns were produced last-first */
    for (int32_t a = 0, b = ncols - 1; a < b; ++a, --b) {
        uint8_t t = out_masks[a];
        out_masks[a] = out_masks[b];
        out_masks[b] = t;
    }
    *out_ncols = ncols;

    if (!out_H) free(H);
    if (!out_tb) free(TB);
    return 0;
}
