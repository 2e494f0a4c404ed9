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

/*
 * Exact search-space pruning, the restriction of the search space the paper
 * leaves for future work (section 6), by the bound of Carrillo and Lipman: the
 * score of an alignment is the sum over pairs of sequences of the scores of its
 * pairwise projections (section 5.2 scores gap against gap 0, so dropping those
 * columns leaves each projection's score unchanged), and a projection of an
 * alignment through cell x is a pairwise alignment through (x_i, x_j).
 *
 * oracle_pair_tables: for residue codes a (na) and b (nb), two (na+1) x (nb+1)
 * int64 arrays in row-major order,
 *   fwd[p][q] = optimal global score of a[0:p] against b[0:q],
 *   bwd[p][q] = optimal global score of a[p:na] against b[q:nb],
 * by the pairwise recurrence (Eq. 1) with sub[x*A + y] for residue x of a
 * against residue y of b and `gap` for a residue against a gap.
 * Returns 0, or -1 on bad arguments.
 */
#define ORACLE_NEG (INT64_MIN / 4)

int oracle_pair_tables(const uint8_t *a, int32_t na, const uint8_t *b, int32_t nb, int A,
                       const int32_t *sub, int32_t gap, int64_t *fwd, int64_t *bwd)
{
    if (na < 0 || nb < 0 || A < 1 || !sub || !fwd || !bwd || (na > 0 && !a) || (nb > 0 && !b))
        return -1;
    for (int32_t p = 0; p < na; ++p)
        if (a[p] >= A)
            return -1;
    for (int32_t q = 0; q < nb; ++q)
        if (b[q] >= A)
            return -1;
    const int64_t W = (int64_t)nb + 1;
    for (int64_t p = 0; p <= na; ++p) {
        for (int64_t q = 0; q <= nb; ++q) {
            if (p == 0 && q == 0) {
                fwd[0] = 0;
                continue;
            }
            int64_t best = ORACLE_NEG;
            if (p > 0 && fwd[(p - 1) * W + q] + gap > best)
                best = fwd[(p - 1) * W + q] + gap;
            if (q > 0 && fwd[p * W + q - 1] + gap > best)
                best = fwd[p * W + q - 1] + gap;
            if (p > 0 && q > 0 && fwd[(p - 1) * W + q - 1] + sub[a[p - 1] * A + b[q - 1]] > best)
                best = fwd[(p - 1) * W + q - 1] + sub[a[p - 1] * A + b[q - 1]];
            fwd[p * W + q] = best;
        }
    }
    for (int64_t p = na; p >= 0; --p) {
        for (int64_t q = nb; q >= 0; --q) {
            if (p == na && q == nb) {
                bwd[p * W + q] = 0;
                continue;
            }
            int64_t best = ORACLE_NEG;
            if (p < na && bwd[(p + 1) * W + q] + gap > best)
                best = bwd[(p + 1) * W + q] + gap;
            if (q < nb && bwd[p * W + q + 1] + gap > best)
                best = bwd[p * W + q + 1] + gap;
            if (p < na && q < nb && bwd[(p + 1) * W + q + 1] + sub[a[p] * A + b[q]] > best)
                best = bwd[(p + 1) * W + q + 1] + sub[a[p] * A + b[q]];
            bwd[p * W + q] = best;
        }
    }
    return 0;
}

/*
 * oracle_msa restricted to the cells x whose bound
 *   U(x) = sum_{i<j} fwd_ij[x_i][x_j] + bwd_ij[x_i][x_j]
 * reaches lower_bound (any alignment through x scores at most U(x)). A cell left
 * out is never a predecessor and never on the path. When lower_bound does not
 * exceed the optimum, no cell of any optimal alignment is left out, and neither
 * is any optimal predecessor of such a cell, so score and alignment equal
 * oracle_msa's (same tie rule: masks ascending, strict >).
 *
 * out_excluded receives the number of cells left out by the bound.
 * Returns 0; -1 bad arguments; -2 out of memory; -3 when no path of kept cells
 * reaches the corner or the best one scores below lower_bound (the bound was
 * above the optimum).
 */
int oracle_msa_pruned(int k, const int32_t *lens, const uint8_t *codes, int A,
                      const int32_t *sub, int32_t gap, int64_t lower_bound,
                      int64_t *out_score, uint8_t *out_masks, int32_t *out_ncols,
                      int64_t *out_excluded)
{
    if (k < 2 || k > ORACLE_MAXK || !lens || !sub || A < 1 || !out_score ||
        !out_masks || !out_ncols || !out_excluded)
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

    /* pairwise tables, pair (i, j) with i < j */
    int64_t *fwd[ORACLE_MAXK][ORACLE_MAXK] = {{0}};
    int64_t *bwd[ORACLE_MAXK][ORACLE_MAXK] = {{0}};
    int rc = 0;
    for (int i = 0; i < k && rc == 0; ++i)
        for (int j = i + 1; j < k && rc == 0; ++j) {
            size_t n = (size_t)(rho[i] * rho[j]);
            fwd[i][j] = (int64_t *)malloc(n * sizeof(int64_t));
            bwd[i][j] = (int64_t *)malloc(n * sizeof(int64_t));
            if (!fwd[i][j] || !bwd[i][j])
                rc = -2;
            else
                rc = oracle_pair_tables(seq[i], lens[i], seq[j], lens[j], A, sub, gap,
                                        fwd[i][j], bwd[i][j]);
        }
    int64_t *H = rc ? NULL : (int64_t *)malloc((size_t)N * sizeof(int64_t));
    uint8_t *TB = rc ? NULL : (uint8_t *)malloc((size_t)N);
    if (rc == 0 && (!H || !TB))
        rc = -2;

    const int nmoves = (1 << k) - 1;
    int64_t excluded = 0;
    int64_t x[ORACLE_MAXK];
    for (int64_t l = 0; rc == 0 && l < N; ++l) {
        int64_t rem = l;
        for (int i = 0; i < k; ++i) {
            x[i] = rem / stride[i];
            rem -= x[i] * stride[i];
        }
        int64_t U = 0;
        for (int i = 0; i < k; ++i)
            for (int j = i + 1; j < k; ++j) {
                int64_t idx = x[i] * rho[j] + x[j];
                U += fwd[i][j][idx] + bwd[i][j][idx];
            }
        TB[l] = 0;
        if (U < lower_bound) {
            H[l] = ORACLE_NEG;
            ++excluded;
            continue;
        }
        if (l == 0) {
            H[0] = 0;
            continue;
        }
        int64_t best = ORACLE_NEG;
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
            if (!valid || H[pred] == ORACLE_NEG)
                continue;
            int64_t sp = 0;
            for (int i = 0; i < k; ++i) {
                int in_i = (m >> i) & 1;
                for (int j = i + 1; j < k; ++j) {
                    int in_j = (m >> j) & 1;
                    if (in_i && in_j)
                        sp += sub[seq[i][x[i] - 1] * A + seq[j][x[j] - 1]];
                    else if (in_i || in_j)
                        sp += gap;
                }
            }
            int64_t cand = H[pred] + sp;
            if (best_m == 0 || cand > best) {
                best = cand;
                best_m = m;
            }
        }
        H[l] = best_m ? best : ORACLE_NEG;
        TB[l] = (uint8_t)best_m;
    }

    if (rc == 0 && (H[N - 1] == ORACLE_NEG || H[N - 1] < lower_bound))
        rc = -3;
    if (rc == 0) {
        *out_score = H[N - 1];
        *out_excluded = excluded;
        int32_t ncols = 0;
        int64_t l = N - 1;
        while (l != 0) {
            int m = TB[l];
            out_masks[ncols++] = (uint8_t)m;
            for (int i = 0; i < k; ++i)
                if ((m >> i) & 1)
                    l -= stride[i];
        }
        for (int32_t a = 0, b = ncols - 1; a < b; ++a, --b) {
            uint8_t t = out_masks[a];
            out_masks[a] = out_masks[b];
            out_masks[b] = t;
        }
        *out_ncols = ncols;
    }
    free(H);
    free(TB);
    for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j) {
            free(fwd[i][j]);
            free(bwd[i][j]);
        }
    return rc;
}

/*
 * Optimal and near-optimal alignments, the other extension the paper proposes
 * (section 6: further solutions by forking at equally ranked paths, or within a
 * user threshold). Every alignment scoring at least OPT - delta (delta >= 0;
 * delta = 0: every optimal alignment), enumerated from the far corner with the
 * moves of each column tried in increasing mask order, so alignments come in
 * increasing lexicographic order of their reversed column sequence (for
 * delta = 0 the first one is oracle_msa's). A move from x to its predecessor p is followed only
 * when H(p) + SP(move) + (score of the columns already fixed) >= OPT - delta,
 * H being the full forward tensor: H(p) is the best any completion through p
 * can add, so no qualifying alignment is missed and none below the threshold is
 * produced.
 *
 * Up to max_count alignments are stored: alignment a's masks (first column
 * first) at out_masks + a * sum(lens), its column count in out_ncols[a], its
 * score in out_scores[a]. *out_count receives the number stored, *out_more 1 when
 * the enumeration stopped at max_count with more alignments left, else 0.
 * Returns 0; -1 bad arguments; -2 out of memory.
 */
int oracle_msa_near_optimal(int k, const int32_t *lens, const uint8_t *codes, int A,
                            const int32_t *sub, int32_t gap, int64_t delta, int32_t max_count,
                            uint8_t *out_masks, int32_t *out_ncols, int64_t *out_scores,
                            int32_t *out_count, int32_t *out_more)
{
    if (k < 1 || k > ORACLE_MAXK || !lens || !sub || A < 1 || delta < 0 || max_count < 1 ||
        !out_masks || !out_ncols || !out_scores || !out_count || !out_more)
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
    int64_t N = 1;
    for (int i = k - 1; i >= 0; --i) {
        stride[i] = N;
        N *= rho[i];
    }
    int64_t *H = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    uint8_t *tbuf = (uint8_t *)malloc((size_t)N);
    uint8_t *path = (uint8_t *)malloc((size_t)total_len + 1);
    int64_t *cell = (int64_t *)malloc(((size_t)total_len + 1) * sizeof(int64_t));
    int64_t *acc = (int64_t *)malloc(((size_t)total_len + 1) * sizeof(int64_t));
    int *next_m = (int *)malloc(((size_t)total_len + 1) * sizeof(int));
    int rc = 0;
    if (!H || !tbuf || !path || !cell || !acc || !next_m)
        rc = -2;
    int64_t score = 0;
    int32_t nc = 0;
    if (rc == 0)
        rc = oracle_msa(k, lens, codes, A, sub, gap, &score, tbuf, H, path, &nc);
    const int nmoves = (1 << k) - 1;
    const int64_t threshold = score - delta;
    int32_t count = 0;
    *out_more = 0;
    if (rc == 0) {
        /* depth d: cell[d] reached after d columns fixed (from the corner), acc[d]
           their score, next_m[d] the next move to try there */
        int32_t d = 0;
        cell[0] = N - 1;
        acc[0] = 0;
        next_m[0] = 1;
        while (d >= 0) {
            const int64_t l = cell[d];
            if (l == 0) { /* reached the origin: an alignment */
                if (count == max_count) {
                    *out_more = 1;
                    break;
                }
                uint8_t *dst = out_masks + (size_t)count * (size_t)total_len;
                for (int32_t c = 0; c < d; ++c)
                    dst[c] = path[d - 1 - c];
                out_ncols[count] = d;
                out_scores[count] = acc[d];
                ++count;
                --d;
                continue;
            }
            int64_t x[ORACLE_MAXK];
            int64_t rem = l;
            for (int i = 0; i < k; ++i) {
                x[i] = rem / stride[i];
                rem -= x[i] * stride[i];
            }
            int advanced = 0;
            while (next_m[d] <= nmoves) {
                const int m = next_m[d]++;
                int valid = 1;
                int64_t pred = l;
                for (int i = 0; i < k; ++i)
                    if ((m >> i) & 1) {
                        if (x[i] < 1) {
                            valid = 0;
                            break;
                        }
                        pred -= stride[i];
                    }
                if (!valid)
                    continue;
                int64_t sp = 0;
                for (int i = 0; i < k; ++i) {
                    int in_i = (m >> i) & 1;
                    for (int j = i + 1; j < k; ++j) {
                        int in_j = (m >> j) & 1;
                        if (in_i && in_j)
                            sp += sub[seq[i][x[i] - 1] * A + seq[j][x[j] - 1]];
                        else if (in_i || in_j)
                            sp += gap;
                    }
                }
                if (H[pred] + sp + acc[d] >= threshold) {
                    path[d] = (uint8_t)m;
                    cell[d + 1] = pred;
                    acc[d + 1] = acc[d] + sp;
                    next_m[d + 1] = 1;
                    ++d;
                    advanced = 1;
                    break;
                }
            }
            if (!advanced)
                --d;
        }
    }
    *out_count = count;
    free(H);
    free(tbuf);
    free(path);
    free(cell);
    free(acc);
    free(next_m);
    return rc;
}

/*
 * Per-tile bound for pruning whole partitions (section 6 proposes searching only
 * the partitions where an optimal alignment can lie). Tiles have extents E[i]
 * per axis (tile grid G_i = ceil((len_i + 1) / E_i), tiles numbered row-major,
 * last axis fastest); out_bound[t] = sum over pairs i < j of the largest
 * fwd_ij + bwd_ij over the tile's range of axis i times its range of axis j.
 * A sum of maxima, so never below the largest cell bound U(x) inside the tile:
 * a tile whose bound is below a lower bound on the optimum holds no cell of any
 * optimal alignment. out_bound needs prod G_i entries.
 * Returns 0; -1 bad arguments; -2 out of memory.
 */
int oracle_tile_bounds(int k, const int32_t *lens, const uint8_t *codes, int A,
                       const int32_t *sub, int32_t gap, const int32_t *E, int64_t *out_bound)
{
    if (k < 2 || k > ORACLE_MAXK || !lens || !sub || A < 1 || !E || !out_bound)
        return -1;
    int64_t rho[ORACLE_MAXK], G[ORACLE_MAXK], gstride[ORACLE_MAXK];
    const uint8_t *seq[ORACLE_MAXK];
    int64_t total_len = 0;
    for (int i = 0; i < k; ++i) {
        if (lens[i] < 0 || E[i] < 1)
            return -1;
        rho[i] = (int64_t)lens[i] + 1;
        G[i] = (rho[i] + E[i] - 1) / E[i];
        seq[i] = codes + total_len;
        total_len += lens[i];
    }
    if (total_len > 0 && !codes)
        return -1;
    int64_t NT = 1;
    for (int i = k - 1; i >= 0; --i) {
        gstride[i] = NT;
        NT *= G[i];
    }
    for (int64_t t = 0; t < NT; ++t)
        out_bound[t] = 0;
    int rc = 0;
    for (int i = 0; i < k && rc == 0; ++i)
        for (int j = i + 1; j < k && rc == 0; ++j) {
            size_t n = (size_t)(rho[i] * rho[j]);
            int64_t *fwd = (int64_t *)malloc(n * sizeof(int64_t));
            int64_t *bwd = (int64_t *)malloc(n * sizeof(int64_t));
            int64_t *blk = (int64_t *)malloc((size_t)(G[i] * G[j]) * sizeof(int64_t));
            if (!fwd || !bwd || !blk)
                rc = -2;
            else
                rc = oracle_pair_tables(seq[i], lens[i], seq[j], lens[j], A, sub, gap, fwd, bwd);
            if (rc == 0) {
                /* largest fwd + bwd over each block of the (i, j) plane */
                for (int64_t b = 0; b < G[i] * G[j]; ++b)
                    blk[b] = ORACLE_NEG;
                for (int64_t p = 0; p < rho[i]; ++p)
                    for (int64_t q = 0; q < rho[j]; ++q) {
                        int64_t v = fwd[p * rho[j] + q] + bwd[p * rho[j] + q];
                        int64_t b = (p / E[i]) * G[j] + q / E[j];
                        if (v > blk[b])
                            blk[b] = v;
                    }
                for (int64_t t = 0; t < NT; ++t) {
                    int64_t ci = (t / gstride[i]) % G[i], cj = (t / gstride[j]) % G[j];
                    out_bound[t] += blk[ci * G[j] + cj];
                }
            }
            free(fwd);
            free(bwd);
            free(blk);
        }
    return rc;
}

/*
 * oracle_msa with the cells flagged in `excluded` (N bytes, row-major, nonzero:
 * left out) never used: not computed, never a predecessor, never on the path.
 * For parity of a fill that skips tiles: when every flagged cell has a bound
 * below a lower bound on the optimum, score and alignment equal oracle_msa's.
 * Returns 0; -1 bad arguments; -2 out of memory; -3 when no path of kept cells
 * reaches the corner.
 */
int oracle_msa_excluding(int k, const int32_t *lens, const uint8_t *codes, int A,
                         const int32_t *sub, int32_t gap, const uint8_t *excluded,
                         int64_t *out_score, uint8_t *out_masks, int32_t *out_ncols)
{
    if (k < 1 || k > ORACLE_MAXK || !lens || !sub || A < 1 || !excluded || !out_score ||
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
    int64_t *H = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    uint8_t *TB = (uint8_t *)malloc((size_t)N);
    if (!H || !TB) {
        free(H);
        free(TB);
        return -2;
    }
    const int nmoves = (1 << k) - 1;
    int64_t x[ORACLE_MAXK];
    for (int64_t l = 0; l < N; ++l) {
        int64_t rem = l;
        for (int i = 0; i < k; ++i) {
            x[i] = rem / stride[i];
            rem -= x[i] * stride[i];
        }
        TB[l] = 0;
        if (excluded[l]) {
            H[l] = ORACLE_NEG;
            continue;
        }
        if (l == 0) {
            H[0] = 0;
            continue;
        }
        int64_t best = ORACLE_NEG;
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
            if (!valid || H[pred] == ORACLE_NEG)
                continue;
            int64_t sp = 0;
            for (int i = 0; i < k; ++i) {
                int in_i = (m >> i) & 1;
                for (int j = i + 1; j < k; ++j) {
                    int in_j = (m >> j) & 1;
                    if (in_i && in_j)
                        sp += sub[seq[i][x[i] - 1] * A + seq[j][x[j] - 1]];
                    else if (in_i || in_j)
                        sp += gap;
                }
            }
            int64_t cand = H[pred] + sp;
            if (best_m == 0 || cand > best) {
                best = cand;
                best_m = m;
            }
        }
        H[l] = best_m ? best : ORACLE_NEG;
        TB[l] = (uint8_t)best_m;
    }
    int rc = 0;
    if (H[N - 1] == ORACLE_NEG) {
        rc = -3;
    } else {
        *out_score = H[N - 1];
        int32_t ncols = 0;
        int64_t l = N - 1;
        while (l != 0) {
            int m = TB[l];
            out_masks[ncols++] = (uint8_t)m;
            for (int i = 0; i < k; ++i)
                if ((m >> i) & 1)
                    l -= stride[i];
        }
        for (int32_t a = 0, b = ncols - 1; a < b; ++a, --b) {
            uint8_t t = out_masks[a];
            out_masks[a] = out_masks[b];
            out_masks[b] = t;
        }
        *out_ncols = ncols;
    }
    free(H);
    free(TB);
    return rc;
}
