"""Independent restatements used to pin the oracle (no code shared with it).

* ``column_score`` scores one alignment column by the sum-of-pairs rule of
  section 5.2 (residue/residue: table, residue/gap: gap value, gap/gap: 0).
* ``brute_force`` enumerates every alignment (every monotone path of non-empty
  0/1 moves from the corner back to the origin) and keeps the best; masks are
  tried in increasing order at every step and only a strictly better score
  replaces the incumbent, so the survivor is the optimal alignment whose
  reversed column sequence is lexicographically smallest -- the tie rule the
  build adopts (lowest move mask wins at every cell).
* ``needleman_wunsch`` is the textbook pairwise recurrence of Eq. 1 with the same
  tie preference (up, then left, then diagonal = masks 1, 2, 3).
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple


def column_score(chars: Sequence[Optional[str]], alphabet: str, subst, gap: int) -> int:
    idx = {c: i for i, c in enumerate(alphabet)}
    total = 0
    k = len(chars)
    for i in range(k):
        for j in range(i + 1, k):
            a, b = chars[i], chars[j]
            if a is None and b is None:
                continue
            if a is None or b is None:
                total += gap
            else:
                total += int(subst[idx[a]][idx[b]])
    return total


def rescore_rows(rows: Sequence[str], alphabet: str, subst, gap: int, gap_char: str = "-") -> int:
    ncols = len(rows[0]) if rows else 0
    total = 0
    for c in range(ncols):
        total += column_score([None if r[c] == gap_char else r[c] for r in rows], alphabet, subst, gap)
    return total


def brute_force(seqs: Sequence[str], alphabet: str, subst, gap: int) -> Tuple[int, List[int]]:
    """(best score, masks first-column-first) by exhaustive enumeration."""
    k = len(seqs)
    best = [None, None]
    path: List[int] = []

    def rec(x: List[int], acc: int) -> None:
        if all(v == 0 for v in x):
            if best[0] is None or acc > best[0]:
                best[0] = acc
                best[1] = list(path)
            return
        for m in range(1, 1 << k):
            if any(((m >> i) & 1) and x[i] == 0 for i in range(k)):
                continue
            chars = [seqs[i][x[i] - 1] if (m >> i) & 1 else None for i in range(k)]
            s = column_score(chars, alphabet, subst, gap)
            y = [x[i] - ((m >> i) & 1) for i in range(k)]
            path.append(m)
            rec(y, acc + s)
            path.pop()

    rec([len(s) for s in seqs], 0)
    return best[0], list(reversed(best[1]))


def count_paths(lens: Sequence[int]) -> int:
    """Number of alignments of sequences with these lengths (brute force size)."""
    from functools import lru_cache

    k = len(lens)

    @lru_cache(maxsize=None)
    def c(x: Tuple[int, ...]) -> int:
        if all(v == 0 for v in x):
            return 1
        tot = 0
        for m in range(1, 1 << k):
            if any(((m >> i) & 1) and x[i] == 0 for i in range(k)):
                continue
            tot += c(tuple(x[i] - ((m >> i) & 1) for i in range(k)))
        return tot

    return c(tuple(lens))


def needleman_wunsch(a: str, b: str, alphabet: str, subst, gap: int) -> Tuple[int, List[int]]:
    """Textbook global pairwise DP (Eq. 1) with linear gap; returns (score, masks)."""
    idx = {c: i for i, c in enumerate(alphabet)}
    n, m = len(a), len(b)
    F = [[0] * (m + 1) for _ in range(n + 1)]
    P = [[0] * (m + 1) for _ in range(n + 1)]
    for i in range(1, n + 1):
        F[i][0] = i * gap
        P[i][0] = 1
    for j in range(1, m + 1):
        F[0][j] = j * gap
        P[0][j] = 2
    for i in range(1, n + 1):
        for j in range(1, m + 1):
            up = F[i - 1][j] + gap
            left = F[i][j - 1] + gap
            diag = F[i - 1][j - 1] + int(subst[idx[a[i - 1]]][idx[b[j - 1]]])
            best = max(up, left, diag)
            F[i][j] = best
            P[i][j] = 1 if up == best else (2 if left == best else 3)
    masks = []
    i, j = n, m
    while i or j:
        mk = P[i][j]
        masks.append(mk)
        if mk & 1:
            i -= 1
        if mk & 2:
            j -= 1
    return F[n][m], list(reversed(masks))
