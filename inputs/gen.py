"""Seeded synthetic workloads for optimal DP multiple sequence alignment.

This module only draws random inputs (sequences, substitution tables, request
streams). It holds none of the alignment arithmetic, so both the CPU oracle and
the CUDA path can take their inputs from here without sharing any method code.

Workload recipe (the paper publishes no datasets; these stand in for the
workload sizes it describes, section 5):

* an ancestor of uniform residues is mutated independently per descendant:
  at each ancestor position an indel event happens with probability
  ``indel`` (half deletions, half insertions; length Geometric(p=0.5), mean 2,
  inserted residues uniform), otherwise the residue is substituted with
  probability ``sub`` by a uniformly drawn *different* residue, otherwise copied;
* each descendant is then cut or padded (uniform residues) to its exact target
  length, so the DP tensor has a fixed number of cells;
* DNA uses match +5 / mismatch -4 / gap -8; protein uses a symmetric 20x20 table
  with diagonal uniform in [4, 11] and off-diagonal uniform in [-4, 3], gap -6.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

DNA = "ACGT"
PROTEIN = "ARNDCQEGHILKMFPSTWYV"


@dataclasses.dataclass
class Problem:
    """One alignment problem: k sequences over ``alphabet`` with a linear gap."""

    name: str
    seqs: List[str]
    alphabet: str
    subst: np.ndarray  # int32, |alphabet| x |alphabet|, row-major
    gap: int
    seed: Optional[int] = None

    @property
    def k(self) -> int:
        return len(self.seqs)

    @property
    def lens(self) -> List[int]:
        return [len(s) for s in self.seqs]

    @property
    def cells(self) -> int:
        n = 1
        for s in self.seqs:
            n *= len(s) + 1
        return n

    def prefix(self, lens: List[int], name: Optional[str] = None) -> "Problem":
        """The same problem restricted to sequence prefixes of the given lengths."""
        return Problem(name or f"{self.name}[prefix {lens}]",
                       [s[:n] for s, n in zip(self.seqs, lens)],
                       self.alphabet, self.subst.copy(), self.gap, self.seed)


def dna_table(match: int = 5, mismatch: int = -4) -> np.ndarray:
    t = np.full((4, 4), mismatch, dtype=np.int32)
    np.fill_diagonal(t, match)
    return t


# The scoring behind the similarity scores of section 5.2: identical residues
# score +1, different residues 0, a residue facing a gap -1, two gaps 0.
PAPER_GAP = -1


def paper_table(size: int) -> np.ndarray:
    """Match +1 / mismatch 0 over an alphabet of ``size`` letters."""
    return np.eye(size, dtype=np.int32)


def paper_problem(seed: int, k: int, lens: List[int], alphabet: str = DNA, related: bool = True) -> Problem:
    """A seeded problem scored with the paper's +1/0/-1/0 scheme."""
    p = random_problem(seed, k, lens, alphabet=alphabet, table=paper_table(len(alphabet)), gap=PAPER_GAP,
                       related=related)
    return Problem(f"paper_s{seed}_k{k}_{'x'.join(map(str, lens))}", p.seqs, alphabet, p.subst, PAPER_GAP, seed)


def protein_table(rng: np.random.Generator, size: int = 20) -> np.ndarray:
    """Symmetric table: diagonal U[4,11], off-diagonal U[-4,3] (inclusive)."""
    t = np.zeros((size, size), dtype=np.int32)
    for i in range(size):
        t[i, i] = rng.integers(4, 12)
        for j in range(i + 1, size):
            v = rng.integers(-4, 4)
            t[i, j] = v
            t[j, i] = v
    return t


def random_seq(rng: np.random.Generator, alphabet: str, n: int) -> str:
    idx = rng.integers(0, len(alphabet), size=n)
    return "".join(alphabet[i] for i in idx)


def _geometric_len(rng: np.random.Generator) -> int:
    return int(rng.geometric(0.5))


def evolve(rng: np.random.Generator, ancestor: str, alphabet: str, sub: float,
           indel: float, target_len: int) -> str:
    """One descendant of ``ancestor`` (see the module docstring for the model)."""
    out: List[str] = []
    i = 0
    n = len(ancestor)
    while i < n:
        if rng.random() < indel:
            ln = _geometric_len(rng)
            if rng.random() < 0.5:  # deletion: skip ln ancestor residues
                i += ln
                continue
            out.extend(random_seq(rng, alphabet, ln))  # insertion before residue i
        c = ancestor[i]
        if rng.random() < sub:
            others = [a for a in alphabet if a != c]
            c = others[int(rng.integers(0, len(others)))]
        out.append(c)
        i += 1
    s = "".join(out)
    if len(s) >= target_len:
        return s[:target_len]
    return s + random_seq(rng, alphabet, target_len - len(s))


def related_family(rng: np.random.Generator, alphabet: str, lens: List[int],
                   sub: float, indel: float) -> List[str]:
    anc_len = int(round(sum(lens) / len(lens))) if lens else 0
    anc = random_seq(rng, alphabet, anc_len)
    return [evolve(rng, anc, alphabet, sub, indel, n) for n in lens]


# --------------------------------------------------------------------------
# The single-problem workloads and the serving stream.
# --------------------------------------------------------------------------

def pr1(seed: int = 1) -> Problem:
    """k=3 DNA, three iid uniform sequences of length 128 (129^3 tensor)."""
    rng = np.random.default_rng(seed)
    seqs = [random_seq(rng, DNA, 128) for _ in range(3)]
    return Problem("pr1_k3_dna_128", seqs, DNA, dna_table(), -8, seed)


def k3_protein(seed: int = 2) -> Problem:
    """k=3 protein, lengths 700/760/800 from one ancestor (sub 0.2, indel 0.05)."""
    rng = np.random.default_rng(seed)
    table = protein_table(rng)
    seqs = related_family(rng, PROTEIN, [700, 760, 800], 0.2, 0.05)
    return Problem("k3_protein_700_760_800", seqs, PROTEIN, table, -6, seed)


def k4_dna(seed: int = 3) -> Problem:
    """k=4 DNA, lengths 110/118/124/130 from one ancestor (sub 0.15, indel 0.05)."""
    rng = np.random.default_rng(seed)
    seqs = related_family(rng, DNA, [110, 118, 124, 130], 0.15, 0.05)
    return Problem("k4_dna_110_118_124_130", seqs, DNA, dna_table(), -8, seed)


def k6_protein(seed: int = 4, table_seed: int = 2) -> Problem:
    """k=6 protein, six lengths uniform in 18..24 (sub 0.25, indel 0.05).

    Uses the same substitution table as :func:`k3_protein` (drawn from seed 2).
    """
    table = protein_table(np.random.default_rng(table_seed))
    rng = np.random.default_rng(seed)
    lens = [int(x) for x in rng.integers(18, 25, size=6)]
    seqs = related_family(rng, PROTEIN, lens, 0.25, 0.05)
    return Problem("k6_protein_18_24", seqs, PROTEIN, table, -6, seed)


def k4_dna_profile(seed: int = 3) -> Problem:
    """k=4 DNA at a size for full counter captures (lengths 70/70/70/100, 36M cells;
    the fill's faces and traceback bytes still exceed the L2), same recipe as k4_dna."""
    rng = np.random.default_rng(seed)
    seqs = related_family(rng, DNA, [70, 70, 70, 100], 0.15, 0.05)
    return Problem("k4_dna_profile_70_70_70_100", seqs, DNA, dna_table(), -8, seed)


def k6_protein_profile(seed: int = 4, table_seed: int = 2) -> Problem:
    """k=6 protein at a size for full counter captures (six lengths of 17, 34M cells),
    same recipe and table as k6_protein."""
    table = protein_table(np.random.default_rng(table_seed))
    rng = np.random.default_rng(seed)
    seqs = related_family(rng, PROTEIN, [17] * 6, 0.25, 0.05)
    return Problem("k6_protein_profile_17", seqs, PROTEIN, table, -6, seed)


def k2_protein(seed: int = 6, table_seed: int = 2) -> Problem:
    """k=2 protein pair, lengths 5000/4800 from one ancestor (sub 0.2, indel 0.05).

    The pairwise case of the method (section 2, Eq. 1), at 2.4e7 cells.
    Uses the substitution table of :func:`k3_protein`.
    """
    table = protein_table(np.random.default_rng(table_seed))
    rng = np.random.default_rng(seed)
    seqs = related_family(rng, PROTEIN, [5000, 4800], 0.2, 0.05)
    return Problem("k2_protein_5000_4800", seqs, PROTEIN, table, -6, seed)


WORKLOADS = {
    "pr1": pr1,
    "k2_protein": k2_protein,
    "k3_protein": k3_protein,
    "k4_dna": k4_dna,
    "k6_protein": k6_protein,
    # smaller cases of the same recipes, for full counter captures
    "k4_dna_profile": k4_dna_profile,
    "k6_protein_profile": k6_protein_profile,
}

SERVING_LEN_RANGE = {2: (200, 2000), 3: (40, 300), 4: (20, 80)}


def serving_request(i: int, base_seed: int = 5) -> Problem:
    """Request ``i`` of the serving stream (seed 5*10^6 + i)."""
    rng = np.random.default_rng(base_seed * 10**6 + i)
    k = int(rng.choice([2, 3, 4], p=[0.5, 0.35, 0.15]))
    lo, hi = SERVING_LEN_RANGE[k]
    lens = [int(x) for x in rng.integers(lo, hi + 1, size=k)]
    if rng.random() < 0.5:
        seqs = related_family(rng, DNA, lens, 0.15, 0.05)
        return Problem(f"req{i}_k{k}_dna", seqs, DNA, dna_table(), -8, i)
    table = protein_table(rng)
    seqs = related_family(rng, PROTEIN, lens, 0.2, 0.05)
    return Problem(f"req{i}_k{k}_protein", seqs, PROTEIN, table, -6, i)


def serving_arrivals(n: int, rate: float, seed: int = 5) -> np.ndarray:
    """Poisson arrival times (seconds) for ``n`` requests at ``rate`` per second."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def random_problem(seed: int, k: int, lens: List[int], alphabet: str = DNA,
                   table: Optional[np.ndarray] = None, gap: Optional[int] = None,
                   related: bool = False) -> Problem:
    """Small seeded problem for parity tests (iid or related sequences)."""
    rng = np.random.default_rng(seed)
    if table is None:
        table = dna_table() if alphabet == DNA else protein_table(rng, len(alphabet))
    if gap is None:
        gap = -8 if alphabet == DNA else -6
    if related:
        seqs = related_family(rng, alphabet, lens, 0.2, 0.05)
    else:
        seqs = [random_seq(rng, alphabet, n) for n in lens]
    return Problem(f"rand_s{seed}_k{k}_{'x'.join(map(str, lens))}", seqs, alphabet,
                   np.asarray(table, dtype=np.int32), int(gap), seed)
