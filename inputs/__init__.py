"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench."""
from .gen import (DNA, PAPER_GAP, PROTEIN, Problem, WORKLOADS, dna_table, k2_protein, k3_protein, k4_dna,
                  k6_protein, paper_problem, paper_table, pr1, protein_table, random_problem,
                  random_seq, serving_arrivals, serving_request)

__all__ = ["DNA", "PAPER_GAP", "PROTEIN", "Problem", "WORKLOADS", "dna_table", "k2_protein", "k3_protein", "k4_dna",
           "k6_protein", "paper_problem", "paper_table", "pr1", "protein_table", "random_problem",
           "random_seq", "serving_arrivals", "serving_request"]
