"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench."""
from .gen import (DNA, PROTEIN, Problem, WORKLOADS, dna_table, k3_protein, k4_dna,
                  k6_protein, pr1, protein_table, random_problem, random_seq,
                  serving_arrivals, serving_request)

__all__ = ["DNA", "PROTEIN", "Problem", "WORKLOADS", "dna_table", "k3_protein", "k4_dna",
           "k6_protein", "pr1", "protein_table", "random_problem", "random_seq",
           "serving_arrivals", "serving_request"]
