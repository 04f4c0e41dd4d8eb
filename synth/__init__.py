"""Seeded synthetic workloads and scoring tables.

This package is the only code shared by the CPU oracle (``oracle/``) and the
CUDA path (``paper_2205_07610_gb300``): it produces inputs (residue codes in
CSR form, substitution matrices) and contains none of the alignment
arithmetic.  Every generator takes an explicit seed and uses numpy's PCG64
(portable across x86-64 and aarch64), so the oracle and the GPU see
byte-identical inputs.
"""
from .tables import (DNA_ALPHABET, PROTEIN_ALPHABET, BLOSUM62, PROTEIN_BACKGROUND,
                     dna_matrix, blosum62, encode)
from .workloads import (SEED_BASE, Batch, CrossBatch, Stream, pack_csr, uniform_dna_pairs,
                        mutated_dna_pairs, protein_database, long_dna_pairs, serving_stream,
                        random_sequences, mutate)
from .band import NPARAMS as MLP_NPARAMS, mlp_init, minibatches

__all__ = [
    "DNA_ALPHABET", "PROTEIN_ALPHABET", "BLOSUM62", "PROTEIN_BACKGROUND", "dna_matrix",
    "blosum62", "encode", "SEED_BASE", "Batch", "CrossBatch", "Stream", "pack_csr",
    "uniform_dna_pairs", "mutated_dna_pairs", "protein_database", "long_dna_pairs",
    "serving_stream", "random_sequences", "mutate", "MLP_NPARAMS", "mlp_init", "minibatches",
]
