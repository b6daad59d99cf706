"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This package holds no arithmetic of the method: it only draws data matrices,
labels and the random numbers a sketch consumes (hash buckets, signs, sampled
rows), and converts storage formats (fp32 <-> bf16 bit patterns).  Both the
CPU oracle and the GPU path receive the same arrays from here.
"""
from .inputs import (  # noqa: F401
    bf16_bits_to_f32,
    f32_to_bf16_bits,
    cca_latent_problem,
    lda_problem,
    countsketch_draws,
    srht_draws,
    random_tall,
    latent_scales,
    make_workload,
    CONFIGS,
)
