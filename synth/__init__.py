"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package draws random numbers and lays them out; it holds none of the
arithmetic of the CI method itself (no Slater–Condon rule, no sigma, no
eigen-solve, no increment algebra).
"""
from .chain import (  # noqa: F401
    ChainSystem,
    make_chain,
    chain_4x2,
    chain_24_uneven,
    chain_7x2,
    chain_40_uneven,
    pair_index,
    random_ci_vector,
)
