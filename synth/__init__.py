"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This package draws random numbers and assembles test Hamiltonians with a known
spectrum. It holds none of the purification or Ozaki arithmetic, so both the
oracle and the CUDA path can take their inputs from it without sharing method
code.
"""

from .hamiltonians import (  # noqa: F401
    CONFIGS,
    Hamiltonian,
    batch_sizes,
    config_hamiltonian,
    make_hamiltonian,
    random_orthogonal,
    spectrum,
    symmetric_gaussian,
)
