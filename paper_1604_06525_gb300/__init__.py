"""GB300-native GN / LM PCG solver library for sum-of-squares energies
(matrix-free stencil and graph passes, materialized CSR variant).

The compute path is the CUDA shared library built from ``csrc/``; the Python
modules only marshal arguments to its C ABI.  Importing this package does not
load the library; ``paper_1604_06525_gb300.api`` does, and fails loudly when it
is missing.
"""
__all__ = ["synth", "api"]
