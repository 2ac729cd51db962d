"""GB300-native Chebyshev-filtered subspace iteration for SPARC's real-space Kohn-Sham
Hamiltonian of isolated clusters (arXiv:1603.04334).

The compute path is the C-ABI library libsparc_gb300.so (hand-written sm_103a CUDA);
`paper_1603_04334_gb300.sparc` is a thin ctypes binding with the same call names.
Importing this package does not load the library; `sparc.load()` does, and raises if it
is missing.
"""
__all__ = ["sparc", "synth"]
