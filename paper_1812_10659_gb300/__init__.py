"""GB300 (sm_103a) implementation of LoLa's data-parallel hot path.

RNS-BFV ciphertext arithmetic (negacyclic NTT per prime, ct x pt, ct x ct
with exact scaling, relinearisation, Galois rotations with key switching)
and the LoLa message representations / matrix-vector algorithms built on
it, behind the C-ABI in include/lola.h.  ``paper_1812_10659_gb300.lola`` is
the Python binding; ``paper_1812_10659_gb300.build`` compiles the library.
Importing this package does not load CUDA.
"""
__all__ = ["lola", "build"]
