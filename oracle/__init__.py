"""CPU oracle for LoLa's RNS-BFV hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of what the paper's method computes (BFV arithmetic, batch
encoding and the LoLa message representations / matrix-vector algorithms).
It exists so that the tests, the smoke check and the CPU-baseline leg of the
benchmark can check the CUDA path against it.  It shares no code with the
product: the only module both sides import is the seeded input generator
``workloads``, which holds none of the method's arithmetic.  The product
library never imports, links or runs anything in here.

Modules:
  _native   builds/loads the plain-C ring helper (c/oracle_ring.c)
  ring      Z_q[x]/(x^n+1) arithmetic, CRT lifting, automorphisms
  sampling  Philox4x64-10 streams; uniform, ternary, Gaussian samplers
  bfv       BFV keygen / encrypt / decrypt / add / mul_plain / mul_scalar /
            multiply / relinearize / rotate (definitions)
  encoding  slot <-> coefficient batch encoding
  lola      the paper's representations and matrix-vector algorithms,
            the slot simulator and the integer network
"""
