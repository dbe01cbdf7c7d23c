"""Oracle for the SEEDS hot path (arXiv 1309.3848): TEST INFRASTRUCTURE.

A plain, slow CPU implementation of what the GPU library computes, written
from the paper.  Only the test suite, the package smoke check and the
benchmark's CPU-baseline / reference leg may import this package; the GPU
library never does, and the two share no code.

Modules:
  seeds_ref.c  the parity schedule and the sequential mode, in plain C
  ref.py       ctypes access to the compiled oracle (numpy in / numpy out)
  energy.py    E(s) = H(s) + gamma*G(s) from its definitions, in fractions
  build.py     compiles seeds_ref.c with gcc
"""
