"""CPU oracle for RNS-CKKS multi-input ciphertext multiplication.

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import this package. The product library
(`paper_2601_15401_gb300`) never imports it, and this package imports nothing
from the product library: the two share no code, headers, tables or constant
generators. Both take their random inputs from `synth`.

Layout
  prims.c  exact modular primitives (unsigned __int128 products, `%`), the
           O(N^2) NTT definition, the schoolbook negacyclic product and the
           textbook radix-2 transform (pinned to the definition by the tests)
  ring.py  ctypes binding of prims.c, the choice of psi, helpers
  ckks.py  the paper's method, step by step: tensor product (Eq. 13),
           rescaling (Eq. 6, Eq. 7, Algorithm 1 with Eq. 16/17), basis
           conversion (Eq. 4), ModUp/ModDown (Eq. 5), relinearisation with
           extra keys (Eq. 2, 9, 14, 15), tree evaluation (Section V-C),
           key generation, encode/encrypt/decrypt/decode (Section II)
  plan.py  input partitions: parsing, the depth rule, rescale-unit counts,
           exhaustive search (Section V-C, Table II)
"""
