"""CPU oracle for the PDQ hot path (Mask -> Comp) and Decomp.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
reference that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
it; the library (``paper_2408_17063_gb300``) never does, and the two share no
code (the only shared module is ``workloads``, which draws random inputs and
holds none of the method's arithmetic).

* ``ref_ring.c`` — modular arithmetic with 128-bit division, the textbook
  negacyclic transform, schoolbook product, automorphisms, basis conversion.
* ``bfv``       — parameters, slot encoding, BFV encryption/decryption (big
  integers), hybrid key switching, rotations (Sec. 5.1).
* ``pdq``       — Mask, Comp (Alg. 7 in the SIMD form of Sec. 5.2), the
  plaintext closed form C v / C d (Eq. 1) and Decomp (Alg. 1, 4, 6).
* ``mutants``   — planted mistakes in the modules above, each of which the
  pins must catch (``python -m oracle.mutants``).

Every function is pinned by ``tests/test_oracle_*.py`` against definitions,
brute force and invariants that do not reuse the oracle's own code path.
"""
from . import bfv, pdq, ring  # noqa: F401
