"""CPU oracle for the RNS-CKKS encrypted-query path.

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call or load anything in this
package. The GPU library in ``paper_2412_13269_gb300`` neither imports nor
links it, and the two share no code: they meet only in the seeded draws of
``synth`` (which holds none of the scheme's arithmetic).

Layout
  ckks_oracle.c  plain C core (Barrett mulmod, textbook NTT used as a library
                 primitive for negacyclic products, base conversion, rescale,
                 ModDown, hybrid SwitchKey, automorphism), coefficient domain
  rns.py         ctypes bindings, prime/root selection, CRT
  ckks.py        encoding, keys, encryption, homomorphic operations
  query.py       the circuit's plan, its plain execution, the FP64 pipeline

Every function cites the passage of the paper (arXiv 2412.13269) it follows.
Parity status: every function is pinned by a test in tests/test_oracle_*.py
against something other than itself (brute-force definitions on tiny rings,
big-integer CRT, decryption identities, closed forms).
"""
