"""Oracle: a plain, slow CPU implementation of the paper's RNS-CKKS hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference``) may import
this package.  The product library under ``paper_2305_17341_gb300`` never
imports, links or executes anything here, and this package never imports the
product library: the two share no code.

Layout
  oracle.c     integer / FP64 primitives written out from their definitions
  _c.py        ctypes bindings of oracle.c (builds liboracle.so on first use)
  ckks.py      the RNS-CKKS scheme of App. A in coefficient form
  hmm.py       linear transforms (eq. 2, eq. 3'), double hoisting (Sec. 3.3),
               JKLS matrix multiplication (eq. 4, Sec. 4.1, Table 1)
  pca.py       Aggregate, covariance (HCovMtrx), Lazy Normalization, PowerMethod

Parity status: every function is pinned by tests/ against closed forms,
brute force or the paper's printed values; the encode rounding on
near-half-integers is pinned only by the direct O(N^2) sum on small N.
"""
