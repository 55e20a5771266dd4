"""CPU oracle for norm-ranging LSH (Yan et al., NeurIPS 2018).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 NumPy restatement
of the method, written from the paper: Algorithm 1 (index building), Eq. 8
(SIMPLE-LSH transform), Eq. 4 (sign random projection), Eq. 12 and the sorted
(U_j, l) structure of Section 3.3 (multi-probe bucket ranking), then an exact
re-rank and top-k (Eq. 1).  It shares no code with the CUDA library and the
library never imports it.  Only the tests, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU baseline may use it.

Modules:
  philox       counter-based generator for the projection matrix A
  nrlsh        index build, query probing, re-rank and top-k
  multitable   Algorithm 2 with T hash tables and one probe per table
  simple_lsh   SIMPLE-LSH with one global U (Eq. 8), written separately
  exact        exact MIPS by rational arithmetic (Eq. 1) and recall@k
"""
