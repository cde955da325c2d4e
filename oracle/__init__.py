"""CPU oracle for the fast directional matrix-vector product (Of & Watschinger).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import, call or link anything in this folder.
The library (paper_2004_14229_gb300) never does: it has no CPU fallback.

Two oracles, both plain FP64 and independent of the CUDA path:

* O_direct (oracle/direct.c, oracle/direct.py): the exact product of Eq. (1).
* O_fdm (oracle/fdm.py): the paper's method itself, Alg. 1 - Alg. 4 with the
  matrices of Eqs. (8)-(10) and (13), written out in the paper's order; its
  mode "aca" compresses the coupling matrices by the partially pivoted ACA of
  Sect. 2.7's closing remark (oracle/aca.py).
"""
