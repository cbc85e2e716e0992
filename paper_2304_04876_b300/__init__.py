"""GDSW two-level overlapping Schwarz preconditioned Krylov solver for B300 (sm_103a).

The compute path lives in the C-ABI library ``libgdsw.so`` (hand-written CUDA);
``paper_2304_04876_b300.gdsw`` is its thin Python binding and
``paper_2304_04876_b300.problems`` builds seeded synthetic inputs.  Importing
the package loads nothing native; the binding loads the library on first use.
"""
