"""ORACLE — test infrastructure only.

Plain, slow, FP64 CPU implementations of what the GPU tensor-train path
computes, written from arXiv 2309.03347 and used only by ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg.  It shares no
code with the CUDA library and never imports the product package.

* ``oracle.transport`` — full-grid vertex diamond-difference operators
  H, S, F and the power iteration of Eq. (k_eff_fixed_points), in plain C
  (``sweep.c``) driven through ctypes.
* ``oracle.ttref`` — dense-reconstruct tensor-train reference (TT-SVD,
  TT rounding, TT-matrix/vector products, QTT of matrices per Algorithm 1).
* ``oracle.operators`` — the operators assembled as sums of Kronecker products
  of the one-dimensional factors of Sec. 3.2 (sparse, for tiny grids), and the
  generalized eigensolve (GES) used as a cross-check.
"""
