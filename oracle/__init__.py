"""CPU FP64 oracle for the QTT linear-elasticity solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link or execute
anything in this package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA path (``paper_2501_12151_gb300``)
except the seeded input descriptions in ``paper_2501_12151_gb300.workloads``, which hold none of
the method's arithmetic.

Two halves:

* ``oracle.fem``  -- oracle A: plain element-loop Q1 (2D) / trilinear (3D) assembly of the
  Galerkin system A u = f (Section 3, Eq. finbilform / femsys / elassembly / grads) in sparse
  form, with the load f = M f0 of Section 5.3, solved by a sparse direct solver or CG.
* ``oracle.tt`` and ``oracle.amen`` -- oracle B: a plain CPU tensor-train toolkit (TT-SVD,
  rounding, TT-matrix times TT, QTT index maps of Section 4) and the AMEn sweep named in
  Section 5.4 / Algorithm 2.
"""
