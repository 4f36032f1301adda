"""CPU FP64 oracle for the DD-DLRA time step (arXiv 2602.14854).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import or run anything in this
package.  The product path (the CUDA library and its Python binding) never
imports it, and the two share no code: the only module both sides read is the
seeded problem-data generator ``paper_2602_14854_gb300.inputs``.

Contents
  sn.py      full-rank discrete-ordinates (S_N) solver of the same split
             discretisation (Section 3 splitting, first-order upwind, Section 4).
  dd_dlra.py the domain-decomposition dynamical low-rank step, Algorithm 6 with
             Algorithms 1-5 and the upwind rule of Appendix A, written in the
             paper's weighted inner products.

Pin status of every function is listed in the header of each module.
"""
