"""FP64 CPU oracle for the voxel-gravity forward model.

TEST INFRASTRUCTURE ONLY: the plain, slow reference that the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA library (``paper_1107_5951_gb300``) and never imports it.

Contents
--------
``direct``  -- ctypes wrapper of ``gf_oracle.c``: the discretised Eq. 1 sum
               (Sec. 2.1 quadrature, Eq. 7 N-body form), its transpose, the
               closed-form prism field (all three components), the SUM-AN
               sum over a voxel grid built from it and its transpose, the
               Appendix A norms, and the field of weighted point sources: the
               quadrature points of deformed hexahedral cells (general SUM-G1,
               Sec. 2.1) or scattered density points with their volumes
               (Sec. 4).
``tree``    -- numpy octree: Morton keys, box tables, near lists and
               interaction lists (Sec. 2.3 "Overview of the algorithm") and the
               surface-to-volume work model of Eqs. 14-19.
"""
