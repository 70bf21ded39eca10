"""Plain FP64 CPU oracle of HIF-DE (Ho & Ying, arXiv:1307.2895).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The product path (the CUDA library and its Python
binding) never imports it, and it imports nothing from the product path: it
shares no code, tables or helpers with the CUDA implementation.

Modules:

* :mod:`oracle.stencil`  -- five/seven-point variable-coefficient stencil
  (Section 3.1 and 3.2).
* :mod:`oracle.hifde`    -- MF (Algorithm 3.1) and HIF-DE (Algorithm 4.1, 2D and
  3D with face skeletonization), the apply of F and F^-1 (Eq. 3.1 / 4.2),
  PCG and the power-method error estimates of Section 5.

Parity status per function is stated in each module header.
"""
