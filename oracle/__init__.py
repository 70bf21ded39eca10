"""Plain FP64 CPU oracle of HIF-DE (Ho & Ying, arXiv:1307.2895).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The product path (the CUDA library and its Python
binding) never imports it, and it imports nothing from the product path: it
shares no code, tables or helpers with the CUDA implementation.

Modules:

* :mod:`oracle.stencil`  -- five/seven-point variable-coefficient stencil
  (Section 3.1 and 3.2), and a central-difference convection term for the
  unsymmetric operators of Section 6.
* :mod:`oracle.hifde`    -- MF (Algorithm 3.1) and HIF-DE (Algorithm 4.1, 2D and
  3D with face skeletonization; Algorithm 4.2, hifde3x), the apply of F and
  F^-1 (Eq. 3.1 / 4.2), the SVD skeletonization (Section 4.4), the two-sided
  unsymmetric variant (Section 6), PCG, GMRES and the power-method error
  estimates of Section 5.
* :mod:`oracle.learned`  -- the randomized ID of Section 4.3 and the rank MLP.

Parity status per function is stated in each module header.
"""
