"""GB300 implementation of the hierarchical interpolative factorization for
elliptic differential operators (HIF-DE; Ho & Ying, arXiv:1307.2895).

* :mod:`paper_1307_2895_gb300.hif`    -- binding of the C ABI (``include/hif.h``)
* :mod:`paper_1307_2895_gb300.build`  -- builds ``_lib/libhif.so`` for sm_103a
* :mod:`paper_1307_2895_gb300.inputs` -- seeded synthetic workloads

Importing the package loads nothing; the CUDA library is loaded on first use
of :mod:`paper_1307_2895_gb300.hif`.
"""
