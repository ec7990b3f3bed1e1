"""GB300-native (sm_103a) separable isotropic NPCF estimator (arXiv:2106.10278).

The compute path is the C-ABI library ``libnpcf.so`` built from ``csrc/``;
``paper_2106_10278_gb300.npcf`` is its thin ctypes binding.  Submodules are
imported explicitly (``from paper_2106_10278_gb300 import npcf``) so that
``catalogs`` works on machines without the built library.
"""
