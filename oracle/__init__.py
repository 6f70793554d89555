"""Plain FP64 CPU oracle for the multipole-to-local (M2L) translation of the 3D Laplace kiFMM.

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run it. The product
path (the CUDA library and its Python binding) never imports it and shares no code with it:
no kernels, headers, helpers, tables or constant generators.

What it computes (arxiv 2408.07436):
  * geometry of the uniform octree, surfaces and interaction lists (Sec. 2, Sec. 2.1.1, Sec. 2.2)
  * the M2L map as the plain dense sum of Eq. 11 followed by the pseudo-inverse of Eqs. 7-10
  * the SVD-compressed variant of Sec. 3.1-3.2 (Eqs. 12-14)
  * the FFT convolution variant of App. A.1
  * a tiny complete FMM (P2M, M2M, M2L, L2L, L2P, P2P; Sec. 2) for end-to-end pins
  * the relative L2 error of Eq. 16

Everything is float64. Where the paper is silent the readings used are stated in
``geometry.py`` beside the code that takes them.
"""

from . import geometry, operators, m2l, fmm  # noqa: F401
