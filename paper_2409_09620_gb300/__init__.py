"""GB300-native BP RI-OEDG solver (2D Euler, P1/P2 modal DG on triangles).

Method: Ding, Cui & Wu, arXiv 2409.09620.  The solver is a CUDA library with a
C ABI (``include/dg.h``); ``native`` is its Python binding and ``workloads``
holds seeded synthetic inputs.  Importing the package loads nothing; the CUDA
library is loaded on first use of ``native``.
"""

__all__ = ["native", "workloads", "build"]
