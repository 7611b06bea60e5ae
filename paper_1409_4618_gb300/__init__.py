"""GB300 (sm_103a) assembly of lowest-order Raviart-Thomas and Nedelec mass and
div/curl stiffness matrices into CSR (Anjam & Valdman, arXiv 1409.4618).

The compute path is libedgefem.so (CUDA, ``csrc/``) behind the C ABI of
``include/edgefem.h``; ``edgefem`` is its Python binding. ``meshgen`` makes
the seeded synthetic meshes. Importing this package loads nothing; the CUDA
library is loaded on first use of ``edgefem``.
"""
__all__ = ["edgefem", "meshgen", "build"]
