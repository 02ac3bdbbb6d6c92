"""GB300-native solver for the finite-difference spherical Laplace equation
(coronal potential field, arXiv:1709.01126): Jacobi-preconditioned CG in
hand-written sm_103a CUDA kernels behind a C ABI (include/pot3d.h).

Importing the package does not load the CUDA library; ``pot3d.load()`` does,
and fails loudly if it has not been built."""

from . import _build  # noqa: F401

__all__ = ["pot3d", "serve", "_build"]
