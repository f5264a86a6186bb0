"""GB300-native auxiliary-space preconditioned conjugate gradients for P_k Lagrange
discretisations of -div(kappa grad u) = f on tetrahedral meshes (Lee, Leng & Zhang,
"A Scalable Auxiliary Space Preconditioner for High-Order Finite Element Methods").

The compute path is libpkasp.so (hand-written CUDA for sm_103a behind the C ABI of
include/pkasp.h); this package marshals arguments and uses PyTorch for device buffers
and streams only.
"""
from . import _lib
from ._lib import PkaspError, default_options, load
from .solver import Problem, dofmap_host, nodes_host, pmis, reference_tensors

__all__ = ["Problem", "PkaspError", "default_options", "load", "pmis", "dofmap_host", "nodes_host",
           "reference_tensors", "_lib"]
