"""GB300 (sm_103a) FFT-based actions of block lower-triangular Toeplitz
operators: F, F* and the Gauss-Newton Hessian F* Gamma^-1 F.

The compute path is the C-ABI library libbtt.so (include/btt.h), built from
csrc/ with nvcc; this package only marshals arguments to it.  Tensors may
be torch CUDA tensors (used in place, on torch's current stream), torch CPU
tensors or numpy arrays (staged by the library).
"""
from ._lib import BttError, PRECISIONS, load, library_path
from .operator import Operator

__all__ = ["Operator", "BttError", "PRECISIONS", "load", "library_path"]
