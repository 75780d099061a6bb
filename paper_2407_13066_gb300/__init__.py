"""GB300 (sm_103a) FFT-based actions of block lower-triangular Toeplitz
operators: F, F* and the Gauss-Newton Hessian F* Gamma^-1 F.

The compute path is the C-ABI library libbtt.so (include/btt.h), built from
csrc/ with nvcc; this package only marshals arguments to it.  Tensors may
be torch CUDA tensors (used in place, on torch's current stream), torch CPU
tensors or numpy arrays (staged by the library).
"""
from ._lib import BttError, FAULTS, PRECISIONS, check, load, library_path
from .operator import Operator


def inject_fault(kind, count=1):
    """Host-side fault injection: the next `count` device allocations
    (kind 'alloc') or actions ('launch') fail; 'none' clears."""
    check(load().btt_inject_fault(FAULTS[kind], int(count)))


__all__ = ["Operator", "BttError", "PRECISIONS", "FAULTS", "inject_fault", "load", "library_path"]
