"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module draws numbers and nothing else: it holds none of the
arithmetic of the block-Toeplitz method.  One counter-based generator
(Philox4x32-10 + Box-Muller, ``philox.h``) exists in three builds:

* ``philox.py``   -- NumPy, the readable reference;
* ``synth_host.c`` -- C/OpenMP, fast host fills (compiled with gcc);
* ``synth_dev.cu`` -- CUDA, fills device memory directly for large inputs.

Tensor ids: 0 blocks F_k, 1 parameter vectors m, 2 data vectors d,
3 noise variances, 4 data-side envelope, 5 arrival trace, 6 parameter-side
envelope, 7 probe directions, 8 weights.
"""
from .workloads import (Workload, WORKLOADS, SERVING_OPERATORS, envelope, blocks,
                        block_entries, vectors, noise_gamma_inv, uniforms, normals,
                        host_lib, dev_lib, build)

__all__ = ["Workload", "WORKLOADS", "SERVING_OPERATORS", "envelope", "blocks",
           "block_entries", "vectors", "noise_gamma_inv", "uniforms", "normals",
           "host_lib", "dev_lib", "build"]
