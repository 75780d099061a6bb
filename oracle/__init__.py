"""FP64 CPU oracle for the block lower-triangular Toeplitz operator.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, link or
run this package: it exists so that tests, the smoke check and the timed CPU
baseline of the benchmark have an independent, obviously correct answer.
It shares no code with the CUDA library (``paper_2407_13066_gb300``) and
imports nothing from it.

Contents
  direct.py      the plain definition (Eq. ShiftInvariance / Eq. p2o):
                 d_i = sum_{j<=i} F_{i-j} m_j, its transpose (the adjoint,
                 Sec. 2.2 footnote on F*), the Gauss-Newton Hessian
                 F* Gamma^-1 F, and sampled entries of each for operators too
                 large to apply whole.
  naive.c        the same definition as literal loops in plain C (second,
                 independent oracle for small sizes).
  fft_method.py  the paper's algorithm (Alg. 1 setup, Alg. 2 F matvec,
                 Alg. 3 F* matvec, Sec. 2.4 circulant embedding) in FP64 with
                 numpy's FFT as a library step; pinned to direct.py, it fixes
                 the readings of the FFT normalisation, the number of
                 frequency slices and the padding side.
  cg.py          conjugate gradients (Hestenes-Stiefel) on the regularised
                 Gauss-Newton Hessian, the solve the Hessian action serves.
  quantize.py    rounding of F-hat to the reduced storage precisions
                 (FP16 with a per-frequency scale, BF16, a BF16 hi+lo pair),
                 as plain numpy element maps.

Every function here is pinned by the CPU tests (tests/test_oracle_*.py)
against closed forms, a dense assembled matrix, a textbook convolution and
invariants -- not against itself.
"""
