"""The paper's FFT-based algorithm, FP64, with numpy's FFT as a library step.

TEST INFRASTRUCTURE ONLY.  Follows the steps of Alg. 1 (setup), Alg. 2
(F matvec) and Alg. 3 (F* matvec) on one GPU (no partitioning, so the
broadcast/reduction steps are identities), using the circulant embedding of
Sec. 2.4 (Eq. CirculantMatrix, Eq. FFTMatrixVectorProduct):

  setup     pad each first-column time series F_k[s][l], k < N_t, with N_t
            zeros at the end, take the real DFT of length 2 N_t along k,
            keep the N_t + 1 non-negative frequencies:  Fhat[w][s][l].
  F         mhat = rfft(pad(m)) along time; dhat[w] = Fhat[w] @ mhat[w];
            d = irfft(dhat)[:N_t]            (Alg. 2)
  F*        dhat = rfft(pad(d)); mhat[w] = Fhat[w]^H @ dhat[w];
            m = irfft(mhat)[:N_t]            (Alg. 3, Eq. AdjointFFTMatvec)

Readings (where the paper is loose): the forward DFT is unnormalised with
kernel exp(-2 pi i w t / 2N_t); the inverse carries 1/(2N_t) and nothing
else (Eq. FFTMatrixVectorProduct's 1/sqrt(2n) is not applied on top);
padding is at the end; frequency slices are w = 0..N_t (N_t + 1 of them,
the count of Table ComputationalCost).  tests/test_oracle_pins.py checks
that these readings reproduce the direct definition in direct.py.
"""
import numpy as np


def setup(F):
    """Fhat[w][s][l] (complex128), w = 0..N_t, from blocks F [N_t][N_d][N_m]."""
    F = np.asarray(F, dtype=np.float64)
    N_t = F.shape[0]
    return np.fft.rfft(F, n=2 * N_t, axis=0)


def transform(x):
    """xhat[..., w, :] = sum_{t<N_t} x[..., t, :] exp(-2 pi i w t / 2N_t)."""
    x = np.asarray(x, dtype=np.float64)
    N_t = x.shape[-2]
    return np.fft.rfft(x, n=2 * N_t, axis=-2)


def inverse_transform(xhat, N_t):
    """First N_t samples of the length-2N_t inverse real DFT (1/(2N_t))."""
    return np.fft.irfft(xhat, n=2 * N_t, axis=-2)[..., :N_t, :]


def apply_fhat(Fhat, xhat):
    """dhat[..., w, s] = sum_l Fhat[w, s, l] xhat[..., w, l]."""
    return np.einsum("wsl,...wl->...ws", Fhat, xhat)


def apply_fhat_adjoint(Fhat, yhat):
    """mhat[..., w, l] = sum_s conj(Fhat[w, s, l]) yhat[..., w, s]."""
    return np.einsum("wsl,...ws->...wl", np.conj(Fhat), yhat)


def forward(Fhat, m):
    N_t = np.asarray(m).shape[-2]
    return inverse_transform(apply_fhat(Fhat, transform(m)), N_t)


def adjoint(Fhat, d):
    N_t = np.asarray(d).shape[-2]
    return inverse_transform(apply_fhat_adjoint(Fhat, transform(d)), N_t)


def hessian(Fhat, m, gamma_inv=None):
    d = forward(Fhat, m)
    if gamma_inv is not None:
        d = d * gamma_inv
    return adjoint(Fhat, d)
