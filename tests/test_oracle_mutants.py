"""Plausible mistakes planted in copies of the oracle, on the CPU, must each
fail at least one pin of test_oracle_pins.py."""
import numpy as np
import pytest

from oracle import direct
from tests.test_oracle_pins import _golden, dense_matrix

RNG = np.random.default_rng(7)


def _fwd_dropped_last_lag(F, m):
    N_t = m.shape[-2]
    d = np.zeros(m.shape[:-1] + (F.shape[1],))
    for k in range(N_t - 1):
        d[k:] += m[: N_t - k] @ F[k].T
    return d


def _fwd_lag_off_by_one(F, m):
    N_t = m.shape[-2]
    d = np.zeros(m.shape[:-1] + (F.shape[1],))
    for k in range(N_t):
        d[k:] += m[: N_t - k] @ F[min(k + 1, N_t - 1)].T
    return d


def _fwd_upper_triangular(F, m):
    N_t = m.shape[-2]
    d = np.zeros(m.shape[:-1] + (F.shape[1],))
    for k in range(N_t):
        d[: N_t - k] += m[k:] @ F[k].T
    return d


def _adj_wrong_direction(F, d):
    N_t = d.shape[-2]
    m = np.zeros(d.shape[:-1] + (F.shape[2],))
    for k in range(N_t):
        m[k:] += d[: N_t - k] @ F[k]
    return m


def _adj_sign(F, d):
    return -direct.adjoint(F, d)


def _fft_forward_unitary_scaling(F, m):
    N_t = m.shape[-2]
    Fh = np.fft.rfft(F, n=2 * N_t, axis=0)
    mh = np.fft.rfft(m, n=2 * N_t, axis=0)
    dh = np.einsum("wsl,wl->ws", Fh, mh) / np.sqrt(2 * N_t)
    return np.fft.irfft(dh, n=2 * N_t, axis=0)[:N_t]


def _fft_forward_no_padding(F, m):
    N_t = m.shape[-2]
    Fh = np.fft.rfft(F, axis=0)
    mh = np.fft.rfft(m, axis=0)
    return np.fft.irfft(np.einsum("wsl,wl->ws", Fh, mh), n=N_t, axis=0)


def _fft_adjoint_without_conj(F, d):
    N_t = d.shape[-2]
    Fh = np.fft.rfft(F, n=2 * N_t, axis=0)
    dh = np.fft.rfft(d, n=2 * N_t, axis=0)
    return np.fft.irfft(np.einsum("wsl,ws->wl", Fh, dh), n=2 * N_t, axis=0)[:N_t]


def _fft_keep_last_block(F, m):
    N_t = m.shape[-2]
    Fh = np.fft.rfft(F, n=2 * N_t, axis=0)
    mh = np.fft.rfft(m, n=2 * N_t, axis=0)
    return np.fft.irfft(np.einsum("wsl,wl->ws", Fh, mh), n=2 * N_t, axis=0)[N_t:]


def _pins_pass(fwd, adj):
    """True if every pin holds for this (forward, adjoint) pair."""
    ok = True
    g = _golden()
    A = g["A"]
    F = A["f"].reshape(4, 1, 1)
    ok &= np.allclose(fwd(F, A["x"].reshape(4, 1)).ravel(), A["Fx"])
    ok &= np.allclose(adj(F, A["y"].reshape(4, 1)).ravel(), A["FTy"])
    for shape in [(5, 3, 4), (7, 2, 9)]:
        F = RNG.standard_normal(shape)
        m = RNG.standard_normal((shape[0], shape[2]))
        d = RNG.standard_normal((shape[0], shape[1]))
        D = dense_matrix(F)
        ok &= np.allclose(fwd(F, m).ravel(), D @ m.ravel())
        ok &= np.allclose(adj(F, d).ravel(), D.T @ d.ravel())
        ok &= np.isclose(np.vdot(fwd(F, m), d), np.vdot(m, adj(F, d)))
    return bool(ok)


def test_unmutated_oracle_passes():
    assert _pins_pass(direct.forward, direct.adjoint)


@pytest.mark.parametrize("fwd,adj", [
    (_fwd_dropped_last_lag, direct.adjoint),
    (_fwd_lag_off_by_one, direct.adjoint),
    (_fwd_upper_triangular, direct.adjoint),
    (direct.forward, _adj_wrong_direction),
    (direct.forward, _adj_sign),
    (_fft_forward_unitary_scaling, direct.adjoint),
    (_fft_forward_no_padding, direct.adjoint),
    (direct.forward, _fft_adjoint_without_conj),
    (_fft_keep_last_block, direct.adjoint),
])
def test_planted_mistake_is_caught(fwd, adj):
    assert not _pins_pass(fwd, adj)
