"""The plain definition of the block lower-triangular Toeplitz operator.

Eq. ShiftInvariance and Eq. p2o (Sec. 2.1): the data block i is

    d_i = sum_{j=0}^{i} F_{i-j} m_j ,   i = 0 .. N_t-1,

with F_k (N_d x N_m) the first block column (0-based on both sides, F_0 on
the diagonal).  The adjoint (Sec. 2.2, footnote on F*: block upper
triangular; real data, so * is the transpose) is

    m_j = sum_{i=j}^{N_t-1} F_{i-j}^T d_i .

The Gauss-Newton Hessian of the misfit weighted by a diagonal noise
precision Gamma^-1 (one entry per data value) is H m = F* (Gamma^-1 (F m)),
Eq. LinearInverseProblem with the data misfit weighted by Gamma^-1.

Everything is float64.  Vectors are time-outer: m[..., t, l] and d[..., t, s];
leading dimensions are independent right-hand sides.

A block source is either a float64 array [N_t][N_d][N_m] or a callable
``block(k) -> [N_d][N_m]`` (for operators too large to hold whole).
A library matmul serves as the inner step: for each lag k, all pairs (i, j)
with i - j = k are summed at once.
"""
import numpy as np


def _block_fn(F):
    if callable(F):
        return F
    F = np.asarray(F, dtype=np.float64)
    return lambda k: F[k]


def forward(F, m, N_t=None):
    """d = F m (Eq. ShiftInvariance)."""
    m = np.asarray(m, dtype=np.float64)
    N_t = m.shape[-2] if N_t is None else N_t
    blk = _block_fn(F)
    d = None
    for k in range(N_t):
        Fk = blk(k)
        if d is None:
            d = np.zeros(m.shape[:-2] + (N_t, Fk.shape[0]), dtype=np.float64)
        # every (i, j = i - k): d_i += F_k m_{i-k}
        d[..., k:, :] += m[..., : N_t - k, :] @ Fk.T
    return d


def adjoint(F, d, N_t=None):
    """m = F* d, the block upper-triangular transpose."""
    d = np.asarray(d, dtype=np.float64)
    N_t = d.shape[-2] if N_t is None else N_t
    blk = _block_fn(F)
    m = None
    for k in range(N_t):
        Fk = blk(k)
        if m is None:
            m = np.zeros(d.shape[:-2] + (N_t, Fk.shape[1]), dtype=np.float64)
        # every (j, i = j + k): m_j += F_k^T d_{j+k}
        m[..., : N_t - k, :] += d[..., k:, :] @ Fk
    return m


def hessian(F, m, gamma_inv=None, N_t=None):
    """H m = F* Gamma^-1 F m with diagonal Gamma^-1 [N_t][N_d] (None = I)."""
    d = forward(F, m, N_t)
    if gamma_inv is not None:
        d = d * np.asarray(gamma_inv, dtype=np.float64)
    return adjoint(F, d, N_t)


def forward_entries(row_fn, m, samples):
    """Sampled entries d_i[s] of F m for one vector m [N_t][N_m].

    ``row_fn(ks, s)`` returns the rows F_k[s, :] for the lags ``ks`` as an
    array [len(ks)][N_m].  ``samples`` is a list of (i, s).
    d_i[s] = sum_{k=0}^{i} F_k[s, :] . m_{i-k}
    """
    m = np.asarray(m, dtype=np.float64)
    out = np.empty(len(samples), dtype=np.float64)
    for n, (i, s) in enumerate(samples):
        ks = np.arange(i + 1)
        rows = row_fn(ks, s)
        out[n] = np.sum(rows * m[i - ks, :])
    return out


def adjoint_entries(col_fn, d, samples):
    """Sampled entries m_j[l] of F* d for one vector d [N_t][N_d].

    ``col_fn(ks, l)`` returns the columns F_k[:, l] as [len(ks)][N_d].
    m_j[l] = sum_{k=0}^{N_t-1-j} F_k[:, l] . d_{j+k}
    """
    d = np.asarray(d, dtype=np.float64)
    N_t = d.shape[0]
    out = np.empty(len(samples), dtype=np.float64)
    for n, (j, l) in enumerate(samples):
        ks = np.arange(N_t - j)
        cols = col_fn(ks, l)
        out[n] = np.sum(cols * d[j + ks, :])
    return out


def rel_l2(x, ref):
    """Relative l2 error ||x - ref|| / ||ref|| in float64."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref.ravel())
    num = np.linalg.norm((x - ref).ravel())
    return num / den if den > 0 else num
