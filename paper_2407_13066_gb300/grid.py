"""Processor-grid selection and the parameter-split layout (Sec. 3.2, 3.7).

Host-side planning for running the operator over p GPUs; the kernels of
this package run on one GPU, and these functions say how the work would be
split and where the collectives would go.

comm_cost(r, p, l)
    The modified asymptotic communication cost of Eq. comm-cost,
    C(r; p, l) = (r/p) log r + (10^l / r) log(p/r), for an r x (p/r) grid and
    l = log10(N_d / N_m): the broadcast of the input down the r rows and
    the reduction over the p/r columns of one F and one F* matvec, with the
    latency and bandwidth constants removed.
select_grid(p, l, k)
    Alg. 4: the real minimiser of comm_cost, then a divisor pair of p near
    it, preferring k | r (k GPUs per node: rows within a node), and r >= c
    when l >= 0, r < c otherwise.
weak_scaling_grid(n_d, n_m, p)
    The remark on scaling tests: with fixed local sizes the cost is
    (1 - n_d/n_m) log r, so 1 x p if n_d < n_m, p x 1 if n_d > n_m.
column_slices(N_m, p)
    The 1 x p layout (each GPU holds Fhat[:, :, slice] and its slice of m;
    F needs one sum-reduction of the N_t N_d data vector, F* none).
split_forward(op, m, allreduce), split_hessian(op, m, gamma_inv, allreduce)
    The actions of the 1 x p layout on one GPU's operator: that GPU's
    column slice through the library, with the caller's sum-reduction
    (allreduce(d) in place, e.g. torch.distributed.all_reduce over NCCL)
    between the passes.  F* d needs no exchange: op.adjoint(d).
"""
import math


def comm_cost(r, p, l):
    """C(r; p, l) of Eq. comm-cost (natural logarithms; the base only scales it)."""
    if not (1 <= r <= p):
        raise ValueError("r must lie in [1, p]")
    return (r / p) * math.log(r) + (10.0 ** l / r) * math.log(p / r)


def _argmin_continuous(p, l):
    """Real minimiser of comm_cost over [1, p]: a dense scan of log r, then
    golden-section refinement around the best sample."""
    if p == 1:
        return 1.0
    lp = math.log(p)
    f = lambda t: comm_cost(min(max(math.exp(t), 1.0), float(p)), p, l)
    n = 4096
    i = min(range(n + 1), key=lambda j: f(lp * j / n))
    if i == 0:
        return 1.0
    if i == n:
        return float(p)
    a, b = lp * (i - 1) / n, lp * (i + 1) / n
    g = (math.sqrt(5) - 1) / 2
    for _ in range(100):
        c, d = b - g * (b - a), a + g * (b - a)
        if f(c) < f(d):
            b = d
        else:
            a = c
    return math.exp((a + b) / 2)


def select_grid(p, l, k=1):
    """Alg. 4: returns (r, c) with r * c = p.

    The continuous minimiser decides the two boundary cases.  Otherwise r is
    a divisor of p on the side the sign of l asks for (r >= c when l >= 0,
    r < c otherwise), nearest to the minimiser on a log scale, taking first
    the divisors with k | r (column traffic stays on a node once k | r, so
    r = k costs no more than r = 2 along columns and shortens the rows),
    then those with k | c, then any."""
    if p < 1 or k < 1:
        raise ValueError("p and k must be >= 1")
    rt = _argmin_continuous(p, l)
    if rt <= 1.0:
        return 1, p
    if rt >= p:
        return p, 1
    divisors = [r for r in range(1, p + 1) if p % r == 0]
    side = [r for r in divisors if (r >= p // r) == (l >= 0)] or divisors
    near = lambda r: abs(math.log(r) - math.log(rt))
    for tier in ([r for r in side if k > 1 and r % k == 0],
                 [r for r in side if k > 1 and (p // r) % k == 0],
                 side):
        if tier:
            r = min(tier, key=near)
            return r, p // r
    raise AssertionError("unreachable")


def weak_scaling_grid(n_d, n_m, p):
    """Grid for weak scaling with fixed local sizes (remark after Alg. 4)."""
    if n_d < n_m:
        return 1, p
    if n_d > n_m:
        return p, 1
    return 1, p


def column_slices(N_m, p):
    """[start, stop) of the parameter columns held by each of p GPUs in the
    1 x p layout, sizes ceil(N_m / p) (the last may be shorter or empty)."""
    n = -(-N_m // p)
    return [(min(q * n, N_m), min((q + 1) * n, N_m)) for q in range(p)]


def split_forward(op, m, allreduce=None, out=None):
    """d = F m in the 1 x p layout: this GPU's partial F_q m_q (btt_matvec on
    the operator of its column slice), then the sum over the GPUs (the
    reduce of Alg. 2; allreduce(d) sums in place, None for p = 1)."""
    d = op.matvec(m, out=out)
    if allreduce is not None:
        allreduce(d)
    return d


def split_hessian(op, m, gamma_inv=None, allreduce=None, out=None, work=None):
    """This GPU's slice of F* Gamma^-1 F m in the 1 x p layout: the forward
    pass and its sum-reduction (split_forward, into `work` if given), then
    the weighted adjoint on the replicated data (btt_adjoint_weighted),
    which needs no exchange: one all-reduce of N_t N_d values per vector
    between the passes."""
    d = split_forward(op, m, allreduce, out=work)
    return op.adjoint(d, out=out, gamma_inv=gamma_inv)
