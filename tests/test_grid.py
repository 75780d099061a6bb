"""Grid selection (Alg. 4, Eq. comm-cost) pinned to the paper's observed
optima, and the 1 x p parameter-split layout checked with gloo ranks on the
CPU against the oracle: the split itself, and the composition of the split
actions (grid.split_forward / split_hessian) around a sum-reduction."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2407_13066_gb300 import grid


def test_comm_cost_closed_form():
    # C(1) has no broadcast term; C(p) no reduction term
    assert grid.comm_cost(1, 80, -2) == pytest.approx(0.01 * math.log(80))
    assert grid.comm_cost(80, 80, -2) == pytest.approx(math.log(80))
    assert grid.comm_cost(2, 80, -2) == pytest.approx(2 / 80 * math.log(2) + 0.005 * math.log(40))


@pytest.mark.parametrize("l,expected", [(-4, (1, 80)), (-3, (1, 80)), (-2, (4, 20))])
def test_select_grid_reproduces_observed_optima(l, expected):
    """Fig. GridTest: 80 GPUs, 4 per node (Frontera), observed optimal rows
    r = 1, 1, 4 for l = -4, -3, -2."""
    assert grid.select_grid(80, l, k=4) == expected


def test_select_grid_properties():
    for p in (1, 2, 6, 12, 48, 80):
        for l in (-4, -2, -1, 0, 1, 2):
            r, c = grid.select_grid(p, l, k=4)
            assert r * c == p
            if p > 1 and r not in (1, p):
                assert (r >= c) == (l >= 0)
    assert grid.select_grid(48, 3, k=3)[0] > grid.select_grid(48, -3, k=3)[0]


def test_weak_scaling_grid():
    assert grid.weak_scaling_grid(10, 20000, 48) == (1, 48)   # the paper's runs (Sec. 4.2)
    assert grid.weak_scaling_grid(500, 20, 8) == (8, 1)


def test_column_slices():
    assert grid.column_slices(10, 3) == [(0, 4), (4, 8), (8, 10)]
    assert grid.column_slices(5, 8)[-1] == (5, 5)
    sl = grid.column_slices(10007, 16)
    assert sl[0][0] == 0 and sl[-1][1] == 10007 and all(a[1] == b[0] for a, b in zip(sl, sl[1:]))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import synth
    from oracle import direct
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.Workload("split", 12, 5, 23, tau=4.0, seed=3)
        F = synth.blocks(w)
        m = synth.vectors(w, "m", 1)[0]
        d = synth.vectors(w, "d", 1)[0]
        a, b = grid.column_slices(w.N_m, world)[rank]
        # F: each rank applies its column slice; one sum-reduction of N_t N_d values
        part = torch.from_numpy(direct.forward(F[:, :, a:b], m[:, a:b]))
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        # F*: d is replicated, each rank produces its own slice; no communication
        mine = direct.adjoint(F[:, :, a:b], d)
        out.put((rank, part.numpy(), mine, a, b))
    finally:
        dist.destroy_process_group()


def test_parameter_split_two_gloo_ranks():
    import synth
    from oracle import direct
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = synth.Workload("split", 12, 5, 23, tau=4.0, seed=3)
    F = synth.blocks(w)
    m = synth.vectors(w, "m", 1)[0]
    d = synth.vectors(w, "d", 1)[0]
    full_d = direct.forward(F, m)
    full_m = direct.adjoint(F, d)
    for rank, dsum, mine, a, b in res:
        np.testing.assert_allclose(dsum, full_d, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(mine, full_m[:, a:b], rtol=1e-12, atol=1e-12)


def test_boundary_threshold_from_derivative():
    """dC/dr at r = 1 is 1/p - 10^l (ln p + 1): the minimiser leaves r = 1
    exactly when l exceeds log10(1 / (p (ln p + 1)))."""
    p = 80
    l_star = math.log10(1.0 / (p * (math.log(p) + 1.0)))
    assert grid._argmin_continuous(p, l_star - 0.02) == 1.0
    assert grid._argmin_continuous(p, l_star + 0.02) > 1.0
    assert grid.select_grid(p, l_star - 0.02, k=1) == (1, p)
    # just past the threshold the minimiser is still nearest to r = 1
    assert grid.select_grid(p, l_star + 0.02, k=1) == (1, p)


class _OracleSlice:
    """Stand-in for an operator on one column slice (CPU, FP64 oracle): the
    same matvec / adjoint(gamma_inv=) calls the library's Operator offers."""

    def __init__(self, F):
        self.F = F

    def matvec(self, m, out=None):
        from oracle import direct
        d = torch.from_numpy(direct.forward(self.F, m.numpy()))
        return d if out is None else out.copy_(d)

    def adjoint(self, d, out=None, gamma_inv=None):
        from oracle import direct
        x = d.numpy() if gamma_inv is None else d.numpy() * gamma_inv.numpy()
        m = torch.from_numpy(direct.adjoint(self.F, x))
        return m if out is None else out.copy_(m)


def _split_rank(rank, world, port, out):
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.Workload("split", 12, 5, 23, tau=4.0, seed=3)
        F = synth.blocks(w)
        m = torch.from_numpy(synth.vectors(w, "m", 2))
        g = torch.from_numpy(synth.noise_gamma_inv(w))
        a, b = grid.column_slices(w.N_m, world)[rank]
        op = _OracleSlice(np.ascontiguousarray(F[:, :, a:b]))
        ar = lambda x: dist.all_reduce(x, op=dist.ReduceOp.SUM)
        d = grid.split_forward(op, m[:, :, a:b].contiguous(), ar)
        y = grid.split_hessian(op, m[:, :, a:b].contiguous(), g, ar)
        out.put((rank, d.numpy(), y.numpy(), a, b))
    except Exception as e:   # reported to the parent instead of leaving it waiting
        out.put((rank, None, repr(e), 0, 0))
        raise
    finally:
        dist.destroy_process_group()


def test_split_hessian_three_gloo_ranks():
    """grid.split_forward / split_hessian over three gloo ranks (ragged
    slices), each rank's operator an oracle stand-in: the assembled F m and
    F* Gamma^-1 F m equal the unsplit oracle's."""
    import synth
    from oracle import direct
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank, args=(r, 3, port, q)) for r in range(3)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in range(3)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
    assert all(r[1] is not None for r in res), [r[2] for r in res if r[1] is None]
    assert all(p.exitcode == 0 for p in procs)
    w = synth.Workload("split", 12, 5, 23, tau=4.0, seed=3)
    F = synth.blocks(w)
    m = synth.vectors(w, "m", 2)
    g = synth.noise_gamma_inv(w)
    full_d = direct.forward(F, m)
    full_h = direct.hessian(F, m, g)
    y = np.concatenate([r[2] for r in res], axis=-1)
    for rank, d, _, a, b in res:
        np.testing.assert_allclose(d, full_d, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(y, full_h, rtol=1e-12, atol=1e-12)
