"""The 1 x p parameter split (Sec. 3.2 partition, Sec. 3.5 reduce) through the
library: each part is an operator on a column slice Fhat[:, :, a:b]; F m is
the sum of the parts' btt_matvec outputs (one sum-reduction of N_t x N_d
values), F* d needs no exchange, and a Hessian action is btt_matvec, the
sum, then btt_adjoint_weighted on the replicated data.  Checked against the
FP64 oracle of the whole operator (whole outputs), in one process (the sum
taken on the device, standing in for the all-reduce) and in two processes
sharing one GPU whose partial data vectors are summed by a gloo all-reduce
of host copies (no kernel of one process waits on the other)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from oracle import direct
import paper_2407_13066_gb300 as btt
from paper_2407_13066_gb300 import grid

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# (N_t, N_d, N_m, p, nrhs, precision, gemm, tol): the generic transforms,
# the fixed-plan (cluster) length of the bandwidth workload, and the BF16
# tensor-core path on 16 vectors
CASES = [
    (100, 7, 203, 3, 2, "f32", "auto", 1e-5),
    (1000, 10, 301, 3, 1, "f32", "auto", 1e-5),
    (64, 24, 250, 2, 16, "bf16x2", "tensor", 1e-5),
    (64, 24, 250, 2, 16, "bf16", "tensor", 1e-2),
]


@pytest.mark.parametrize("case", CASES, ids=["L200", "L2000", "L128-bf16x2-tc", "L128-bf16-tc"])
def test_column_split_one_process(case):
    N_t, N_d, N_m, p, nrhs, prec, gemm, tol = case
    w = synth.Workload("split", N_t, N_d, N_m, tau=N_t / 4, seed=5)
    F = synth.blocks(w)
    m = synth.vectors(w, "m", nrhs).astype(np.float32)
    d = synth.vectors(w, "d", nrhs).astype(np.float32)
    g = synth.noise_gamma_inv(w).astype(np.float32)
    gd = _dev(g)
    parts = []
    for a, b in grid.column_slices(N_m, p):
        op = btt.Operator(np.ascontiguousarray(F[:, :, a:b]), precision=prec, max_nrhs=nrhs, gemm=gemm)
        parts.append((op, a, b, _dev(m[:, :, a:b])))
    # F m: partials summed (the all-reduce); F* d: each part its own columns
    dsum = torch.zeros((nrhs, N_t, N_d), device="cuda")
    for op, a, b, mq in parts:
        dsum += op.matvec(mq)
    fstar = [op.adjoint(_dev(d)) for op, a, b, mq in parts]
    y = [op.adjoint(dsum, gamma_inv=gd) for op, a, b, mq in parts]
    for op, *_ in parts:
        op.device_status()
    torch.cuda.synchronize()
    ref_f, ref_a, ref_h = direct.forward(F, m), direct.adjoint(F, d), direct.hessian(F, m, g)
    assert direct.rel_l2(dsum.double().cpu().numpy(), ref_f) < tol
    assert direct.rel_l2(torch.cat(fstar, -1).double().cpu().numpy(), ref_a) < tol
    y = torch.cat(y, -1).double().cpu().numpy()
    assert direct.rel_l2(y, ref_h) < tol
    # with p = 1 the two calls equal btt_hessian (fused hand-off)
    with btt.Operator(F, precision=prec, max_nrhs=nrhs, gemm=gemm) as whole:
        md = _dev(m)
        y1 = grid.split_hessian(whole, md, gd)
        yh = whole.hessian(md, gd)
        torch.cuda.synchronize()
        assert direct.rel_l2(y1.double().cpu().numpy(), yh.double().cpu().numpy()) < tol
    for op, *_ in parts:
        op.close()


def test_adjoint_weighted_host_vectors_in_chunks():
    """btt_adjoint_weighted with host data and a host noise precision, five
    vectors through an operator holding two per pass (three chunks)."""
    w = synth.Workload("split", 128, 9, 77, tau=30.0, seed=6)
    F = synth.blocks(w)
    d = synth.vectors(w, "d", 5).astype(np.float32)
    g = synth.noise_gamma_inv(w).astype(np.float32)
    with btt.Operator(F, precision="f32", max_nrhs=2) as op:
        got = op.adjoint(d, gamma_inv=g)
        ref = direct.adjoint(F, d.astype(np.float64) * g)
        assert direct.rel_l2(got, ref) < 1e-5
        # the workspace query for a larger batch: more than this operator's
        assert op.workspace_bytes(8) > op.workspace_bytes() == op.workspace_bytes(2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


SPLIT2 = (200, 12, 311)


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        N_t, N_d, N_m = SPLIT2
        w = synth.Workload("split", N_t, N_d, N_m, tau=N_t / 4, seed=7)
        F = synth.blocks(w)
        m = synth.vectors(w, "m", 2).astype(np.float32)
        g = _dev(synth.noise_gamma_inv(w).astype(np.float32))
        a, b = grid.column_slices(N_m, world)[rank]

        def host_allreduce(x):
            h = x.cpu()
            dist.all_reduce(h, op=dist.ReduceOp.SUM)
            x.copy_(h)

        with btt.Operator(np.ascontiguousarray(F[:, :, a:b]), precision="f32", max_nrhs=2) as op:
            y = grid.split_hessian(op, _dev(m[:, :, a:b]), g, allreduce=host_allreduce)
            op.device_status()
            torch.cuda.synchronize()
            out.put((rank, y.cpu().numpy(), a, b))
    finally:
        dist.destroy_process_group()


def test_column_split_two_processes_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    N_t, N_d, N_m = SPLIT2
    w = synth.Workload("split", N_t, N_d, N_m, tau=N_t / 4, seed=7)
    F = synth.blocks(w)
    m = synth.vectors(w, "m", 2).astype(np.float32)
    g = synth.noise_gamma_inv(w).astype(np.float32)
    y = np.concatenate([r[1] for r in res], axis=-1)
    assert [(r[2], r[3]) for r in res] == grid.column_slices(N_m, 2)
    assert direct.rel_l2(y, direct.hessian(F, m, g)) < 1e-5
