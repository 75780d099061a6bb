"""The serving loop (native scheduler, continuous batching, admission under
a device-memory pool): each result is the same alone and in the mix,
results match the oracle, admission respects the pool, and injected
host-side failures fail only their own requests."""
import numpy as np
import pytest
import torch

import synth
from oracle import direct
import paper_2407_13066_gb300 as btt
from paper_2407_13066_gb300.serve import Server, FAULT_ADMIT, FAULT_BATCH

pytestmark = pytest.mark.gpu

OPS = [  # (N_t, N_d, N_m, precision, gemm)
    (40, 12, 100, "bf16", "tensor"),
    (64, 8, 50, "f32", "simt"),
    (25, 30, 200, "bf16", "tensor"),
]


def make_ops(max_batch):
    ops, Fs, gs = [], [], []
    for i, (N_t, N_d, N_m, prec, gemm) in enumerate(OPS):
        w = synth.Workload("srv%d" % i, N_t, N_d, N_m, tau=N_t / 4, seed=40 + i)
        F = synth.blocks(w)
        Fs.append(F)
        gs.append(synth.noise_gamma_inv(w).astype(np.float32))
        ops.append(btt.Operator(F, precision=prec, max_nrhs=max_batch, gemm=gemm))
    return ops, Fs, gs


def requests(n, seed, max_vec):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        op = int(rng.integers(0, len(OPS)))
        nvec = int(rng.integers(1, max_vec + 1))
        N_t, _, N_m = OPS[op][:3]
        m = synth.normals(seed, 100 + k, nvec * N_t * N_m).astype(np.float32).reshape(nvec, N_t, N_m)
        out.append((op, m))
    return out


def test_each_result_same_alone_and_in_the_mix():
    ops, Fs, gs = make_ops(32)
    gam = [torch.from_numpy(g).cuda() for g in gs]
    reqs = requests(40, 7, 8)
    with Server(ops, gamma_inv=gam, pool_bytes=64 << 20, max_batch=32) as srv:
        alone = []
        for op, m in reqs:                      # one request at a time
            x = torch.from_numpy(m).cuda()
            y = torch.empty_like(x)
            srv.wait(srv.submit(op, x, y))
            alone.append(y.cpu().numpy())
        mix_in = [torch.from_numpy(m).cuda() for _, m in reqs]
        mix_out = [torch.empty_like(x) for x in mix_in]
        tickets = [srv.submit(op, x, y) for (op, _), x, y in zip(reqs, mix_in, mix_out)]
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
    assert st["completed"] == 80 and st["failed"] == 0
    assert st["mean_batch_vectors"] > 1.0          # the mix was batched
    bitwise = 0
    for (op, m), a, y in zip(reqs, alone, mix_out):
        b = y.cpu().numpy()
        assert direct.rel_l2(b, a) < 1e-6
        bitwise += int(np.array_equal(a, b))
        tol = 1e-2 if OPS[op][3] == "bf16" else 1e-5
        ref = direct.hessian(Fs[op], m.astype(np.float64), gs[op].astype(np.float64))
        assert direct.rel_l2(b, ref) < tol
    # the tensor-core path accumulates each vector in a fixed order whatever
    # the batch: its results are bit-identical alone and in the mix
    assert bitwise >= sum(1 for op, _ in reqs if OPS[op][4] == "tensor")
    for o in ops:
        o.close()


def test_host_requests_wait_for_pool_memory():
    ops, Fs, gs = make_ops(16)
    reqs = requests(24, 11, 6)
    # host vectors need input + output slots; the pool holds about two requests
    largest = max(2 * m.nbytes for _, m in reqs)
    pool = 2 * largest + 4096
    with Server(ops, pool_bytes=pool, max_batch=16) as srv:
        ins = [torch.from_numpy(m).pin_memory() for _, m in reqs]
        outs = [torch.empty(x.shape, dtype=torch.float32).pin_memory() for x in ins]
        tickets = [srv.submit(op, x, y) for (op, _), x, y in zip(reqs, ins, outs)]
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
    assert st["completed"] == 24
    assert 0 < st["pool_high_water"] <= pool
    assert st["pool_in_use"] == 0
    for (op, m), y in zip(reqs, outs):
        tol = 1e-2 if OPS[op][3] == "bf16" else 1e-5
        assert direct.rel_l2(y.numpy(), direct.hessian(Fs[op], m.astype(np.float64))) < tol
    for o in ops:
        o.close()


def test_injected_failures_fail_only_their_requests():
    ops, Fs, gs = make_ops(8)
    reqs = requests(6, 3, 4)
    with Server(ops, pool_bytes=32 << 20, max_batch=8) as srv:
        xs = [torch.from_numpy(m).cuda() for _, m in reqs]
        ys = [torch.empty_like(x) for x in xs]
        srv.inject(FAULT_BATCH)
        t0 = srv.submit(reqs[0][0], xs[0], ys[0])
        with pytest.raises(btt.BttError):
            srv.wait(t0)
        srv.inject(FAULT_ADMIT)
        t1 = srv.submit(reqs[1][0], xs[1], ys[1])
        with pytest.raises(btt.BttError) as e:
            srv.wait(t1)
        assert e.value.status == btt._lib.BTT_ERR_OOM
        ts = [srv.submit(op, x, y) for (op, _), x, y in zip(reqs[2:], xs[2:], ys[2:])]
        for t in ts:
            srv.wait(t)
        st = srv.stats()
        assert st["failed"] == 2 and st["completed"] == 4
        # arguments the server can never serve are refused at submit
        o = OPS[0]
        big = torch.zeros((9, o[0], o[2]), device="cuda")
        with pytest.raises(btt.BttError):
            srv.submit(0, big, big.clone())
        huge = torch.zeros((8, o[0], o[2]))
        with Server(ops[:1], pool_bytes=1 << 16, max_batch=8) as small:
            with pytest.raises(btt.BttError) as e:
                small.submit(0, huge, huge.clone())
            assert e.value.status == btt._lib.BTT_ERR_OOM
    for o in ops:
        o.close()
