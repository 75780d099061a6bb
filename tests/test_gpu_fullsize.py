"""Parity at the full workload sizes, in the launch configuration bench.py
times (operator built from device-generated blocks, FP32 vectors resident
on the device): whole outputs of F, F* and the Hessian against the FP64
oracle (relative l2 over every entry; the oracle reads the seeded blocks
one lag at a time), and properties that hold at any size (the adjoint
identity, Hessian symmetry, H = F* Gamma^-1 F through separate calls).
The four serving operators are checked on sampled entries computed one by
one from the seeded generator."""
import numpy as np
import pytest
import torch

import synth
from oracle import direct
import paper_2407_13066_gb300 as btt

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "bf16x2": 1e-5, "f16s": 2e-3, "bf16": 1e-2, "fp8s": 6e-2}


def device_blocks(w):
    t = torch.empty((w.N_t, w.N_d, w.N_m), dtype=torch.float64, device="cuda")
    ed, em = synth.envelope(w, "d"), synth.envelope(w, "m")
    ed_t = None if ed is None else torch.from_numpy(ed).cuda()
    em_t = None if em is None else torch.from_numpy(em).cuda()
    rc = synth.dev_lib().synth_dev_blocks(w.seed, w.N_d, w.N_m, float(w.tau),
                                          None if ed_t is None else ed_t.data_ptr(),
                                          None if em_t is None else em_t.data_ptr(),
                                          0, w.N_t, t.data_ptr(), None)
    assert rc == 0
    torch.cuda.synchronize()
    return t


def device_normals(w, tid, shape):
    x = torch.empty(shape, dtype=torch.float32, device="cuda")
    assert synth.dev_lib().synth_dev_normal(w.seed, tid, 0, x.numel(), None, x.data_ptr(), None) == 0
    return x


def device_gamma_inv(w):
    g = torch.empty((w.N_t, w.N_d), dtype=torch.float32, device="cuda")
    assert synth.dev_lib().synth_dev_uniform(w.seed, synth.workloads.T_NOISE, 0, g.numel(), 0.5, 2.0,
                                             None, g.data_ptr(), None) == 0
    return 1.0 / g


def lag_source(blocks):
    """Block source for the oracle: lag k of the seeded blocks (generated on
    the device by the input generator) as a float64 host array."""
    return lambda k: blocks[k].cpu().numpy()


def whole(w, blocks, m, d, g):
    """FP64 oracle F m, F* d and F* Gamma^-1 F m (Eq. ShiftInvariance, its
    transpose, Sec. 2.2) over every entry; m [..., N_t, N_m], d [..., N_t, N_d]."""
    src = lag_source(blocks)
    return (direct.forward(src, m, w.N_t), direct.adjoint(src, d, w.N_t),
            direct.hessian(src, m, g, w.N_t))


def host(x):
    return x.double().cpu().numpy()


def samples(w, n, seed):
    rng = np.random.default_rng(seed)
    fs = [(int(i), int(s)) for i, s in zip(rng.integers(0, w.N_t, n), rng.integers(0, w.N_d, n))]
    fs += [(w.N_t - 1, w.N_d - 1), (0, 0)]
    as_ = [(int(j), int(l)) for j, l in zip(rng.integers(0, w.N_t, n), rng.integers(0, w.N_m, n))]
    as_ += [(0, 0), (w.N_t - 1, w.N_m - 1)]
    return fs, as_


def oracle_samples(w, m, d, fs, as_):
    row_fn = lambda ks, s: synth.block_entries(w, ks[:, None], s, np.arange(w.N_m)[None, :])
    col_fn = lambda ks, l: synth.block_entries(w, ks[:, None], np.arange(w.N_d)[None, :], l)
    return direct.forward_entries(row_fn, m, fs), direct.adjoint_entries(col_fn, d, as_)


def check_entries(w, m, d, dm, md, n, tol, seed):
    """Sampled entries of F m and F* d (one vector each) against the oracle."""
    fs, as_ = samples(w, n, seed)
    ref_f, ref_a = oracle_samples(w, m, d, fs, as_)
    got_f = np.array([dm[i, s] for i, s in fs])
    got_a = np.array([md[j, l] for j, l in as_])
    ef, ea = direct.rel_l2(got_f, ref_f), direct.rel_l2(got_a, ref_a)
    assert ef < tol and ea < tol, (ef, ea)
    return ef, ea


def inner(a, b):
    return float(torch.sum(a.double() * b.double()))


def norm(a):
    return float(torch.linalg.vector_norm(a.double()))


def test_bandwidth_workload_fp32():
    """Config 2 (1000, 100, 10 000), FP32 storage, one vector (the bench step):
    whole F m, F* d and F* Gamma^-1 F m against the FP64 oracle at 1e-5."""
    w = synth.WORKLOADS["bandwidth"]
    blocks = device_blocks(w)
    op = btt.Operator(blocks, precision="f32", max_nrhs=1)
    m = device_normals(w, synth.workloads.T_PARAM, (1, w.N_t, w.N_m))
    d = device_normals(w, synth.workloads.T_DATA, (1, w.N_t, w.N_d))
    g = device_gamma_inv(w)
    dm, md = op.matvec(m), op.adjoint(d)
    hm = op.hessian(m, g)
    x = device_normals(w, synth.workloads.T_DIRS, (1, w.N_t, w.N_m))
    hx = op.hessian(x, g)
    hm2 = op.adjoint(op.matvec(m) * g)
    op.device_status()
    torch.cuda.synchronize()
    ref_f, ref_a, ref_h = whole(w, blocks, host(m[0]), host(d[0]), host(g))
    del blocks
    errs = (direct.rel_l2(host(dm[0]), ref_f), direct.rel_l2(host(md[0]), ref_a),
            direct.rel_l2(host(hm[0]), ref_h))
    assert max(errs) < TOL["f32"], errs
    # <F m, d> = <m, F* d>
    assert abs(inner(dm, d) - inner(m, md)) <= 1e-5 * norm(dm) * norm(d)
    # <H m, x> = <m, H x>, <H m, m> > 0, H = F* Gamma^-1 F through separate calls
    assert abs(inner(hm, x) - inner(m, hx)) <= 1e-5 * norm(hm) * norm(x)
    assert inner(hm, m) > 0
    assert norm(hm - hm2) <= 1e-5 * norm(hm)
    op.close()


@pytest.fixture(scope="module")
def precision_case():
    """Config 3's blocks on the device, one vector each of m and d, the
    noise precision, and the FP64 oracle's whole F m, F* d and Hessian
    (the same for every storage format)."""
    w = synth.WORKLOADS["precision"]
    t = device_blocks(w)
    m = device_normals(w, synth.workloads.T_PARAM, (1, w.N_t, w.N_m))
    d = device_normals(w, synth.workloads.T_DATA, (1, w.N_t, w.N_d))
    g = device_gamma_inv(w)
    refs = whole(w, t, host(m[0]), host(d[0]), host(g))
    yield w, t, m, d, g, refs
    del t
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["f32", "f16s", "bf16", "bf16x2", "fp8s"])
def test_precision_workload_formats(precision_case, prec):
    """Config 3 (512, 600, 20 000, smooth envelopes), every storage format:
    whole F m, F* d and F* Gamma^-1 F m against the FP64 oracle at the
    format's tolerance."""
    w, blocks, m, d, g, (ref_f, ref_a, ref_h) = precision_case
    op = btt.Operator(blocks, precision=prec, max_nrhs=1)
    dm, md = op.matvec(m), op.adjoint(d)
    hm = op.hessian(m, g)
    op.device_status()
    torch.cuda.synchronize()
    errs = (direct.rel_l2(host(dm[0]), ref_f), direct.rel_l2(host(md[0]), ref_a),
            direct.rel_l2(host(hm[0]), ref_h))
    assert max(errs) < TOL[prec], errs
    assert abs(inner(dm, d) - inner(m, md)) <= 4 * TOL[prec] * norm(dm) * norm(d)
    op.close()
    torch.cuda.empty_cache()


PICK = [0, 21, 42, 63]


@pytest.fixture(scope="module")
def multi_rhs_case():
    """Config 4's blocks on the device, the 64-vector batches m, d and x,
    the noise precision, and the FP64 oracle's whole F m, F* d and Hessian
    for vectors 0, 21, 42 and 63 (the same for every format and path)."""
    w = synth.WORKLOADS["multi-rhs"]
    B = w.nrhs
    t = device_blocks(w)
    m = device_normals(w, synth.workloads.T_PARAM, (B, w.N_t, w.N_m))
    d = device_normals(w, synth.workloads.T_DATA, (B, w.N_t, w.N_d))
    x = device_normals(w, synth.workloads.T_DIRS, (B, w.N_t, w.N_m))
    g = device_gamma_inv(w)
    refs = whole(w, t, host(m[PICK]), host(d[PICK]), host(g))
    yield w, t, m, d, x, g, refs
    del t
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec,gemm,tol", [("bf16", "tensor", 1e-2), ("bf16", "simt", 1e-2),
                                           ("bf16x2", "tensor", 1e-5)])
def test_multi_rhs_workload(multi_rhs_case, prec, gemm, tol):
    """Config 4 (256, 200, 50 000), 64 vectors, BF16 storage (or the split
    pair, whose forward there drains 7 accumulation chains per CTA):
    whole outputs of vectors 0, 21, 42, 63 of F, F* and the Hessian batch
    against the FP64 oracle; all 64 through the adjoint identity; the
    Hessian batch is symmetric."""
    w, blocks, m, d, x, g, (ref_f, ref_a, ref_h) = multi_rhs_case
    B = w.nrhs
    op = btt.Operator(blocks, precision=prec, max_nrhs=B, gemm=gemm)
    dm, md = op.matvec(m), op.adjoint(d)
    hm = op.hessian(m, g)
    hx = op.hessian(x, g)
    op.device_status()
    torch.cuda.synchronize()
    for n, b in enumerate(PICK):
        errs = (direct.rel_l2(host(dm[b]), ref_f[n]), direct.rel_l2(host(md[b]), ref_a[n]),
                direct.rel_l2(host(hm[b]), ref_h[n]))
        assert max(errs) < tol, (b, errs)
    for b in range(B):
        assert abs(inner(dm[b], d[b]) - inner(m[b], md[b])) <= 4 * tol * norm(dm[b]) * norm(d[b])
        assert abs(inner(hm[b], x[b]) - inner(m[b], hx[b])) <= 4 * tol * norm(hm[b]) * norm(x[b])
    op.close()
    del dm, md, hm, hx
    torch.cuda.empty_cache()


def test_serving_operators_resident():
    """Config 5: the four serving operators resident at once (BF16, tensor
    cores, 47 GB), each checked on sampled entries of F and F*."""
    ops, ws = [], []
    for w in synth.workloads.SERVING_OPERATORS:
        blocks = device_blocks(w)
        ops.append(btt.Operator(blocks, precision="bf16", max_nrhs=8, gemm="tensor"))
        ws.append(w)
        del blocks
        torch.cuda.empty_cache()
    for k, (w, op) in enumerate(zip(ws, ops)):
        m = device_normals(w, synth.workloads.T_PARAM, (8, w.N_t, w.N_m))
        d = device_normals(w, synth.workloads.T_DATA, (8, w.N_t, w.N_d))
        dm, md = op.matvec(m), op.adjoint(d)
        op.device_status()
        torch.cuda.synchronize()
        check_entries(w, m[3].double().cpu().numpy(), d[3].double().cpu().numpy(),
                      dm[3].double().cpu().numpy(), md[3].double().cpu().numpy(), 6, 1e-2, 30 + k)
    for op in ops:
        op.close()
    torch.cuda.empty_cache()
