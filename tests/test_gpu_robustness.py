"""Operator files (save, load), host-side fault injection, and run-to-run
determinism of every product path."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import synth
from oracle import direct
import paper_2407_13066_gb300 as btt
from paper_2407_13066_gb300 import _lib

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("prec", ["f32", "f16s", "bf16x2", "fp8s", "f64"])
def test_save_load_round_trip(tmp_path, prec):
    w = synth.Workload("file", 30, 5, 47, tau=6.0, envelope=True, seed=21)
    F = synth.blocks(w)
    path = tmp_path / ("op_%s.btt" % prec)
    dt = torch.float64 if prec == "f64" else torch.float32
    m = torch.from_numpy(synth.vectors(w, "m", 2)).to(dt).cuda()
    with btt.Operator(F, precision=prec, max_nrhs=2) as op:
        op.save(path)
        raw, sc = op.copy_fhat()
        y = op.matvec(m)
    with btt.Operator.load(path, max_nrhs=2) as op2:
        assert op2.precision == prec and (op2.N_t, op2.N_d, op2.N_m) == (w.N_t, w.N_d, w.N_m)
        raw2, sc2 = op2.copy_fhat()
        y2 = op2.matvec(m)
        op2.device_status()
    scaled = prec in ("f16s", "fp8s")
    assert np.array_equal(raw, raw2)
    if scaled:
        assert np.array_equal(sc, sc2)
    assert torch.equal(y, y2)
    size = os.path.getsize(path)
    assert size == 80 + raw.nbytes + (sc.nbytes if scaled else 0)
    # a truncated file is refused and leaves no operator behind
    short = tmp_path / "short.btt"
    short.write_bytes(open(path, "rb").read()[: size // 2])
    with pytest.raises(btt.BttError) as e:
        btt.Operator.load(short)
    assert e.value.status == _lib.BTT_ERR_ARG and "truncated" in str(e.value)


def test_injected_allocation_and_launch_failures():
    w = synth.Workload("inj", 20, 4, 33, tau=5.0, seed=2)
    F = synth.blocks(w)
    btt.inject_fault("alloc", 1)
    with pytest.raises(btt.BttError) as e:
        btt.Operator(F, precision="f32")
    assert e.value.status == _lib.BTT_ERR_OOM and "injected" in str(e.value)
    m = torch.from_numpy(synth.vectors(w, "m", 1).astype(np.float32)).cuda()
    with btt.Operator(F, precision="f32") as op:       # the next allocation succeeds
        btt.inject_fault("launch", 2)
        for _ in range(2):
            with pytest.raises(btt.BttError) as e:
                op.matvec(m)
            assert e.value.status == _lib.BTT_ERR_CUDA
        y = op.matvec(m)                               # the operator is still usable
        op.device_status()
    assert direct.rel_l2(y.double().cpu().numpy(), direct.forward(F, m.double().cpu().numpy())) < 1e-5
    btt.inject_fault("none")


def test_fault_injection_from_the_environment():
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import numpy as np, paper_2407_13066_gb300 as btt\n"
            "F = np.random.default_rng(0).standard_normal((8, 2, 3))\n"
            "try:\n    btt.Operator(F)\n    print('created')\n"
            "except btt.BttError as e:\n    print('refused', e.status)\n"
            "btt.Operator(F).close(); print('then created')\n") % ROOT
    out = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, BTT_FAULT="alloc:1"),
                         capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert "refused %d" % _lib.BTT_ERR_OOM in out.stdout and "then created" in out.stdout


@pytest.mark.parametrize("prec,gemm,nrhs", [("f32", "simt", 3), ("bf16", "tensor", 20), ("bf16x2", "tensor", 20),
                                            ("fp8s", "simt", 2)])
def test_results_are_bit_identical_run_to_run(prec, gemm, nrhs):
    """Fixed reduction orders everywhere (no atomics in the products): the
    same call twice gives the same bits."""
    w = synth.Workload("det", 64, 40, 300, tau=12.0, seed=7)
    F = synth.blocks(w)
    m = torch.from_numpy(synth.vectors(w, "m", nrhs).astype(np.float32)).cuda()
    g = torch.from_numpy(synth.noise_gamma_inv(w).astype(np.float32)).cuda()
    with btt.Operator(F, precision=prec, max_nrhs=nrhs, gemm=gemm) as op:
        a = [op.matvec(m), op.adjoint(op.matvec(m)), op.hessian(m, g)]
        b = [op.matvec(m), op.adjoint(op.matvec(m)), op.hessian(m, g)]
        op.device_status()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
