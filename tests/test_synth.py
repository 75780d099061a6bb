"""The seeded input generator: published Philox known answers, the three
builds agreeing, and the distributions the workloads ask for."""
import os

import numpy as np
import pytest

import synth
from synth import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v, 16) for v in line.split()])
    return rows


@pytest.mark.parametrize("row", _kat())
def test_philox_numpy_known_answers(row):
    out = philox.philox4x32_10(*row[:6])
    assert [int(v) for v in out] == row[6:]


@pytest.mark.parametrize("row", _kat())
def test_philox_c_known_answers(row):
    import ctypes
    buf = (ctypes.c_uint32 * 4)()
    synth.host_lib().synth_host_philox(*row[:6], buf)
    assert list(buf) == row[6:]


def test_host_build_matches_numpy():
    e = np.arange(0, 4096, dtype=np.uint64) * np.uint64(7919) + np.uint64(12345)
    ref = philox.normal(3, 1, e)
    got = np.array([synth.normals(3, 1, 1, start=int(i))[0] for i in e[:64]])
    np.testing.assert_allclose(got, ref[:64], rtol=1e-14, atol=1e-15)
    u = philox.uniform(5, 3, np.arange(1000, dtype=np.uint64))
    np.testing.assert_allclose(synth.uniforms(5, 3, 1000), u, rtol=1e-15, atol=0)


def test_blocks_match_entries_and_numpy():
    w = synth.WORKLOADS["precision"]
    small = synth.Workload("t", 5, 6, 7, tau=3.0, envelope=True, seed=2)
    F = synth.blocks(small)
    k, s, l = np.meshgrid(np.arange(5), np.arange(6), np.arange(7), indexing="ij")
    ref = philox.block_entries(2, 6, 7, 3.0, synth.envelope(small, "d"), synth.envelope(small, "m"), k, s, l)
    np.testing.assert_allclose(F, ref, rtol=1e-14, atol=1e-300)
    np.testing.assert_array_equal(synth.block_entries(small, k, s, l), F)
    # entries of a large workload are drawn on their own
    ks, ss, ls = np.array([0, 511, 100]), np.array([0, 599, 7]), np.array([19999, 0, 123])
    got = synth.block_entries(w, ks, ss, ls)
    ref = philox.block_entries(0, 600, 20000, 0.0, synth.envelope(w, "d"), synth.envelope(w, "m"), ks, ss, ls)
    np.testing.assert_allclose(got, ref, rtol=1e-14)


def test_distributions():
    z = synth.normals(0, 1, 400000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    assert abs(np.mean(z ** 4) - 3) < 0.05
    u = synth.uniforms(0, 3, 100000, 0.5, 2.0)
    assert u.min() >= 0.5 and u.max() <= 2.0 and abs(u.mean() - 1.25) < 0.01
    w = synth.WORKLOADS["precision"]
    for side in "dm":
        e = synth.envelope(w, side)
        assert e.min() >= 0.1 - 1e-12 and e.max() <= 1.0 + 1e-12
        # smooth: neighbouring values differ by far less than the range
        assert np.abs(np.diff(e)).max() < 0.1
    g = synth.noise_gamma_inv(synth.WORKLOADS["bandwidth"])
    assert g.shape == (1000, 100) and g.min() >= 0.5 - 1e-12 and g.max() <= 2.0 + 1e-12


def test_decay():
    w = synth.WORKLOADS["bandwidth"]
    F = synth.blocks(synth.Workload("b", 400, 4, 300, tau=200.0), 0, 400)
    r = F[300:].std() / F[:100].std()
    assert 0.2 < r < 0.45  # exp(-300/200 .. ) over exp(0 .. 100/200)
