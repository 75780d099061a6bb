#!/usr/bin/env python
"""Benchmark of the FFT-based block-Toeplitz actions on GB300.

One step = one pass of the hot path over the bandwidth workload
(N_t = 1000, N_d = 100, N_m = 10 000; complex64 Fhat of 8.0 GB):
F m, F* d and the Hessian F* Gamma^-1 F m on one vector each, i.e. four
streams of Fhat.  Inputs are generated on the device (seeded generator,
synthetic data of the paper's shape) and resident before timing; Fhat is
far larger than L2, so no flush is needed between steps.

Prints one JSON line: the metric is GB/s of Fhat streamed (the roofline
quantity of the paper's Sec. 4.1), with the dominant kernel's roofline
fraction, an end-to-end figure through the C ABI with host buffers, the
relative l2 error of the whole F, F* and Hessian outputs against the FP64
oracle, clock samples, the FP64 oracle's rate on the host cores, and
(`served`) the metric's second half: a bounded pass of the serving workload
(four resident BF16 operators, continuous batching, p50/p99 latency and
Hessians/s beside the plain FP32 single-vector rate on the same trace).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

METRIC = "F/F* matvec GB/s (% HBM peak) @ rel err 1e-5; served Hessian p50/p99 ms"
GEMV_SRC = os.path.join(ROOT, "paper_2407_13066_gb300", "csrc", "gemv_kernels.cu")

# Single-GPU shape sweeps of Sec. 4.1 (N_t, N_d, N_m):
#   nt  Fig. SingleGPUTimeScalingLine: N_m = 800, N_d = 100, N_t = 1000 .. 10 000
#   nd  Fig. SingleGPUScalingLine: N_t = 2000, N_d = 20 .. 100, N_m = 1000 .. 4000
#   nm  Fig. SingleGPUScaling: N_t = 2000, N_d = 7, N_m = 10^4 .. 6 10^4, continued
#       to operators sized for this GPU's memory (Fhat up to 67 GB)
SWEEPS = {
    "nt": [(nt, 100, 800) for nt in range(1000, 10001, 1000)],
    "nd": [(2000, nd, nm) for nd in (20, 40, 60, 80, 100) for nm in (1000, 2000, 3000, 4000)],
    "nm": [(2000, 7, nm) for nm in (10000, 20000, 30000, 40000, 50000, 60000, 200000, 600000)],
    # time transforms: (N_t, N_d, N_m, precision, vectors, products) over the
    # fixed-plan lengths, FP32 8-vector batches and BF16 64-vector batches
    # on the tensor cores, N_t N_m fixed per set
    "tx": [(nt, 8, 12800000 // nt, "f32", 8, "simt") for nt in (64, 128, 256, 512, 1000, 1024, 2000, 2048, 4000)]
    + [(nt, 16, 6400000 // nt, "bf16", 64, "tensor") for nt in (128, 256, 512, 1000, 1024, 2000, 2048, 4000)],
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="bandwidth")
    p.add_argument("--precision", default=None, choices=["f32", "f16s", "bf16", "bf16x2", "fp8s", "f64"],
                   help="Fhat storage (default f32; bf16 for the multi-rhs workload); f64 runs the FP64 "
                        "instantiation (complex128 Fhat, FP64 vectors and arithmetic: the paper's precision)")
    p.add_argument("--nrhs", type=int, default=None, help="right-hand sides per action (default: the workload's)")
    p.add_argument("--gemm", default="auto", choices=["auto", "simt", "tensor"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--requests", type=int, default=160, help="serving: requests in the trace")
    p.add_argument("--no-check", action="store_true", help="skip the whole-output FP64 oracle check")
    p.add_argument("--split", default="none", choices=["none", "cols"],
                   help="none: an independent operator per GPU; cols: one operator split over the GPUs by "
                        "parameter columns (1 x p layout), all-reduce between the Hessian's passes")
    p.add_argument("--serve-requests", type=int, default=300,
                   help="requests of the served pass after the step (config: four resident operators, "
                        "device vectors); 0 skips it")
    p.add_argument("--cg", action="store_true",
                   help="time the device CG solve of (H + alpha I) x = b on the workload (one JSON line)")
    p.add_argument("--sweep", default=None, choices=sorted(SWEEPS),
                   help="time F and F* over one of the paper's single-GPU shape sweeps (nt, nd, nm), or the "
                        "per-stage times of the time transforms over the fixed-plan lengths (tx); one JSON line per point")
    p.add_argument("--serve-device", action="store_true",
                   help="serving: request vectors live in device memory (clients on the GPU)")
    return p.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons (200 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------- helpers
def combine_ranks(ms, units, device="cpu"):
    """Whole-job timing over the ranks of the default process group (if any):
    the slowest rank's time and the units all ranks processed.  Each rank
    works on its own operator (weak scaling); this is the only exchange."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def ncu_traffic(kernel_key):
    """DRAM bytes per launch recorded from an ncu capture in profiles/, if the
    kernel source is unchanged since (sha256 recorded beside the number).
    kernel_key names the workload, the storage format and the stage
    (e.g. bandwidth/f32/gemv_f): a capture stands only for its own case."""
    src_sha = hashlib.sha256(open(GEMV_SRC, "rb").read()).hexdigest()[:16]
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith((".txt", ".md")):
            continue
        txt = open(os.path.join(pdir, fn)).read()
        m = re.search(r"^traffic_per_launch\[%s\]:\s*([0-9.eE+]+)\s+source_sha256=(\w+)" % re.escape(kernel_key),
                      txt, re.M)
        if m and m.group(2) == src_sha:
            return float(m.group(1))
    return None


def oracle_sample(w, target_s):
    """A bounded sample of the workload for the FP64 oracle (oracle/direct.py,
    as it stands) on the host cores: F on the first n_s time blocks of the
    same operator (N_d, N_m unchanged), n_s doubled until one application
    takes about target_s seconds.  Returns (blocks, m, n_s, seconds)."""
    import synth
    from oracle import direct
    n_s = 8
    while True:
        sub = synth.Workload(w.name, n_s, w.N_d, w.N_m, tau=w.tau, envelope=w.envelope, seed=w.seed)
        F = synth.blocks(sub)
        m = synth.vectors(sub, "m", 1)[0]
        t0 = time.perf_counter()
        direct.forward(F, m)
        dt = time.perf_counter() - t0
        if dt > target_s / 3 or n_s >= w.N_t:
            return F, m, n_s, dt
        n_s = min(w.N_t, n_s * 2)


def oracle_rate(w, n_s, dt):
    """Fhat GB/s equivalent of one oracle F application taking dt seconds on
    n_s time blocks, extrapolated to N_t by the number of (i, j) block pairs
    (the oracle's work is proportional to it)."""
    scale = (w.N_t * (w.N_t + 1) / 2) / (n_s * (n_s + 1) / 2)
    t_full = dt * scale
    sample = ("oracle F (numpy FP64 lag-GEMM) on the first %d of %d time blocks of the %s operator "
              "(N_d=%d, N_m=%d): %.3f s, extrapolated by block pairs x%.1f"
              % (n_s, w.N_t, w.name, w.N_d, w.N_m, dt, scale))
    return w.fhat_bytes(8) / t_full / 1e9, sample


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (x86 'model name', Arm part number)."""
    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    for key in ("model name", "Model"):
        m = re.search(r"^%s\s*:\s*(.+)$" % key, info, re.M)
        if m:
            return m.group(1).strip()
    imp = re.search(r"^CPU implementer\s*:\s*(\S+)", info, re.M)
    part = re.search(r"^CPU part\s*:\s*(\S+)", info, re.M)
    if part:
        return "Arm implementer %s part %s" % (imp.group(1) if imp else "?", part.group(1))
    return "unknown"


_ONE_CORE = r'''
import sys, time
sys.path.insert(0, sys.argv[1])
import synth
from oracle import direct
w = synth.Workload("one-core", int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]), tau=float(sys.argv[5]), seed=0)
F = synth.blocks(w); m = synth.vectors(w, "m", 1)[0]
direct.forward(F, m)
t0 = time.perf_counter(); direct.forward(F, m); print(time.perf_counter() - t0)
'''


def one_core_rate(w, n_s):
    """The same oracle on one core (BLAS and OpenMP pools of one thread, in a
    child process), on the first n_s time blocks."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", _ONE_CORE, ROOT, str(n_s), str(w.N_d), str(w.N_m), str(w.tau)],
                             env=env, capture_output=True, text=True, timeout=300, check=True).stdout
        dt = float(out.strip().splitlines()[-1])
    except Exception as e:  # reported, not fatal: the all-core figure stands
        return {"error": str(e)[:200]}
    gbs, sample = oracle_rate(w, n_s, dt)
    return {"value": gbs, "unit": "GB/s", "cores": 1, "sample": sample}


def cpu_oracle_rate(w, budget_s):
    from oracle import direct
    F, m, n_s, _ = oracle_sample(w, budget_s / 2)
    times = []
    t_end = time.perf_counter() + budget_s / 2
    while not times or time.perf_counter() < t_end:
        t0 = time.perf_counter()
        direct.forward(F, m)
        times.append(time.perf_counter() - t0)
    gbs, sample = oracle_rate(w, n_s, statistics.median(times))
    return {"gbs": gbs, "sample": sample + " (median of %d runs)" % len(times),
            "cores": os.cpu_count(), "cpu_model": cpu_model(),
            "single_core": one_core_rate(w, max(2, n_s // 4))}


# ---------------------------------------------------------------- reference
ENTRY_BYTES = {"f32": 8, "f16s": 4, "bf16": 4, "bf16x2": 8, "fp8s": 2, "f64": 16}


def arm_config(w, prec, nrhs, gemm, world, split=False):
    """The `config` object both arms print for a workload."""
    fb = w.fhat_bytes(ENTRY_BYTES[prec])
    return {
        "workload": "%s: N_t=%d N_d=%d N_m=%d, Fhat %s %.3f GB; step = F m + F* d + "
                    "F* Gamma^-1 F m on %d vector%s (4 Fhat streams)"
                    % (w.name, w.N_t, w.N_d, w.N_m, prec, fb / 1e9, nrhs, "s" if nrhs > 1 else ""),
        "N_t": w.N_t, "N_d": w.N_d, "N_m": w.N_m, "nrhs": nrhs, "precision": prec, "gemm": gemm,
        "l2": "inputs larger than L2 (Fhat %.1f GB), no flush" % (fb / 1e9),
        "parallelism": ("1 x %d parameter-column split (Sec. 3.2), one all-reduce of N_t N_d values per F and "
                        "per Hessian" % world) if split else
                       ("independent operator per GPU" if world > 1 else "single GPU"),
    }


def run_reference(args):
    """The CPU oracle as the comparison arm: each step is a bounded sample of
    the workload (see cpu_oracle_rate), timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    from oracle import direct
    w = synth.WORKLOADS[args.workload]
    # each step: one oracle application on a sample sized so that the whole
    # run stays within about two minutes
    per_step = max(0.2, min(5.0, 120.0 / max(1, args.steps + args.warmup)))
    F, m, n_s, _ = oracle_sample(w, per_step)
    rates = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        direct.forward(F, m)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            rates.append(oracle_rate(w, n_s, dt)[0])
    sample = oracle_rate(w, n_s, dt)[1]
    v = statistics.median(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": arm_config(w, args.precision or ("bf16" if (args.nrhs or w.nrhs) > 1 else "f32"),
                             args.nrhs or w.nrhs, args.gemm, args.gpus),
        "cpu_baseline": {"value": v, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample + " (FP64 oracle; the rate counts the same Fhat bytes as the GPU arm)"},
        "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def oracle_check(w, dev, st, m, d, g, d_out, m_out, h_out, cols=None):
    """Relative l2 over every entry of F m, F* d and F* Gamma^-1 F m (the
    outputs of the last untimed calls) against the FP64 oracle
    (oracle/direct.py as it stands), for every vector of a batch of at most
    4, else vectors 0, 21, 42, 63 (those below the batch size).  The oracle
    reads the seeded blocks one lag at a time, regenerated on the device by
    the input generator."""
    import torch
    import synth
    from oracle import direct
    lib_dev = synth.dev_lib()
    blocks = torch.empty((w.N_t, w.N_d, w.N_m), dtype=torch.float64, device=dev)
    ed, em = synth.envelope(w, "d"), synth.envelope(w, "m")
    ed_t = None if ed is None else torch.from_numpy(ed).to(dev)
    em_t = None if em is None else torch.from_numpy(em).to(dev)
    assert lib_dev.synth_dev_blocks(w.seed, w.N_d, w.N_m, float(w.tau),
                                    None if ed_t is None else ed_t.data_ptr(),
                                    None if em_t is None else em_t.data_ptr(),
                                    0, w.N_t, blocks.data_ptr(), st.cuda_stream) == 0
    torch.cuda.synchronize()
    B = m.shape[0]
    pick = list(range(B)) if B <= 4 else [b for b in (0, 21, 42, 63) if b < B]
    h = lambda x: x[pick].double().cpu().numpy()
    src = lambda k: blocks[k].cpu().numpy()
    t0 = time.perf_counter()
    ref_f = direct.forward(src, h(m), w.N_t)
    ref_a = direct.adjoint(src, h(d), w.N_t)
    ref_h = direct.hessian(src, h(m), g.double().cpu().numpy(), w.N_t)
    dt = time.perf_counter() - t0
    del blocks
    torch.cuda.empty_cache()
    # with the parameter split this rank holds columns [a, b) of F* d and H m
    a, b = cols if cols is not None else (0, w.N_m)
    ref_a, ref_h = ref_a[..., a:b], ref_h[..., a:b]
    return {"F": float(direct.rel_l2(h(d_out), ref_f)), "F*": float(direct.rel_l2(h(m_out), ref_a)),
            "H": float(direct.rel_l2(h(h_out), ref_h)), "vectors": pick,
            "entries": 2 * len(pick) * w.N_t * w.N_m + len(pick) * w.N_t * w.N_d,
            "kind": "whole output vs FP64 oracle (relative l2 over every entry)", "oracle_s": dt}


# ----------------------------------------------------------------- serving
def serving_pass(dev, n_req, device_vectors, loads=(), seed=0):
    """Served Hessian actions (config: 4 resident operators, Poisson arrivals
    of requests with 1..32 vectors drawn uniformly across operators, admitted
    under a 150 GB HBM budget, batched per operator).  The library's
    scheduler batches, computes on the tensor cores (BF16 Fhat) and, for
    host vectors, uploads and downloads.  The trace runs once with every
    request submitted at once (closed loop: the capacity), optionally at
    each fraction in `loads` of that capacity, then at 0.8 x capacity (the
    reported pass, clocks sampled meanwhile).  Compared with the plain FP32
    single-vector Hessian on the same trace.  Returns a dict."""
    import torch
    import paper_2407_13066_gb300 as btt
    from paper_2407_13066_gb300.serve import Server
    import synth

    st = torch.cuda.current_stream(dev)
    lib_dev = synth.dev_lib()
    max_batch, budget = 32, 150e9
    ws = synth.SERVING_OPERATORS

    def make_blocks(w):
        blocks = torch.empty((w.N_t, w.N_d, w.N_m), dtype=torch.float64, device=dev)
        assert lib_dev.synth_dev_blocks(w.seed, w.N_d, w.N_m, float(w.tau), None, None, 0, w.N_t,
                                        blocks.data_ptr(), st.cuda_stream) == 0
        return blocks

    def make_gamma(w):
        g = torch.empty((w.N_t, w.N_d), dtype=torch.float32, device=dev)
        lib_dev.synth_dev_uniform(w.seed, synth.workloads.T_NOISE, 0, g.numel(), 0.5, 2.0, None,
                                  g.data_ptr(), st.cuda_stream)
        return 1.0 / g

    ops, gams = [], []
    for w in ws:
        b = make_blocks(w)
        ops.append(btt.Operator(b, precision="bf16", max_nrhs=max_batch, gemm="tensor", host_staging=0,
                                stream=st.cuda_stream))
        del b
        torch.cuda.empty_cache()
        gams.append(make_gamma(w))
    torch.cuda.synchronize()
    resident = sum(o.operator_bytes() + o.workspace_bytes() for o in ops)
    pool = int(budget - resident)
    assert pool > 0, "operators do not fit the budget"

    # arenas: 32 input vectors and a ring of 48 output vectors per operator
    # (pinned host memory, or device memory for clients on the GPU)
    rng = np.random.default_rng(seed)
    arena_in, arena_out = [], []
    for w in ws:
        x = torch.empty((max_batch, w.N_t, w.N_m), dtype=torch.float32, device=dev)
        lib_dev.synth_dev_normal(w.seed, synth.workloads.T_PARAM, 0, x.numel(), None, x.data_ptr(), st.cuda_stream)
        if device_vectors:
            arena_in.append(x)
            arena_out.append(torch.empty((48, w.N_t, w.N_m), dtype=torch.float32, device=dev))
        else:
            arena_in.append(x.cpu().pin_memory())
            del x
            arena_out.append(torch.empty((48, w.N_t, w.N_m), dtype=torch.float32).pin_memory())
    torch.cuda.synchronize()

    n_req = max(8, n_req)
    req_op = rng.integers(0, len(ws), n_req)
    req_n = rng.integers(1, max_batch + 1, n_req)
    req_k0 = [int(rng.integers(0, max_batch - n + 1)) for n in req_n]

    srv = Server(ops, gamma_inv=gams, pool_bytes=pool, max_batch=max_batch)

    def play(rate):
        """Submits the trace at Poisson arrival times (rate requests/s; None =
        all at once); returns the wall seconds."""
        ring = [[0, []] for _ in ws]           # next offset, outstanding (ticket, start, n)
        gaps = rng.exponential(1.0 / rate, n_req) if rate else np.zeros(n_req)
        t0 = time.perf_counter()
        arrive = t0 + np.cumsum(gaps)
        for i in range(n_req):
            op, n, k0 = int(req_op[i]), int(req_n[i]), req_k0[i]
            now = time.perf_counter()
            if arrive[i] > now:
                time.sleep(arrive[i] - now)
            r = ring[op]
            if r[0] + n > 48:
                r[0] = 0
            # wait for outstanding requests whose outputs overlap [r0, r0 + n)
            keep = []
            for (t, a, m) in r[1]:
                if a < r[0] + n and r[0] < a + m:
                    srv.wait(t)
                else:
                    keep.append((t, a, m))
            r[1] = keep
            t = srv.submit(op, arena_in[op][k0:k0 + n], arena_out[op][r[0]:r[0] + n])
            r[1].append((t, r[0], n))
            r[0] += n
        for r in ring:
            for (t, _, _) in r[1]:
                srv.wait(t)
        return time.perf_counter() - t0

    # closed-loop calibration: the whole trace submitted at once
    play(None)
    cal = srv.stats(reset=True)
    capacity = cal["completed"] / max(cal["span_s"], 1e-9)
    lam = 0.8 * capacity
    sweep = []
    for load in loads:
        play(load * capacity)
        sv = srv.stats(reset=True)
        sweep.append({"load": load, "arrival_rate_per_s": load * capacity, "p50_ms": sv["latency_p50_ms"],
                      "p99_ms": sv["latency_p99_ms"],
                      "hessians_per_s": sv["vectors_completed"] / max(sv["span_s"], 1e-9)})
    sampler = ClockSampler(dev.index or 0)
    sampler.start()
    wall = play(lam)
    clocks = sampler.stop()
    stt = srv.stats(reset=True)
    vectors = int(req_n.sum())
    served_hps = stt["vectors_completed"] / max(stt["span_s"], 1e-9)
    srv.close()

    # accuracy of served results: one vector of the last request per operator
    # on the BF16 tensor-core path against the FP32 path on the same operator
    # (both paths are pinned to the FP64 oracle in the tests); and the FP32
    # single-vector Hessian's latency per operator
    errs, fp32_ms = {}, []
    last = {}
    for i in range(n_req):
        last[int(req_op[i])] = i
    for k, w in enumerate(ws):
        i = last.get(k)
        x = (arena_in[k][req_k0[i]:req_k0[i] + 1] if i is not None else arena_in[k][:1]).to(dev)
        y_bf = ops[k].hessian(x, gams[k])
        ops[k].close()
        b = make_blocks(w)
        o32 = btt.Operator(b, precision="f32", max_nrhs=1, stream=st.cuda_stream)
        del b
        torch.cuda.empty_cache()
        torch.cuda.synchronize()
        y32 = o32.hessian(x, gams[k])
        r32 = y32.double().cpu().numpy()
        errs[w.name] = float(np.linalg.norm(y_bf.double().cpu().numpy() - r32) / np.linalg.norm(r32))
        ts = []
        for _ in range(6):
            a = torch.cuda.Event(enable_timing=True)
            bb = torch.cuda.Event(enable_timing=True)
            a.record(st)
            o32.hessian(x, gams[k], out=y32)
            bb.record(st)
            bb.synchronize()
            ts.append(a.elapsed_time(bb))
        fp32_ms.append(statistics.median(ts[1:]))
        o32.close()
        torch.cuda.synchronize()
    del arena_in, arena_out, gams
    torch.cuda.empty_cache()
    serial_s = sum(int(req_n[i]) * fp32_ms[int(req_op[i])] / 1e3 for i in range(n_req))
    fp32_hps = vectors / serial_s
    return {
        "workload": "serving: 4 resident operators %s, BF16 Fhat on the tensor cores, Poisson arrivals at "
                    "0.8 x measured capacity, requests of 1..32 vectors uniform over operators, 150 GB HBM "
                    "budget (pool %.1f GB after operators and workspaces), max batch %d"
                    % ([(w.N_t, w.N_d, w.N_m) for w in ws], pool / 1e9, max_batch),
        "requests": n_req, "vectors": vectors,
        "request_vectors": "device memory" if device_vectors else "pinned host memory",
        "p50_ms": stt["latency_p50_ms"], "p99_ms": stt["latency_p99_ms"], "mean_ms": stt["latency_mean_ms"],
        "latency_kind": "submit to result on the host, per request (scheduler clock)",
        "hessians_per_s": served_hps,
        "arrival_rate_per_s": lam, "capacity_requests_per_s": capacity,
        "load_sweep": sweep,
        "mean_batch_vectors": stt["mean_batch_vectors"], "batches": stt["batches"],
        "pool_high_water_gb": stt["pool_high_water"] / 1e9,
        "fp32_single_vector": {"hessians_per_s": fp32_hps, "hessian_ms_per_op": fp32_ms,
                               "kind": "serial single-vector FP32 Hessians over the same trace, "
                                       "from measured per-operator latencies"},
        "speedup_vs_fp32_single": served_hps / fp32_hps,
        "rel_err_vs_fp32_path": errs,
        "clocks": clocks,
        "wall_s": wall,
    }


def run_serving(args):
    """The serving workload as its own JSON line (value = p50 latency)."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    r = serving_pass(torch.device("cuda", local), args.requests, args.serve_device, loads=(0.5, 1.0))
    if int(os.environ.get("RANK", "0")) == 0:
        line = {
            "metric": METRIC, "value": r["p50_ms"], "unit": "ms", "n_gpus": 1,
            "steps": r["requests"], "warmup": r["requests"], "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16 storage, f32 accumulate", "data": "synthetic",
            "config": {"workload": r["workload"], "requests": r["requests"], "vectors": r["vectors"],
                       "request_vectors": r["request_vectors"]},
            "latency_ms": {"p50": r["p50_ms"], "p99": r["p99_ms"], "mean": r["mean_ms"], "kind": r["latency_kind"]},
            "served": r,
            "clocks": r["clocks"],
        }
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- ours
def run_sweep(args):
    """One JSON line per shape: device time of one F and one F* matvec on
    one vector (CUDA events over --steps calls each), per-stage split of F,
    and the paper's two normalisations: time per block entry, / (N_t N_d N_m)
    (Fig. SingleGPUTimeScalingLine), and per padded entry, / (2 N_t N_d N_m)
    (Fig. SingleGPUScaling)."""
    import torch

    import paper_2407_13066_gb300 as btt
    import synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    st = torch.cuda.current_stream(dev)
    lib_dev = synth.dev_lib()
    prec = args.precision or "f32"
    peak, peak_kind = measured_peaks()
    steps = max(1, min(args.steps, 100))
    for (N_t, N_d, N_m) in SWEEPS[args.sweep]:
        w = synth.Workload("sweep-" + args.sweep, N_t, N_d, N_m, tau=N_t / 5, seed=N_t + N_d + N_m)
        blocks = torch.empty((N_t, N_d, N_m), dtype=torch.float64, device=dev)
        t0 = time.perf_counter()
        assert lib_dev.synth_dev_blocks(w.seed, N_d, N_m, float(w.tau), None, None, 0, N_t,
                                        blocks.data_ptr(), st.cuda_stream) == 0
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        op = btt.Operator(blocks, precision=prec, max_nrhs=1, stream=st.cuda_stream, gemm=args.gemm)
        torch.cuda.synchronize()
        t_create = time.perf_counter() - t1
        del blocks
        torch.cuda.empty_cache()
        m = torch.empty((1, N_t, N_m), dtype=torch.float32, device=dev)
        d = torch.empty((1, N_t, N_d), dtype=torch.float32, device=dev)
        lib_dev.synth_dev_normal(w.seed, synth.workloads.T_PARAM, 0, m.numel(), None, m.data_ptr(), st.cuda_stream)
        lib_dev.synth_dev_normal(w.seed, synth.workloads.T_DATA, 0, d.numel(), None, d.data_ptr(), st.cuda_stream)
        d_out, m_out = torch.empty_like(d), torch.empty_like(m)

        def timed(fn):
            for _ in range(max(args.warmup, 3)):
                fn()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(st)
            for _ in range(steps):
                fn()
            b.record(st)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / steps

        f_ms = timed(lambda: op.matvec(m, out=d_out))
        a_ms = timed(lambda: op.adjoint(d, out=m_out))
        op.profile(True)
        for _ in range(steps):
            op.matvec(m, out=d_out)
        prof = op.profile_read()
        op.profile(False)
        fb = op.operator_bytes()
        n_el = N_t * N_d * N_m
        print(json.dumps({
            "sweep": args.sweep, "N_t": N_t, "N_d": N_d, "N_m": N_m, "precision": prec,
            "fhat_gb": fb / 1e9, "create_s": t_create, "steps": steps,
            "F_ms": f_ms, "Fadj_ms": a_ms,
            "F_s_per_entry": f_ms / 1e3 / n_el, "Fadj_s_per_entry": a_ms / 1e3 / n_el,
            "F_s_per_padded_entry": f_ms / 1e3 / (2 * n_el),
            "F_fhat_gbs": fb / (f_ms / 1e3) / 1e9, "Fadj_fhat_gbs": fb / (a_ms / 1e3) / 1e9,
            "F_pct_hbm_peak": fb / (f_ms / 1e3) / 1e9 / peak, "peak_gbs": peak, "peak_kind": peak_kind,
            "F_stages_ms": {k: v[0] / steps for k, v in prof.items() if v[1]},
        }), flush=True)
        op.close()
        del m, d, d_out, m_out
        torch.cuda.empty_cache()


def run_tx_sweep(args):
    """One JSON line per shape of SWEEPS["tx"]: the library's per-stage
    device times (btt_profile_*) of one F, one F* and one Hessian call on a
    batch, averaged over --steps calls -- the time transforms (rfft, irfft,
    mid) beside the products."""
    import torch

    import paper_2407_13066_gb300 as btt
    import synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    st = torch.cuda.current_stream(dev)
    lib_dev = synth.dev_lib()
    steps = max(1, min(args.steps, 100))
    for (N_t, N_d, N_m, prec, nb, gemm) in SWEEPS["tx"]:
        w = synth.Workload("sweep-tx", N_t, N_d, N_m, tau=N_t / 5, seed=N_t + N_d + N_m)
        blocks = torch.empty((N_t, N_d, N_m), dtype=torch.float64, device=dev)
        assert lib_dev.synth_dev_blocks(w.seed, N_d, N_m, float(w.tau), None, None, 0, N_t,
                                        blocks.data_ptr(), st.cuda_stream) == 0
        op = btt.Operator(blocks, precision=prec, max_nrhs=nb, stream=st.cuda_stream, gemm=gemm)
        del blocks
        torch.cuda.empty_cache()
        m = torch.empty((nb, N_t, N_m), dtype=torch.float32, device=dev)
        d = torch.empty((nb, N_t, N_d), dtype=torch.float32, device=dev)
        g = torch.empty((N_t, N_d), dtype=torch.float32, device=dev)
        lib_dev.synth_dev_normal(w.seed, synth.workloads.T_PARAM, 0, m.numel(), None, m.data_ptr(), st.cuda_stream)
        lib_dev.synth_dev_normal(w.seed, synth.workloads.T_DATA, 0, d.numel(), None, d.data_ptr(), st.cuda_stream)
        lib_dev.synth_dev_uniform(w.seed, synth.workloads.T_NOISE, 0, g.numel(), 0.5, 2.0, None, g.data_ptr(),
                                  st.cuda_stream)
        d_out, m_out = torch.empty_like(d), torch.empty_like(m)
        line = {"sweep": "tx", "N_t": N_t, "L": 2 * N_t, "N_d": N_d, "N_m": N_m, "precision": prec,
                "nrhs": nb, "gemm": gemm, "steps": steps}
        for name, fn in (("F", lambda: op.matvec(m, out=d_out)), ("F*", lambda: op.adjoint(d, out=m_out)),
                         ("H", lambda: op.hessian(m, g, out=m_out))):
            for _ in range(max(args.warmup, 3)):
                fn()
            torch.cuda.synchronize()
            op.profile(True)
            for _ in range(steps):
                fn()
            prof = op.profile_read()
            op.profile(False)
            line[name + "_stages_ms"] = {k: v[0] / steps for k, v in prof.items() if v[1]}
        print(json.dumps(line), flush=True)
        op.close()
        del m, d, g, d_out, m_out
        torch.cuda.empty_cache()


def run_cg(args):
    """Device CG on (F* Gamma^-1 F + alpha I) x = b (btt_cg): alpha = lambda_max / 50
    (power iteration with the Hessian), tol 1e-5.  Reports iterations, time
    per iteration against one Hessian call, and the true relative residual
    ||b - (H + alpha) x|| / ||b|| recomputed with the Hessian."""
    import torch
    import paper_2407_13066_gb300 as btt
    import synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    st = torch.cuda.current_stream(dev)
    base = synth.WORKLOADS[args.workload]
    nrhs = args.nrhs or 1
    prec = args.precision or "f32"
    w = base
    lib_dev = synth.dev_lib()
    blocks = torch.empty((w.N_t, w.N_d, w.N_m), dtype=torch.float64, device=dev)
    assert lib_dev.synth_dev_blocks(w.seed, w.N_d, w.N_m, float(w.tau), None, None, 0, w.N_t,
                                    blocks.data_ptr(), st.cuda_stream) == 0
    op = btt.Operator(blocks, precision=prec, max_nrhs=nrhs, stream=st.cuda_stream, gemm=args.gemm)
    del blocks
    torch.cuda.empty_cache()
    g = torch.empty((w.N_t, w.N_d), dtype=torch.float32, device=dev)
    lib_dev.synth_dev_uniform(w.seed, synth.workloads.T_NOISE, 0, g.numel(), 0.5, 2.0, None, g.data_ptr(),
                              st.cuda_stream)
    g = 1.0 / g
    b = torch.empty((nrhs, w.N_t, w.N_m), dtype=torch.float32, device=dev)
    lib_dev.synth_dev_normal(w.seed, synth.workloads.T_PARAM, 0, b.numel(), None, b.data_ptr(), st.cuda_stream)
    v = b[:1].clone()
    for _ in range(20):
        v = op.hessian(v, g)
        lam = float(torch.linalg.vector_norm(v.double()))
        v = v / lam
    alpha = lam / 50.0
    h_ms = []
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        op.hessian(b, g)
        e1.record(st)
        e1.synchronize()
        h_ms.append(e0.elapsed_time(e1))
    op.cg(b, alpha, gamma_inv=g, tol=1e-5, max_iter=5)     # warm-up (workspace allocation)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, its, rel = op.cg(b, alpha, gamma_inv=g, tol=1e-5, max_iter=300)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    res = b - (op.hessian(x, g) + alpha * x)
    true_rel = [float(torch.linalg.vector_norm(res[j].double()) / torch.linalg.vector_norm(b[j].double()))
                for j in range(nrhs)]
    # the solve checks convergence every 8 iterations: the last vector's
    # iteration count rounded up to 8 Hessian calls ran, plus the initial one
    k = max(its)
    n_hess = 1 + min(300, (k + 7) // 8 * 8)
    print(json.dumps({
        "cg": args.workload, "N_t": w.N_t, "N_d": w.N_d, "N_m": w.N_m, "nrhs": nrhs, "precision": prec,
        "alpha": alpha, "lambda_max": lam, "iterations": its, "relres_recursive": rel, "relres_true": true_rel,
        "wall_ms": wall * 1e3, "ms_per_iteration": wall * 1e3 / n_hess,
        "hessian_ms": statistics.median(h_ms),
        "overhead_vs_hessian": (wall * 1e3 / n_hess) / statistics.median(h_ms) - 1.0,
    }), flush=True)
    op.close()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.cg:
        return run_cg(args)
    if args.sweep == "tx":
        return run_tx_sweep(args)
    if args.sweep:
        return run_sweep(args)
    if args.workload == "serving":
        return run_serving(args)

    import torch
    import torch.distributed as dist

    import paper_2407_13066_gb300 as btt
    from paper_2407_13066_gb300 import grid
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    base = synth.WORKLOADS[args.workload]
    nrhs = args.nrhs or base.nrhs
    prec = args.precision or ("bf16" if nrhs > 1 else "f32")
    split = args.split == "cols"
    if split and prec == "f64":
        raise SystemExit("--split cols needs an FP32-arithmetic operator (btt_adjoint_weighted has no FP64 form)")
    # replicas: an independent operator per rank (weak scaling over
    # independent problems); cols: one operator split over the ranks by
    # parameter columns (the 1 x p layout of Sec. 3.2; strong scaling)
    w = synth.Workload(base.name, base.N_t, base.N_d, base.N_m, tau=base.tau,
                       envelope=base.envelope, nrhs=nrhs, seed=base.seed + (0 if split else rank))
    N_t, N_d, N_m = w.N_t, w.N_d, w.N_m
    ca, cb = grid.column_slices(N_m, world)[rank] if split else (0, N_m)
    lib_dev = synth.dev_lib()
    st = torch.cuda.current_stream(dev)

    # ---- inputs, generated on the device
    blocks = torch.empty((N_t, N_d, N_m), dtype=torch.float64, device=dev)
    ed, em = synth.envelope(w, "d"), synth.envelope(w, "m")
    ed_t = None if ed is None else torch.from_numpy(ed).to(dev)
    em_t = None if em is None else torch.from_numpy(em).to(dev)
    rc = lib_dev.synth_dev_blocks(w.seed, N_d, N_m, float(w.tau),
                                  None if ed_t is None else ed_t.data_ptr(),
                                  None if em_t is None else em_t.data_ptr(),
                                  0, N_t, blocks.data_ptr(), st.cuda_stream)
    assert rc == 0, rc
    if (ca, cb) != (0, N_m):
        blocks = blocks[:, :, ca:cb].contiguous()
    op = btt.Operator(blocks, precision=prec, max_nrhs=nrhs, stream=st.cuda_stream, gemm=args.gemm)
    del blocks
    torch.cuda.empty_cache()
    torch.cuda.synchronize()
    m = torch.empty((nrhs, N_t, N_m), dtype=torch.float32, device=dev)
    d = torch.empty((nrhs, N_t, N_d), dtype=torch.float32, device=dev)
    g = torch.empty((N_t, N_d), dtype=torch.float32, device=dev)
    lib_dev.synth_dev_normal(w.seed, synth.workloads.T_PARAM, 0, m.numel(), None, m.data_ptr(), st.cuda_stream)
    lib_dev.synth_dev_normal(w.seed, synth.workloads.T_DATA, 0, d.numel(), None, d.data_ptr(), st.cuda_stream)
    lib_dev.synth_dev_uniform(w.seed, synth.workloads.T_NOISE, 0, g.numel(), 0.5, 2.0, None,
                              g.data_ptr(), st.cuda_stream)
    g = 1.0 / g
    if prec == "f64":
        # the FP64 instantiation takes double vectors (the same seeded values)
        m, d, g = m.double(), d.double(), g.double()
    m_full = m
    if (ca, cb) != (0, N_m):
        m = m[:, :, ca:cb].contiguous()
    n_loc = cb - ca
    d_out = torch.empty_like(d)
    m_out = torch.empty_like(m)
    h_out = torch.empty_like(m)
    d_mid = torch.empty_like(d)
    allreduce = (lambda x: dist.all_reduce(x, op=dist.ReduceOp.SUM)) if split and world > 1 else None

    def step():
        if split:
            # F m: partial + all-reduce; F* d: own columns, no exchange;
            # H m: partial, all-reduce, weighted adjoint
            grid.split_forward(op, m, allreduce, out=d_out)
            op.adjoint(d, out=m_out)
            grid.split_hessian(op, m, g, allreduce, out=h_out, work=d_mid)
        else:
            op.matvec(m, out=d_out)
            op.adjoint(d, out=m_out)
            op.hessian(m, g, out=h_out)

    passes_per_step = 4
    fhat_bytes = op.operator_bytes()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # ---- timed region (device)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    op.profile(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = btt.load().btt_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    prof = op.profile_read()
    op.profile(False)
    clocks = sampler.stop()
    # the library's own kernel launches in the timed region
    launches = btt.load().btt_launch_count() - launches0
    ms, total_bytes = combine_ranks(ms, passes_per_step * fhat_bytes * args.steps, device=dev)
    ms_per_step = ms / args.steps
    value = total_bytes / (ms / 1e3) / 1e9

    # per-stage breakdown and the dominant kernel's roofline
    peak, peak_kind = measured_peaks()
    stage_ms = {k: v[0] / args.steps for k, v in prof.items()}
    dom = max(("gemv_f", "gemv_adj"), key=lambda k: prof[k][0])
    # a stage of the tensor-core path is several launches (operand prep,
    # GEMM, reduction); its Fhat bytes are counted once per action
    actions_with_dom = 2 * args.steps
    dom_launch_ms = prof[dom][0] / actions_with_dom
    # the product's minimum traffic: Fhat once, plus its input spectra (FP32
    # complex; BF16 operands on the tensor-core path, hi + lo for the split
    # pair) and its output spectra (FP32 complex; the BF16 tensor-core
    # adjoint writes BF16 pairs)
    # the library's dispatch: tensor cores for BF16 storage (plain or split)
    # when asked, or by default from 16 vectors
    tensor_path = prec in ("bf16", "bf16x2") and (args.gemm == "tensor" or (args.gemm == "auto" and nrhs >= 16))
    b_in = (8 if prec == "bf16x2" else 4) if tensor_path else (16 if prec == "f64" else 8)
    n_in, n_out = (n_loc, N_d) if dom == "gemv_f" else (N_d, n_loc)
    b_out = 4 if (tensor_path and prec == "bf16" and dom == "gemv_adj") else (16 if prec == "f64" else 8)
    spectra_bytes = nrhs * (N_t + 1) * (n_in * b_in + n_out * b_out)
    dom_bytes = fhat_bytes + spectra_bytes
    achieved = dom_bytes / (dom_launch_ms / 1e3) / 1e9
    traffic = ncu_traffic("%s/%s/%s" % (args.workload, prec, dom)) if nrhs == 1 else None

    # each action timed alone (CUDA events around every call, 50 calls):
    # median and p10/p90
    def spread(fn, n=50):
        ts = []
        for _ in range(n):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            b.record(st)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        q = np.percentile(ts, [10, 50, 90])
        return {"p10": float(q[0]), "median": float(q[1]), "p90": float(q[2])}

    actions_ms = {"F": spread(lambda: op.matvec(m, out=d_out)), "F*": spread(lambda: op.adjoint(d, out=m_out)),
                  "H": spread(lambda: op.hessian(m, g, out=h_out)), "calls": 50}
    hess_ms = actions_ms["H"]["median"]

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        hm = torch.empty(tuple(m.shape), dtype=m.dtype).pin_memory()
        hd = torch.empty((nrhs, N_t, N_d), dtype=m.dtype).pin_memory()
        hg = torch.empty((N_t, N_d), dtype=m.dtype).pin_memory()
        hm.copy_(m.cpu())
        hd.copy_(d.cpu())
        hg.copy_(g.cpu())
        hd_out = torch.empty_like(hd).pin_memory()
        hm_out = torch.empty_like(hm).pin_memory()
        hh_out = torch.empty_like(hm).pin_memory()
        sh = st.cuda_stream

        hd_mid = torch.empty_like(hd).pin_memory()

        def host_allreduce(x):
            # NCCL sums device buffers: the partial data goes up and back
            t = x.to(dev, non_blocking=True)
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            x.copy_(t)

        har = host_allreduce if allreduce is not None else None

        def host_step():
            if split:
                grid.split_forward(op, hm, har, out=hd_out)
                op.adjoint(hd, out=hm_out, stream=sh)
                grid.split_hessian(op, hm, hg, har, out=hh_out, work=hd_mid)
            else:
                op.matvec(hm, out=hd_out, stream=sh)
                op.adjoint(hd, out=hm_out, stream=sh)
                op.hessian(hm, hg, out=hh_out, stream=sh)
            torch.cuda.synchronize()   # the step's results are on the host

        for _ in range(2):
            host_step()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        n_e2e = max(3, args.steps // 2)
        for _ in range(n_e2e):
            host_step()
        t_e2e = (time.perf_counter() - t0) / n_e2e
        if world > 1:
            t = torch.tensor([t_e2e], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_e2e = float(t.item())
        eb = hm.element_size()
        h2d = (hm.numel() + hd.numel() + hm.numel() + hg.numel()) * eb
        d2h = (hd_out.numel() + hm_out.numel() + hh_out.numel()) * eb
        e2e = {"value": world * passes_per_step * fhat_bytes / t_e2e / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": t_e2e * 1e3}

    # ---- whole outputs against the FP64 oracle (rank 0, outside the timed region)
    rel_err = None
    if rank == 0 and not args.no_check:
        op.device_status()
        torch.cuda.synchronize()
        rel_err = oracle_check(w, dev, st, m_full, d, g, d_out, m_out, h_out, cols=(ca, cb))

    op.close()
    torch.cuda.empty_cache()

    # ---- served Hessians (config: four resident operators), one GPU
    served = None
    if rank == 0 and world == 1 and args.serve_requests > 0:
        served = serving_pass(dev, args.serve_requests, device_vectors=True)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        r = cpu_oracle_rate(base, args.cpu_seconds)
        cpu = {"value": r["gbs"], "unit": "GB/s", "cores": r["cores"], "kind": "oracle",
               "sample": r["sample"], "cpu_model": r["cpu_model"], "single_core": r["single_core"]}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "GB/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": True,
            "scaling": "strong" if split else "weak",
            "vs_baseline": None,
            "dtype": prec if prec in ("f32", "f64") else prec + " storage, f32 accumulate",
            "data": "synthetic",
            "config": arm_config(w, prec, nrhs, args.gemm, world, split),
            "pct_hbm_peak": value / world / peak,
            "matvecs_per_s": world * 3 * nrhs * args.steps / (ms / 1e3),
            "hessian": {"batch": nrhs, "ms": hess_ms, "matvecs_per_s": world * nrhs / (hess_ms / 1e3)},
            "actions_ms": actions_ms,
            "stages_ms_per_step": stage_ms,
            "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic,
                         "algorithmic_bytes_per_launch": dom_bytes, "fhat_bytes": fhat_bytes,
                         "spectra_bytes": spectra_bytes},
            "rel_err": rel_err,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "served": served,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
