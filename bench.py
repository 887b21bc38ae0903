#!/usr/bin/env python
"""Throughput of the CountGauss transform T.X = G.(S.X) on GB300.

One step = one cg_apply_csr call on the largest workload, the precision ladder's input
(n = 2^26 rows, d = 128, Bernoulli density 0.01, N(0,1) values, m = 128, B = 2^18,
seed 3), in FP32: the CountSketch scatter, the in-kernel Gaussian contraction and its
split-K sum.  Inputs are resident in HBM when the timed region starts; the CSR arrays
(~956 MB) exceed L2, so no flush is needed between steps.

Printed JSON line (rank 0):
  value          nnz(X)/s over all ranks (weak scaling: every rank sketches its own
                 shard of n rows, global row offset rank*n; the m x d outputs are
                 summed across ranks each step).  The timed loop records no per-kernel
                 events; the stage times come from a second loop of the same steps
                 (stage_pass)
  roofline       the scatter (dominant; at this size the deferred pair of kernels):
                 algorithmic bytes per launch (8 nnz + 4 (n+1) + 4 B d) over its
                 CUDA-event duration in the stage pass, against the measured HBM copy
                 bandwidth; traffic from one ncu capture of the same launch
  plain          the plain G~.X on the same input and GPU, and the speedup over it
  e2e            the same metric through cg_apply_csr_host: the CSR in pinned host memory
                 copied host->device in chunks that overlap the scatter, Y read back
                 every step, through the same public call; copied_ms and direct_ms time
                 the chunked copies and the scatter reading host memory in place
  cpu_baseline   the FP64 oracle on this machine's host cores (rank 0, N = 1): all cores
                 (row shards and ranges of G's columns in host threads) and one core
  rows           (N = 1) the other workloads, each a row of its own: the NMF-like input
                 (n = 2^24, d = 64), the precision ladder, dense forward and adjoint, the
                 96-instance batch, the small case's latency, the SVM projection, and
                 int64 row offsets (--rows)

--impl reference times that oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "ladder_n64M_d128"
METRIC = "CountGauss nnz(X)/s & HBM-roofline %; speedup vs plain G̃·X, same GB300"
UNIT = "nnz/s"

# dram bytes (read + write) per launch of the scatter kernel(s) from one ncu capture of the
# workload named, keyed by the sha256 of the kernel sources it was taken on (null once a
# source changes).  nmf_n16M_d64: 536.78 MB read + 3.30 MB written, captured at full size.
# ladder_n64M_d128 (the deferred pair, both kernels): pass 1 1221.1 MB read + 575.8 MB
# written, replay 316.9 MB read + 0.1 MB written, captured at full size.
NCU_TRAFFIC = {("6386e39308a65745", "nmf_n16M_d64"): 540_079_104,
               ("56bebdf2e825e2eb", "ladder_n64M_d128"): 2_113_923_072}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--scatter", choices=["auto", "atomic", "partition", "deferred", "binned"], default="auto")
    ap.add_argument("--precision", choices=["fp32", "bf16", "bf16x3", "fp8", "fp8x3"], default="fp32",
                    help="arithmetic of the Gaussian contraction in the timed step (the scatter is fp32)")
    ap.add_argument("--scatter-passes", type=int, default=0, help="bucket-range passes of the scatter (0: automatic)")
    ap.add_argument("--scatter-rows", type=int, default=0, choices=[0, 1, 32, 64, 128],
                    help="CSR rows per warp chunk of the scatter (0: automatic)")
    ap.add_argument("--host-chunk", type=int, default=0,
                    help="nonzeros per chunk of the end-to-end host-input call (0: automatic)")
    ap.add_argument("--reduction-sweep", action="store_true",
                    help="instead of the step: random fp32 reduction rate vs array size (the scatter's ceiling)")
    ap.add_argument("--sweep-mb", default="8,16,32,48,64,80,96,112,128,134,160,192,256",
                    help="array sizes (MB) of --reduction-sweep")
    ap.add_argument("--sweep-count", type=int, default=50_000_000, help="reductions per call of --reduction-sweep")
    ap.add_argument("--kl-sweep", action="store_true",
                    help="instead of the step: Theorem 1's KL / Pinsker bound and Lemma 5's distinguisher vs B")
    ap.add_argument("--no-rows", action="store_true", help="skip the other hot-path rows (ladder, adjoint, batch)")
    ap.add_argument("--step-only", action="store_true",
                    help="time the step alone (no plain product, deterministic mode or host-input call): for profiling")
    ap.add_argument("--rows", default="nmf,ladder,grad,batch,small,svm,wide",
                    help="comma list of the other rows to measure (nmf, ladder, grad, batch, small, svm, wide)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """SM clock and clock-event (throttle) reasons, read through NVML every 2 ms by a
    background thread while the timed region runs (read-only queries)."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device):
        self.dev = torch_device
        self.samples = []
        self.reasons = 0
        self.max_mhz = None
        self.error = None
        self._stop = None
        self._thread = None

    def _open(self):
        import ctypes
        import torch
        nvml = ctypes.CDLL("libnvidia-ml.so.1")
        if nvml.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = ctypes.c_void_p()
        props = torch.cuda.get_device_properties(self.dev)
        bus = None
        if all(hasattr(props, a) for a in ("pci_domain_id", "pci_bus_id", "pci_device_id")):
            bus = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0".encode()
        if bus is None or nvml.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(h)) != 0:
            if nvml.nvmlDeviceGetHandleByIndex_v2(self.dev.index or 0, ctypes.byref(h)) != 0:
                raise RuntimeError("no NVML handle")
        c = ctypes.c_uint()
        if nvml.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(c)) == 0:
            self.max_mhz = float(c.value)
        get_reasons = getattr(nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(nvml, "nvmlDeviceGetCurrentClocksThrottleReasons")
        return nvml, h, get_reasons

    def __enter__(self):
        import ctypes
        import threading
        try:
            nvml, h, get_reasons = self._open()
        except Exception as e:  # noqa: BLE001
            self.error = f"nvml unavailable: {e}"
            return self
        self._stop = threading.Event()

        def poll():
            c = ctypes.c_uint()
            r = ctypes.c_ulonglong()
            while not self._stop.is_set():
                if nvml.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(c)) == 0:
                    self.samples.append(float(c.value))
                if get_reasons(h, ctypes.byref(r)) == 0:
                    self.reasons |= int(r.value)
                time.sleep(0.002)

        self._thread = threading.Thread(target=poll, daemon=True)
        self._thread.start()
        return self

    def __exit__(self, *exc):
        if self._thread is not None:
            self._stop.set()
            self._thread.join(timeout=5)

    def summary(self):
        if self.error:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [self.error]}
        names = [v for k, v in self.REASONS.items() if self.reasons & k]
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None, "sm_max_mhz": self.max_mhz,
                "reasons": names, "samples": len(self.samples)}


def source_hash(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1606_05732_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ------------------------------------------------------------------------------------
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # not on Linux
        return os.cpu_count() or 1


def oracle_fraction_step(X, w, frac, threads):
    """One oracle apply on a fraction `frac` of the workload: the sketch of the first
    frac*n rows and the contraction over the first frac*B columns of G (so both stages
    do `frac` of the whole job's work), on `threads` host threads.  Returns (seconds,
    nonzeros of the sampled rows)."""
    import oracle
    ns = max(1, int(X.n * frac))
    k1 = int(X.row_ptr[ns])
    b1 = max(1, int(w["B"] * frac))
    t0 = time.perf_counter()
    oracle.apply_csr_parallel(w["seed"], ns, X.d, w["m"], w["B"], X.row_ptr[:ns + 1], X.col_idx[:k1],
                              X.vals[:k1], threads, b_range=(0, b1))
    return time.perf_counter() - t0, k1


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    from paper_1606_05732_gb300 import synth
    X, w = synth.workload_csr(args.workload)
    cores = host_cores()
    # the fraction of the workload per step: at most 1/16, and small enough that the
    # whole run (warm-up and timed steps) takes about two minutes on these cores
    frac = 1.0 / 64
    dt, _ = oracle_fraction_step(X, w, frac, cores)
    frac = min(1.0 / 16, frac * max(0.05, 120.0 / max(1, args.steps + args.warmup) / max(dt, 1e-3)))
    times, nnzs = [], []
    for it in range(args.warmup + args.steps):
        dt, k1 = oracle_fraction_step(X, w, frac, cores)
        if it >= args.warmup:
            times.append(dt)
            nnzs.append(k1)
    step = statistics.mean(times)
    value = statistics.mean(nnzs) / step
    sample = (f"per step {frac:.5f} of {args.workload} (n={X.n}, nnz={X.nnz}, m={w['m']}, B={w['B']}): the FP64 "
              f"oracle's sketch of the first {frac:.5f} n rows and its contraction over the first {frac:.5f} B "
              f"columns of G, on {cores} host threads (row shards, ranges of G's columns)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": X.n, "d": X.d, "nnz": X.nnz, "m": w["m"], "B": w["B"],
                   "fraction_per_step": frac},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baselines(X, w):
    """The FP64 oracle on this machine's host cores, the whole workload once on all cores
    (row shards and ranges of G's columns in host threads, summed) and once on one core
    (if that takes under about two minutes: else on a fraction of the rows and of G's
    columns, which scales both stages alike)."""
    import oracle

    from paper_1606_05732_gb300 import synth
    oracle.build()
    cores = host_cores()
    t0 = time.perf_counter()
    oracle.apply_csr_parallel(w["seed"], X.n, X.d, w["m"], w["B"], X.row_ptr, X.col_idx, X.vals, cores)
    t_all = time.perf_counter() - t0
    est_one = t_all * cores
    frac = 1.0 if est_one < 120 else 0.25
    dt, k1 = oracle_fraction_step(X, w, frac, 1)
    # the plain product on a sample of its output rows: row r of G~.X needs row r of G~
    # only, so the time of all m rows is the sample's times m / rows (extrapolated)
    rows = synth.sample_rows(w["m"], w["seed"], 2)
    t0 = time.perf_counter()
    oracle.plain_csr(w["seed"], X.n, X.d, w["m"], X.row_ptr, X.col_idx, X.vals, rows=rows)
    tp = (time.perf_counter() - t0) * w["m"] / rows.size
    return {"value": X.nnz / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the whole workload (n={X.n}, nnz={X.nnz}), FP64, {cores} host threads, {t_all:.2f} s",
            "one_core": {"value": k1 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": ("the whole workload" if frac == 1.0 else f"{frac} of the rows and of the columns of G")
                         + f", FP64, one thread, {dt:.2f} s"},
            "plain_one_core": {"value": X.nnz / tp, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "extrapolated": True,
                               "sample": f"rows {rows.tolist()} of the plain product G~.X, FP64, one thread, "
                                         f"{tp * rows.size / w['m']:.2f} s, scaled to all {w['m']} rows"}}


# ------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------
def _time_calls(fn, reps, stream, warm=2):
    """Mean ms per call of fn over `reps` calls, CUDA events on `stream`."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _time_each(fn, reps, stream, warm=2):
    """Per-call ms of fn over `reps` calls (CUDA events on `stream` around each call, which
    must synchronise before it returns): (median, mean)."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts), sum(ts) / len(ts)


def reduction_ceiling(dev, count, cells, reps=5):
    """Random fp32 reductions per second on this GPU: cg_diag_random_reductions adds 1.0
    at `count` hashed positions of a `cells`-float array (the SX size) with the scatter
    kernel's grid, no loads -- one reduction per nonzero is all the scatter must issue,
    so this rate bounds it from above the way the copy bandwidth bounds a stream."""
    import torch

    from paper_1606_05732_gb300 import countgauss
    acc = torch.zeros(cells, device=dev)
    stream = torch.cuda.current_stream(dev)
    ms = _time_calls(lambda: countgauss.diag_random_reductions(acc, count), reps, stream)
    del acc
    return {"per_s": count / (ms / 1e3), "ms": ms, "count": count, "array_bytes": 4 * cells,
            "how": "cg_diag_random_reductions: count fp32 adds at hashed positions of an SX-sized array"}


def measure_rows(dev, reps, which=("ladder", "grad", "batch", "small", "svm", "wide")):
    """The other rows of the hot path, each on its own workload (sizes in synth.WORKLOADS):
    precision ladder and plain product on the largest workload, dense forward and
    adjoint, the 96-instance batch, deterministic mode, the small case's latency, the
    right projection of the SVM application on the largest TechTC-shaped pair, and the
    64-bit row offsets entry point (past 2^31 nonzeros)."""
    import numpy as np
    import torch

    stream = torch.cuda.current_stream(dev)
    rows = {}

    def csr_dev(X):
        return (torch.from_numpy(X.row_ptr.astype(np.int32)).to(dev), torch.from_numpy(X.col_idx).to(dev),
                torch.from_numpy(X.vals).to(dev))

    if "ladder" in which:
        rows.update(_ladder_row(dev, reps, csr_dev, stream))
    if "grad" in which:
        rows.update(_grad_row(dev, reps, csr_dev, stream))
    if "batch" in which:
        rows.update(_batch_row(dev, reps, csr_dev, stream))
    if "small" in which:
        rows.update(_small_row(dev, reps, csr_dev, stream))
    if "svm" in which:
        rows.update(_svm_row(dev, reps, csr_dev, stream))
    if "wide" in which:
        rows.update(_wide_row(dev, reps, csr_dev, stream))
    return rows


def _wide_row(dev, reps, csr_dev, stream):
    """cg_apply_csr_i64: on the headline input with its row offsets widened to int64
    (against the int32 call), and on a 2^25 x 64 matrix of about 2.4e9 nonzeros (19 GB
    of CSR drawn on the device), which 32-bit offsets cannot index."""
    import torch

    from paper_1606_05732_gb300 import countgauss, synth
    rows = {}
    X, w = synth.workload_csr("nmf_n16M_d64")
    rp, ci, v = csr_dev(X)
    rp64 = rp.long()
    plan = countgauss.CountGauss(X.n, X.d, w["m"], w["B"], w["seed"])
    Y = torch.empty(w["m"], w["d"], dtype=torch.float32, device=dev)
    ms32 = _time_calls(lambda: plan.apply_csr(rp, ci, v, out=Y), reps, stream)
    ms64 = _time_calls(lambda: plan.apply_csr(rp64, ci, v, out=Y), reps, stream)
    plan.check()
    rows["wide_offsets_nmf_n16M_d64"] = {"int32_ms": ms32, "int64_ms": ms64, "nnz": X.nnz}
    del rp, ci, v, rp64, X
    n, d, m, B, seed = 1 << 25, 64, 32, 1 << 17, 37
    rp, ci, v = synth.wide_csr_device(n, d, 72, seed, device=dev)
    nnz = ci.numel()
    plan = countgauss.CountGauss(n, d, m, B, seed)
    Y = torch.empty(m, d, dtype=torch.float32, device=dev)
    ms = _time_calls(lambda: plan.apply_csr(rp, ci, v, out=Y), max(3, reps // 20), stream)
    plan.check()
    rows["wide_n32M_d64_2.4G_nnz"] = {"nnz": nnz, "ms_per_call": ms, "nnz_per_s": nnz / (ms / 1e3),
                                      "csr_bytes": 8 * nnz + 8 * (n + 1)}
    del rp, ci, v
    torch.cuda.empty_cache()
    return rows


def _ladder_row(dev, reps, csr_dev, stream):
    """Every precision of the contraction, and the plain product, at the largest workload."""
    import torch

    from paper_1606_05732_gb300 import _lib, countgauss, synth
    rows = {}
    X, w = synth.workload_csr("ladder_n64M_d128")
    rp, ci, v = csr_dev(X)
    ladder = {}
    for prec in ["fp32", "bf16x3", "bf16", "fp8x3", "fp8"]:
        plan = countgauss.CountGauss(X.n, X.d, w["m"], w["B"], w["seed"], precision=prec)
        Y = torch.empty(w["m"], w["d"], dtype=torch.float32, device=dev)
        plan.apply_csr(rp, ci, v, out=Y)
        ms = _time_calls(lambda: plan.apply_csr(rp, ci, v, out=Y), reps, stream)
        # the contraction kernel alone: event pairs around it, in calls of their own
        plan.enable_timing(True)
        plan.kernel_time(_lib.KERNEL_CONTRACT)
        _time_calls(lambda: plan.apply_csr(rp, ci, v, out=Y), reps, stream, warm=0)
        cms, cn = plan.kernel_time(_lib.KERNEL_CONTRACT)
        plan.enable_timing(False)
        plan.check()
        flops = 2.0 * w["m"] * w["B"] * w["d"]
        ladder[prec] = {"ms_per_call": ms, "nnz_per_s": X.nnz / (ms / 1e3), "contract_kernel_ms": cms / max(1, cn),
                        "contract_tflops": flops / (cms / max(1, cn) / 1e3) / 1e12}
    plan = countgauss.CountGauss(X.n, X.d, w["m"], w["B"], w["seed"])
    Yp = torch.empty(w["m"], w["d"], dtype=torch.float32, device=dev)
    plain_ms = _time_calls(lambda: plan.plain_csr(rp, ci, v, out=Yp), max(2, reps // 4), stream, warm=1)
    rows["ladder_n64M_d128"] = {"nnz": X.nnz, "m": w["m"], "B": w["B"], "d": w["d"], "precisions": ladder,
                                "plain_ms": plain_ms,
                                "speedup_fp32_over_plain": plain_ms / ladder["fp32"]["ms_per_call"]}
    del rp, ci, v, X
    return rows


def _grad_row(dev, reps, csr_dev, stream):
    """Dense forward and adjoint (dense, and at the stored entries of the p = 0.02 variant)."""
    import torch

    from paper_1606_05732_gb300 import countgauss, synth
    rows = {}
    w = synth.WORKLOADS["grad_n1M_d64"]
    Xd = torch.from_numpy(synth.dense_normal(w["n"], w["d"], seed=w["seed"])).to(dev)
    Xs = synth.csr_bernoulli(w["n"], w["d"], w["p"], seed=w["seed"])
    rp, ci, v = csr_dev(Xs)
    from paper_1606_05732_gb300 import _lib
    plan = countgauss.CountGauss(w["n"], w["d"], w["m"], w["B"], w["seed"])
    dY = torch.randn(w["m"], w["d"], device=dev)
    plan.apply_dense(Xd)
    plan.adjoint(dY)
    plan.enable_timing(True)
    for k in (_lib.KERNEL_SKETCH, _lib.KERNEL_GATHER):
        plan.kernel_time(k)
    fwd = _time_calls(lambda: plan.apply_dense(Xd), reps, stream)
    sk_ms, sk_n = plan.kernel_time(_lib.KERNEL_SKETCH)
    bwd = _time_calls(lambda: plan.adjoint(dY), reps, stream)
    ga_ms, ga_n = plan.kernel_time(_lib.KERNEL_GATHER)
    plan.enable_timing(False)
    bwd_s = _time_calls(lambda: plan.adjoint(dY, rp, ci), reps, stream)
    dense_bytes = 4 * w["n"] * w["d"]
    sk = sk_ms / max(1, sk_n)
    ga = ga_ms / max(1, ga_n)
    rows["grad_n1M_d64"] = {"apply_dense_ms": fwd, "adjoint_dense_ms": bwd, "adjoint_csr_ms": bwd_s,
                            "adjoint_csr_nnz": Xs.nnz,
                            # the dense scatter and the dense gather kernels alone (CUDA events)
                            "dense_scatter_kernel_ms": sk, "dense_scatter_gbs": (dense_bytes + 4 * w["B"] * w["d"]) / sk / 1e6,
                            "dense_gather_kernel_ms": ga, "dense_gather_gbs": (dense_bytes + 4 * w["B"] * w["d"]) / ga / 1e6}
    del Xd, rp, ci, v
    return rows


def _batch_row(dev, reps, csr_dev, stream):
    """The 96-instance batch, autotuned, replayed from a CUDA graph."""
    from paper_1606_05732_gb300 import _lib, countgauss, synth
    rows = {}
    params = synth.batch_instances()
    Xs = synth.batch_inputs(params)
    insts = []
    for t, Xb in zip(params, Xs):
        rpb, cib, vb = csr_dev(Xb)
        insts.append(dict(n=t.n, d=t.d, m=t.m, B=t.B, seed=t.seed, row_ptr=rpb, col_idx=cib, vals=vb))
    batch = countgauss.CountGaussBatch(insts)
    batch.autotune(reps=2)
    bms = _time_calls(batch.apply, reps, stream)
    batch.check()
    tot = sum(X.nnz for X in Xs)
    rows["batch96"] = {"ms_per_batch": bms, "nnz_total": tot, "nnz_per_s": tot / (bms / 1e3),
                       "tuning": {"scatter_nnz": batch.get_option(_lib.BATCH_OPT_SCATTER_NNZ),
                                  "contract_fma": batch.get_option(_lib.BATCH_OPT_CONTRACT_FMA),
                                  "ctas_per_sm": batch.get_option(_lib.BATCH_OPT_CTAS_PER_SM)}}
    del insts, batch
    return rows


def _graph_us(fn, reps, dev, per_graph=10):
    """Device time per call of fn (us): `per_graph` calls captured once in a CUDA graph and
    replayed, so that the Python call overhead is not in the measurement."""
    import torch
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(2):
            fn()
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(per_graph):
            fn()
    ms = _time_calls(g.replay, reps, torch.cuda.current_stream(dev))
    del g
    return 1e3 * ms / per_graph


def _small_row(dev, reps, csr_dev, stream):
    """Latency of the small case, CountGauss and plain: device time per call (calls
    replayed from a CUDA graph) and the time of a call from Python."""
    import torch

    from paper_1606_05732_gb300 import countgauss, synth
    rows = {}
    X, w = synth.workload_csr("small_n65536_d16")
    rp, ci, v = csr_dev(X)
    plan = countgauss.CountGauss(X.n, X.d, w["m"], w["B"], w["seed"])
    Y = torch.empty(w["m"], w["d"], dtype=torch.float32, device=dev)
    Yp = torch.empty_like(Y)
    rows["small_n65536_d16"] = {
        "apply_csr_us": _graph_us(lambda: plan.apply_csr(rp, ci, v, out=Y), reps, dev),
        "plain_us": _graph_us(lambda: plan.plain_csr(rp, ci, v, out=Yp), reps, dev),
        "apply_csr_python_call_us": 1e3 * _time_calls(lambda: plan.apply_csr(rp, ci, v, out=Y), reps, stream),
        "plain_python_call_us": 1e3 * _time_calls(lambda: plan.plain_csr(rp, ci, v, out=Yp), reps, stream)}
    plan.check()
    return rows


def _svm_row(dev, reps, csr_dev, stream):
    """The random projection X.R, R = T^T, of the SVM application (Section 9; Table 1
    times it) on the largest TechTC-shaped pair (280 documents x 40,000 words, density
    1e-2), for m = 128, 256, 512 with B = 5m: device time per projection (calls replayed
    from a CUDA graph) in FP32 and BF16, the time of a call from Python, and end to end
    from pinned host memory (CSR copied in, Z copied out, synchronised).  The plain
    product G~.A^T on the same matrix for comparison (the paper's "RG" column)."""
    import numpy as np
    import torch

    from paper_1606_05732_gb300 import countgauss, synth
    A = synth.techtc_pair(21, docs=280, words=40_000)
    At = synth.csr_from_dense(A.to_dense().T)
    rp, ci, v = csr_dev(A)
    rpt, cit, vt = csr_dev(At)
    host = [torch.from_numpy(a).pin_memory() for a in (A.row_ptr.astype(np.int32), A.col_idx, A.vals)]
    dbuf = [torch.empty_like(h, device=dev) for h in host]
    per_m = {}
    for m in (128, 256, 512):
        B = 5 * m
        plan = countgauss.CountGauss(A.d, A.n, m, B, 21)
        plan_bf = countgauss.CountGauss(A.d, A.n, m, B, 21, precision="bf16")
        Z = torch.empty(A.n, m, dtype=torch.float32, device=dev)
        Zh = torch.empty(A.n, m, dtype=torch.float32).pin_memory()

        def e2e():
            for h, dv in zip(host, dbuf):
                dv.copy_(h, non_blocking=True)
            plan.apply_right_csr(*dbuf, out=Z)
            Zh.copy_(Z, non_blocking=True)
            torch.cuda.current_stream(dev).synchronize()

        r = {"B": B,
             "fp32_us": _graph_us(lambda: plan.apply_right_csr(rp, ci, v, out=Z), reps, dev),
             "bf16_us": _graph_us(lambda: plan_bf.apply_right_csr(rp, ci, v, out=Z), reps, dev),
             "python_call_us": 1e3 * _time_calls(lambda: plan.apply_right_csr(rp, ci, v, out=Z), reps, stream),
             "e2e_host_us": 1e3 * _time_calls(e2e, reps, stream)}
        Yp = torch.empty(m, A.n, dtype=torch.float32, device=dev)
        r["plain_us"] = _graph_us(lambda: plan.plain_csr(rpt, cit, vt, out=Yp), reps, dev)
        plan.check()
        plan_bf.check()
        per_m[str(m)] = r
    return {"svm_techtc_w40000_d280": {"docs": A.n, "words": A.d, "nnz": A.nnz, "density": 0.01,
                                       "per_m": per_m,
                                       "input": "synthetic TechTC-shaped pair (shape stand-in, not the dataset)"}}


def scatter_kernels(args, B, d, dev):
    """Names and sources of the scatter kernels cg_apply_csr runs for this plan: the
    deferred pair once SX exceeds 60 % of the L2 (automatic), else the one-pass kernel."""
    import torch
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    if args.scatter == "partition":
        return "partition_kernel+accumulate_kernel", ("cg_sketch_part.cu", "cg_rng.cuh"), 5
    if args.scatter == "binned":
        return "bin_pass_kernel+bin_reduce_kernel", ("cg_sketch_bin.cu", "cg_scatter.cuh", "cg_rng.cuh"), 5
    if args.scatter == "deferred" or (args.scatter == "auto" and args.scatter_passes == 0
                                      and 4 * B * d > 0.6 * l2 and B * d < (1 << 32)):
        return "split_pass_staged_kernel+replay_records_kernel", ("cg_sketch_defer.cu", "cg_scatter.cuh", "cg_rng.cuh"), 4
    return "sketch_csr_kernel", ("cg_sketch.cu", "cg_scatter.cuh", "cg_rng.cuh"), 3


def measure_workload(args, name, dev, rank=0, world=1, pg=None, steps=None, e2e=True, det=True, plain=True):
    """One workload's step: cg_apply_csr timed over `steps` calls with CUDA events (no
    per-kernel events inside), then the same calls again with per-kernel event pairs
    (the stage pass), the plain product, the deterministic mode, and (e2e) the
    host-input call.  Returns (record, X, workload dict)."""
    import numpy as np
    import torch

    from paper_1606_05732_gb300 import _lib, countgauss, synth
    steps = args.steps if steps is None else steps
    wl = dict(synth.WORKLOADS[name])
    n, d, m, B, seed = wl["n"], wl["d"], wl["m"], wl["B"], wl["seed"]
    X = synth.csr_bernoulli(n, d, wl["p"], seed=seed + 7919 * rank, values=wl["values"])
    nnz = X.nnz
    rp_h = torch.from_numpy(X.row_ptr.astype(np.int32)).pin_memory()
    ci_h = torch.from_numpy(X.col_idx).pin_memory()
    v_h = torch.from_numpy(X.vals).pin_memory()
    rp, ci, v = rp_h.to(dev), ci_h.to(dev), v_h.to(dev)
    plan = countgauss.CountGauss(n, d, m, B, seed, row_offset=rank * n, scatter=args.scatter, precision=args.precision,
                                 scatter_passes=args.scatter_passes, scatter_rows=args.scatter_rows)
    kname, ksrc, launches_per_step = scatter_kernels(args, B, d, dev)
    Y = torch.empty(m, d, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.apply_csr(rp, ci, v, out=Y)
        if pg is not None:
            pg.all_reduce(Y)

    for _ in range(args.warmup):
        step()
    plan.check()

    def timed(label):
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev) as clk:
            e0.record(stream)
            for _ in range(steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize(dev)
        if pg is not None:
            pg.barrier()
        ms = e0.elapsed_time(e1)
        if pg is not None:
            t = torch.tensor([ms], device=dev, dtype=torch.float64)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            ms = float(t.item())
        return ms / steps, clk.summary()

    ms_step, clocks = timed("headline")
    # the stage pass: the same steps with an event pair around every kernel
    plan.enable_timing(True)
    plan.kernel_time(_lib.KERNEL_SKETCH)
    plan.kernel_time(_lib.KERNEL_CONTRACT)
    stage_ms_step, _ = timed("stages")
    sketch_ms, sketch_n = plan.kernel_time(_lib.KERNEL_SKETCH)
    contract_ms, contract_n = plan.kernel_time(_lib.KERNEL_CONTRACT)
    plan.enable_timing(False)
    plan.check()
    value = world * nnz / (ms_step / 1e3)

    peak, peak_kind = measured_peaks()
    alg_bytes = 8 * nnz + 4 * (n + 1) + 4 * B * d
    sketch_avg_s = (sketch_ms / max(1, sketch_n)) / 1e3
    achieved = alg_bytes / sketch_avg_s / 1e9
    traffic = NCU_TRAFFIC.get((source_hash(*ksrc), name))
    red_ceiling = reduction_ceiling(dev, nnz, B * d) if rank == 0 else None

    Yp = torch.empty_like(Y)
    plain_ms = _time_calls(lambda: plan.plain_csr(rp, ci, v, out=Yp), max(3, steps // 20), stream) if plain else None
    rec = {
        "workload": name, "n": n, "d": d, "p": wl["p"], "values": wl["values"], "nnz_per_rank": nnz, "m": m, "B": B,
        "seed": seed, "ms_per_step": ms_step, "value": value, "clocks": clocks,
        "stage_pass": {"ms_per_step": stage_ms_step, "sketch_kernel_ms": sketch_ms / max(1, sketch_n),
                       "contract_kernel_ms": contract_ms / max(1, contract_n), "launches": sketch_n},
        "roofline": {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": sketch_avg_s * 1e3, "launches": sketch_n,
                     "reduction_bound": None if red_ceiling is None else {
                         "reductions_per_launch": nnz, "achieved_per_s": nnz / sketch_avg_s,
                         "ceiling_per_s": red_ceiling["per_s"],
                         "frac": (nnz / sketch_avg_s) / red_ceiling["per_s"], "ceiling": red_ceiling}},
        "plain": None if plain_ms is None else {
            "ms_per_step": plain_ms, "value": world * nnz / (plain_ms / 1e3), "unit": UNIT,
            "speedup_countgauss_over_plain": plain_ms / ms_step},
        "gpu_launches_per_step": launches_per_step,
    }
    if det:
        det_plan = countgauss.CountGauss(n, d, m, B, seed, row_offset=rank * n, deterministic=True)
        Yd = torch.empty_like(Y)
        det_ms = _time_calls(lambda: det_plan.apply_csr(rp, ci, v, out=Yd), max(3, steps // 20), stream)
        det_plan.check()
        del det_plan
        rec["deterministic"] = {"ms_per_step": det_ms, "value": world * nnz / (det_ms / 1e3), "unit": UNIT}
    if e2e:
        # end to end through the host-input call: H2D of the CSR, apply, D2H of Y, every step
        # (cg_apply_csr_host: the CSR in pinned host memory is copied in chunks on a second
        # stream while earlier chunks are scattered, or read in place by the scatter; Y comes
        # back to host memory)
        Y_h = torch.empty(m, d, dtype=torch.float32).pin_memory()
        plan.set_host_chunk(args.host_chunk)

        def e2e_step():
            plan.apply_csr_host(rp_h, ci_h, v_h, out=Y_h, device=dev)
            if pg is not None:
                Y.copy_(Y_h, non_blocking=True)
                pg.all_reduce(Y)
                Y_h.copy_(Y, non_blocking=True)

        # each call timed on its own (it synchronises) and the median taken: the host link
        # is shared with a second GPU, and a burst of its traffic can slow a few calls
        e2e_steps = max(7, steps // 10)
        e2e_ms, e2e_mean = _time_each(e2e_step, e2e_steps, stream)
        if pg is not None:
            t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            e2e_ms = float(t.item())
        modes = {}  # the two ways of reading the host CSR, each forced (this rank's time)
        for mode in ("copied", "direct"):
            plan.set_host_read(mode)
            modes[mode + "_ms"] = _time_each(e2e_step, e2e_steps, stream)[0]
        plan.set_host_read("auto")
        h2d = int(rp_h.numel() * 4 + ci_h.numel() * 4 + v_h.numel() * 4)
        rec["e2e"] = {"value": world * nnz / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": int(m * d * 4), "ms_per_step": e2e_ms, "mean_ms": e2e_mean,
                      "calls": e2e_steps, "statistic": "median of per-call times", "call": "cg_apply_csr_host",
                      "host_read": "auto", **modes}
    del rp, ci, v, rp_h, ci_h, v_h, plan
    torch.cuda.empty_cache()
    return rec, X, wl


def run_ours(args):
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    head, X, wl = measure_workload(args, args.workload, dev, rank, world, pg, e2e=not args.step_only,
                                   det=not args.step_only, plain=not args.step_only)

    rows = None
    if rank == 0 and world == 1 and not args.no_rows:
        which = tuple(args.rows.split(","))
        rows = {}
        if "nmf" in which and args.workload != "nmf_n16M_d64":
            rec, _, _ = measure_workload(args, "nmf_n16M_d64", dev, e2e=False)
            rows["nmf_n16M_d64"] = rec
        rows.update(measure_rows(dev, max(5, args.steps // 10), which))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baselines(X, wl)

    if rank == 0:
        h2d = 4 * (head["n"] + 1) + 8 * head["nnz_per_rank"]
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else f"f32+{args.precision}",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": head["n"], "d": head["d"], "p": head["p"],
                       "values": head["values"], "nnz_per_rank": head["nnz_per_rank"], "m": head["m"],
                       "B": head["B"], "seed": head["seed"],
                       "l2": "CSR inputs (%.0f MB) exceed L2; no flush" % (h2d / 1e6)},
            "roofline": head["roofline"],
            "stage_pass": head["stage_pass"],
            "plain": head["plain"],
            "e2e": head.get("e2e"),
            # per step: the scatter's kernels, the contraction and its split-K sum
            "gpu_launches": head["gpu_launches_per_step"] * args.steps,
            "clocks": head["clocks"],
            "deterministic": head.get("deterministic"),
            "rows": rows,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def reduction_sweep(args):
    """One JSON line: random fp32 reductions per second (cg_diag_random_reductions, 50 M
    adds by default) into arrays from 8 MB to 256 MB -- where the L2 stops holding the
    array the rate falls, which is the ceiling of the scatter for an SX of that size."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    count = args.sweep_count
    out = []
    for mb in (float(x) for x in args.sweep_mb.split(",")):
        cells = int(mb * (1 << 20)) // 4
        r = reduction_ceiling(dev, count, cells)
        out.append({"array_mb": mb, "reductions_per_s": r["per_s"], "ms": r["ms"]})
    print(json.dumps({"reduction_sweep": out, "count": count}))


def kl_sweep():
    """One JSON line: Theorem 1's distance bound measured on the device's sketches.  For a
    2^20 x 16 matrix with orthonormal columns and m = 32, over 64 CountSketches per B:
    KL(N(0, I) || N(0, U^T S^T S U)) (Claim 3), ||M - I||_F^2 against its closed form,
    and Pinsker's bound on the distance of the m rows, for B / (d^2 m) from 1/8 to 64.
    Then Lemma 5's distinguisher (block matrix, d = 8, m = 1024) at B = 256 (L = 2,
    B = d^2 m / 256) and at B = 4 d^2 m (L = 64): the fraction of draws whose pair-norm
    statistic for T.U exceeds the 99th percentile of the plain product's.  m is large so
    that the chi-square noise of a pair norm (about 2 sqrt(2 / m)) stays below the 2/L
    shift that a collision between two blocks causes."""
    import numpy as np
    import torch

    from paper_1606_05732_gb300 import diagnostics
    torch.cuda.set_device(0)
    d, m = 16, 32
    U = diagnostics.spread_orthonormal_csr(1 << 20, d)
    Bs = [d * d * m // 8 * (4 ** k) for k in range(6)]
    sweep = diagnostics.kl_sweep(U, m, Bs, range(64))
    lem = []
    for B in (256, 4 * 8 * 8 * 1024):
        r = diagnostics.lemma5_experiment(8, 1024, B, range(200))
        thr = float(np.quantile(r["plain"], 0.99))
        lem.append({"B": B, "L": r["L"], "B_over_d2m": B / (8 * 8 * 1024),
                    "detect_rate": float(np.mean(r["countgauss"] > thr)), "plain_p99": thr})
    print(json.dumps({"kl_sweep": sweep, "d": d, "m": m, "n": U.n, "lemma5": lem}))


def main():
    args = parse_args()
    if args.reduction_sweep:
        reduction_sweep(args)
    elif args.kl_sweep:
        kl_sweep()
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
