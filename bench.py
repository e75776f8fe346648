"""Throughput benchmark of the chi-square hot path on one or more GB300s.

Workload (one "step" = one full chi2_image evaluation: row FFT, pruned column
FFT, gather + phase + chi-square): nxy = 4096 float32 image of three random
elliptical Gaussians plus an exp(-r/0.2") disc, dxy = 0.002", M = 5e6
ALMA-like uv points (43 antennas, 60 hour angles, 93 channels around 100 GHz),
random dRA/dDec in +-0.1" and PA in [0, pi).  Inputs are resident in HBM; L2
is flushed before every timed step (a 256 MiB write, then a 256 MiB read that
takes the write-back of the dirty lines out of the timed region); each step is timed on
the device with CUDA events on the launching stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank evaluates its own replica of the workload (the steps
are independent evaluations, as in an MCMC batch): weak scaling, no
collective on the data path; rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "chi2_image evals/s at nxy=4096, Nuv=5e6 (FP32 bulk, FP64 reduction)"
UNIT = "evals/s"
WORKLOAD = "chi2_image nxy=4096 dxy=0.002as M=5e6 ALMA-like uv, 3 Gaussians + exp disc"
NXY, M_UV = 4096, 5_000_000
L2_FLUSH_BYTES = 256 << 20
STAGES = ["uv_extent", "row_fft", "col_fft", "gather_chi2"]
# kernels launched for this workload (template arguments as ncu prints them)
KERNELS = {1: "row_fft3_ldg_kernel<1, 0>",
           2: "col_fft3_kernel<float, 12, 1, 16>", 3: "gather_kernel<float, 1, 1, 0, 1, 0, 0>"}
# the full-plane (complex-to-complex) spectrum path
KERNELS_FULL = {1: "row_c2c_tma_kernel<float, 12, 1>", 2: "col_fft3_kernel<float, 12, 1, 16>",
                3: "gather_kernel<float, 1, 1, 0, 1, 0, 1>"}
# primary beam of a 12 m antenna at 100 GHz: FWHM = K lambda / D, K = 1.13
PB_FWHM = 1.13 * (299792458.0 / 100e9) / 12.0
VARIANTS = {"plain": {}, "beam": {"pb_fwhm": PB_FWHM}, "full_plane": {"full_plane": True},
            "beam_full_plane": {"pb_fwhm": PB_FWHM, "full_plane": True}}


def algorithmic_bytes(stage: int, nxy: int, M: int, Kc: int, nrw: int,
                      beam: bool = False) -> float:
    """Compulsory DRAM bytes of one launch of a stage (float32 path); Kc is
    the number of window columns (2 Kc - 1 of the half plane's Kc for the
    full plane).

    row FFT:   read the image (4 N^2) + write the kept columns (8 N Kc)
               (+ the beam tables, 2N floats, when a beam is applied)
    col FFT:   read the kept columns (8 N Kc) + write the window (8 nrw Kc)
    gather:    read u, v, Re, Im, w (20 B per point); the window (8 nrw Kc)
               is read once from DRAM and then served from cache
    """
    if stage == 1:
        return 4.0 * nxy * nxy + 8.0 * nxy * Kc + (8.0 * nxy if beam else 0.0)
    if stage == 2:
        return 8.0 * nxy * Kc + 8.0 * nrw * Kc
    if stage == 3:
        return 20.0 * M + 8.0 * nrw * Kc
    return 8.0 * M


def window(rho: float, S: float, N: int):
    """Kept spectrum window (same rule as the library's pruning)."""
    P = N // 2 + 1
    e = rho * S
    if not e < N:
        return P, N
    k = math.floor(e) + 3
    lo, hi = max(0, N // 2 - k), min(N - 1, N // 2 + k)
    return min(k + 1, P), hi - lo + 1


def fft_equivalent(nxy: int, evals_per_s: float) -> dict:
    """Secondary figure: the nominal flop count of an unpruned real-to-complex
    2D FFT of the image, 2.5 N^2 log2(N^2), per evaluation and at the measured
    rate.  The pruned transform executes fewer flops; this is the customary
    FFT-equivalent rate, not a count of executed instructions."""
    gflop = 2.5 * nxy * nxy * math.log2(float(nxy) * nxy) / 1e9
    return {"fft_gflop_per_eval": gflop, "fft_equivalent_tflop_per_s": gflop * evals_per_s / 1e3,
            "note": "nominal 2.5 N^2 log2(N^2) of an unpruned R2C 2D FFT; the pruned "
                    "transform executes fewer"}


def full_window_columns(Kc: int, N: int) -> int:
    """Columns of the full-plane window (same rule as the library): u from
    -(Kc-1) to Kc-1 when pruned, the node range -N/2 .. N/2-1 otherwise."""
    lo = N // 2 if Kc >= N // 2 + 1 else Kc - 1
    hi = min(Kc - 1, N // 2 - 1)
    return lo + hi + 1


# the sources that define the profiled kernels and their launch shapes
KERNEL_SOURCES = ("gal_common.cuh", "gal_fft.cuh", "gal_fft2.cuh", "gal_fft3.cuh",
                  "gal_fft3_launch.cuh", "gal_kernels.cuh", "gal_plane.cuh", "gal_tma.cuh",
                  "gal_internal.h")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1709_06999_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, full: bool = False):
    """DRAM bytes per launch from the committed ncu summary, if the kernels
    have not changed since it was taken (full: the full-plane variant's
    captures, whose column pass keeps more columns under the same name)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != kernel_source_hash():
        return None
    k = rec.get("kernels_full_plane" if full else "kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_launch")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# NVML clock-event reason bits (nvml.h, nvmlClocksEventReason*): the ones the
# timing rules name, plus idle
NVML_REASONS = {0x1: "gpu_idle", 0x4: "sw_power_cap", 0x8: "hw_slowdown",
                0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
                0x80: "hw_power_brake_slowdown"}


def nvml_sample_loop(target: str, period_s: float, out=None) -> int:
    """Child process of ClockSampler: read-only NVML queries of one GPU (SM
    clock, its maximum, power and the clock-event reasons) every period_s
    seconds, one line per sample: "unix_time sm_mhz max_mhz power_w reasons".
    target is "pci:<bus id>", "uuid:<GPU-...>" or "index:<n>".  Runs until
    killed."""
    import ctypes
    out = out or sys.stdout
    try:
        lib = ctypes.CDLL("libnvidia-ml.so.1")
    except OSError:
        return 1
    if lib.nvmlInit_v2() != 0:
        return 1
    h = ctypes.c_void_p()
    kind, _, val = target.partition(":")
    if kind == "pci":
        rc = lib.nvmlDeviceGetHandleByPciBusId_v2(val.encode(), ctypes.byref(h))
    elif kind == "uuid":
        rc = lib.nvmlDeviceGetHandleByUUID(val.encode(), ctypes.byref(h))
    else:
        rc = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(int(val)), ctypes.byref(h))
    if rc != 0:
        return 1
    reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
        lib.nvmlDeviceGetCurrentClocksThrottleReasons
    sm, mx, mw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
    lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))  # NVML_CLOCK_SM = 1
    while True:
        lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(sm))
        lib.nvmlDeviceGetPowerUsage(h, ctypes.byref(mw))
        reasons_fn(h, ctypes.byref(rs))
        out.write(f"{time.time():.6f} {sm.value} {mx.value} {mw.value / 1000.0:.1f} "
                  f"{rs.value}\n")
        out.flush()
        time.sleep(period_s)


def parse_clock_samples(lines, t0: float, t1: float):
    """Summary of sampler lines for the window [t0, t1] (unix seconds).  When
    the window is shorter than the sampling period and holds no sample, the
    last sample before it and the first after it stand for it (said so in
    "window")."""
    rows = []
    for ln in lines:
        parts = ln.split()
        if len(parts) != 5:
            continue
        try:
            rows.append((float(parts[0]), float(parts[1]), float(parts[2]), float(parts[3]),
                         int(parts[4])))
        except ValueError:
            continue
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"],
                "note": "no NVML sample was read"}
    inside = [r for r in rows if t0 <= r[0] <= t1]
    window = "timed region"
    if not inside:
        before = [r for r in rows if r[0] < t0][-1:]
        after = [r for r in rows if r[0] > t1][:1]
        inside = before + after
        window = "nearest samples before and after the timed region (shorter than the period)"
    reasons = set()
    for r in inside:
        for bit, name in NVML_REASONS.items():
            if r[4] & bit and name != "gpu_idle":
                reasons.add(name)
    return {"sm_mhz": statistics.median(r[1] for r in inside),
            "sm_max_mhz": max(r[2] for r in inside),
            "power_w_max": max(r[3] for r in inside),
            "reasons": sorted(reasons), "samples": len(inside), "window": window,
            "source": "NVML, read-only queries"}


class ClockSampler:
    """SM clock, power and clock-event reasons of the bench's GPU, sampled by a
    child process every 0.5 ms through NVML (read-only queries).  Start it
    before the warm-up (the child needs a moment to come up); mark() records
    the timed region, summary() reports the samples inside it."""

    def __init__(self, device_index: int, period_s: float = 0.0005):
        self.device_index = device_index
        self.period = period_s
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def _target(self):
        try:
            import torch
            pr = torch.cuda.get_device_properties(self.device_index)
            if hasattr(pr, "pci_bus_id"):
                return f"pci:{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
            return f"uuid:GPU-{pr.uuid}"
        except Exception:  # pragma: no cover - sampler is best effort
            return f"index:{self.device_index}"

    def start(self):
        try:
            self.proc = subprocess.Popen(
                [sys.executable, os.path.abspath(__file__), "--clock-sampler", self._target(),
                 str(self.period)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            # wait (at most 20 s) for the first sample, so the timed region is covered
            import select
            if select.select([self.proc.stdout], [], [], 20.0)[0]:
                line = self.proc.stdout.readline()
                if line:
                    self.lines.append(line)
        except OSError:
            self.proc = None
        return self

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return
        time.sleep(3 * self.period)  # one sample after the region
        self.proc.kill()
        out, _ = self.proc.communicate()
        self.lines += out.splitlines()
        self.proc = None

    def summary(self):
        if self.t0 is None or self.t1 is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return parse_clock_samples(self.lines, self.t0, self.t1)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------
# reference arm / CPU baseline: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def host_info() -> dict:
    """The host CPU: model name (lscpu, else /proc/cpuinfo), logical CPUs, and
    the CPUs this process may run on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith("model name"):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"cpu_model": model, "nproc": os.cpu_count(), "usable_cpus": usable}


def oracle_eval(p, re, im):
    import oracle
    return oracle.chi2_image(p.image, p.dxy, p.u, p.v, re, im, p.w, p.dRA, p.dDec, p.PA)


def make_problem(seed: int = 2):
    from paper_1709_06999_gb300 import synth
    p = synth.large_image_problem(nxy=NXY, M=M_UV, seed=seed)
    p.image = p.image.astype(np.float32).astype(np.float64)
    for k in ("u", "v", "w", "noise_re", "noise_im"):
        setattr(p, k, getattr(p, k).astype(np.float32).astype(np.float64))
    return p


def oracle_eval_threads(p, re, im, pool, nthreads: int):
    """One full oracle evaluation on all host cores: the oracle's own image FFT
    (one call), then its sampling and chi-square on nthreads contiguous shares
    of the points in a thread pool (numpy releases the GIL in its array loops),
    the shares' exactly rounded sums added with math.fsum.  Every step is the
    unchanged oracle."""
    import oracle
    G = oracle.half_spectrum(p.image)
    n = p.image.shape[0]
    b = np.linspace(0, p.u.size, nthreads + 1).astype(np.int64)

    def part(k):
        s = slice(int(b[k]), int(b[k + 1]))
        vis = oracle.sample_spectrum(G, n, p.dxy, p.u[s], p.v[s], p.dRA, p.dDec, p.PA)
        return oracle.chi2(vis, re[s], im[s], p.w[s])

    return math.fsum(pool.map(part, range(nthreads)))


def oracle_chi2_sharded(p, re, im, dRA, dDec, PA, pool, nthreads: int, pb_fwhm: float = 0.0,
                        full_plane: bool = False, copies=None):
    """The FP64 oracle's chi-square of one evaluation of the workload p (its
    float32-rounded inputs, observed data re, im) at the geometry (dRA, dDec,
    PA): the oracle's spectrum of the image (times its primary beam when
    pb_fwhm > 0, the complex-to-complex one for full_plane) computed once,
    then its sampling on nthreads contiguous shares of the points in a thread
    pool -- summed over the copies (amp, dRA_k, dDec_k) of a multi-source
    model when given, the linear sum that sample_image_multi forms -- and its
    chi-square of each share, the shares' exactly rounded sums added with
    math.fsum."""
    import oracle
    n = p.image.shape[0]
    img = p.image
    if pb_fwhm > 0.0:
        img = img * oracle.primary_beam(n, p.dxy, pb_fwhm, dRA, dDec, PA)
    G = oracle.full_spectrum(img) if full_plane else oracle.half_spectrum(img)
    sample = oracle.sample_full_spectrum if full_plane else oracle.sample_spectrum
    offsets = copies if copies is not None else [(1.0, dRA, dDec)]
    b = np.linspace(0, p.u.size, nthreads + 1).astype(np.int64)

    def part(k):
        s = slice(int(b[k]), int(b[k + 1]))
        vis = 0.0
        for a, x, y in offsets:
            vis = vis + a * sample(G, n, p.dxy, p.u[s], p.v[s], x, y, PA)
        return oracle.chi2(vis, re[s], im[s], p.w[s])

    return math.fsum(pool.map(part, range(nthreads)))


def cpu_baseline(p, re, im, evals: int):
    """The FP64 oracle timed on the host cores on full evaluations of the
    workload: single-threaded (numpy as it stands) and on all usable cores
    (oracle_eval_threads), at least three evaluations each, min and median."""
    from concurrent.futures import ThreadPoolExecutor
    host = host_info()
    evals = max(3, evals)
    single = []
    for _ in range(evals):
        t0 = time.perf_counter()
        oracle_eval(p, re, im)
        single.append(time.perf_counter() - t0)
    nthr = max(1, host["usable_cpus"] or 1)
    allc = []
    with ThreadPoolExecutor(nthr) as pool:
        oracle_eval_threads(p, re, im, pool, nthr)  # warm the pool
        for _ in range(evals):
            t0 = time.perf_counter()
            oracle_eval_threads(p, re, im, pool, nthr)
            allc.append(time.perf_counter() - t0)
    med = statistics.median(allc)
    return {"value": 1.0 / med, "unit": UNIT, "cores": nthr, "kind": "oracle",
            "sample": f"{evals} full FP64 oracle chi2_image evaluations of the same workload on "
                      f"{nthr} threads (image FFT in one numpy call, then sampling and chi2 on "
                      f"{nthr} contiguous shares of the points); value = 1 / median",
            "seconds_per_eval": {"min": min(allc), "median": med},
            "single_thread": {"value": 1.0 / statistics.median(single), "cores": 1,
                              "seconds_per_eval": {"min": min(single),
                                                   "median": statistics.median(single)},
                              "evals": evals},
            "host": host}


REF_SAMPLE_POINTS = 100_000   # uv points per reference step when full evaluations do not fit
REF_BUDGET_S = 150.0          # whole --steps K --warmup W run of the reference arm


def run_reference(args):
    """The FP64 oracle on the host cores, on the same workload and metric.

    Each step is one full evaluation on all usable cores (oracle_eval_threads)
    when K + W of them fit in about REF_BUDGET_S seconds (the first warm-up
    evaluation sets the estimate); the rate is then measured, 1 / mean step
    time.  Otherwise (a very large --steps) each step samples and reduces
    REF_SAMPLE_POINTS consecutive points after one timed image FFT, and the
    rate is an estimate, FFT time + mean step time x M / sample, labelled so
    in the line."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    p = make_problem()
    rng = np.random.default_rng(7)
    re = rng.standard_normal(p.u.size)
    im = rng.standard_normal(p.u.size)
    host = host_info()
    nthr = max(1, host["usable_cpus"] or 1)
    pool = ThreadPoolExecutor(nthr)
    t0 = time.perf_counter()
    oracle_eval_threads(p, re, im, pool, nthr)
    t_full = time.perf_counter() - t0
    full = (args.steps + args.warmup) * t_full <= REF_BUDGET_S
    if full:
        for _ in range(max(0, args.warmup - 1)):
            oracle_eval_threads(p, re, im, pool, nthr)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle_eval_threads(p, re, im, pool, nthr)
        dt = time.perf_counter() - t0
        value = args.steps / dt
        sample = (f"each step: one full FP64 oracle chi2_image evaluation of the workload on "
                  f"{nthr} threads (image FFT, then sampling and chi2 on {nthr} shares); "
                  f"measured, value = steps / time")
        estimate = False
    else:
        t0 = time.perf_counter()
        G = oracle.half_spectrum(p.image)
        t_fft = time.perf_counter() - t0
        m = min(REF_SAMPLE_POINTS, p.u.size)
        nsamp = p.u.size // m

        def step(i):
            lo = (i % nsamp) * m
            sl = slice(lo, lo + m)
            vis = oracle.sample_spectrum(G, NXY, p.dxy, p.u[sl], p.v[sl], p.dRA, p.dDec, p.PA)
            return oracle.chi2(vis, re[sl], im[sl], p.w[sl])

        for i in range(args.warmup):
            step(i)
        t0 = time.perf_counter()
        for i in range(args.steps):
            step(i)
        dt = time.perf_counter() - t0
        value = 1.0 / (t_fft + (dt / args.steps) * (p.u.size / m))
        nthr = 1
        sample = (f"ESTIMATE: each step samples and reduces {m} of the {p.u.size} points on one "
                  f"thread; image FFT timed once ({t_fft:.2f} s); value = 1 / (FFT + step x "
                  f"{p.u.size // m}) (full evaluations would not fit {REF_BUDGET_S:.0f} s)")
        estimate = True
    pool.shutdown()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nxy": NXY, "M": M_UV},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthr, "kind": "oracle",
                         "sample": sample, "estimate": estimate, "host": host},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# accuracy against the FP64 oracle
# ---------------------------------------------------------------------------
def oracle_model_threads(p, pool, nthreads: int):
    """The oracle's visibilities of the workload at its own geometry, computed
    by the unchanged oracle on nthreads contiguous shares of the points."""
    import oracle
    G = oracle.half_spectrum(p.image)
    n = p.image.shape[0]
    b = np.linspace(0, p.u.size, nthreads + 1).astype(np.int64)
    parts = pool.map(lambda k: oracle.sample_spectrum(G, n, p.dxy, p.u[b[k]:b[k + 1]],
                                                      p.v[b[k]:b[k + 1]], p.dRA, p.dDec, p.PA),
                     range(nthreads))
    return np.concatenate(list(parts))


def measure_accuracy(torch, ctx, dev, p, re_h, im_h):
    """Error of each result against the FP64 oracle on the very inputs the
    path sees (the workload's float32-rounded image, uv and weights; observed
    data re_h, im_h as float32 values), for the float32 and float64 paths:

    vis_normwise     max_k |V_k - V_oracle,k| / max_k |V_oracle,k|, all M points
    vis_rms          sqrt(mean_k |V_k - V_oracle,k|^2) / max_k |V_oracle,k|
    chi2_rel         |chi2 - chi2_oracle| / chi2_oracle, observed = model + noise
    chi2_model_rms   observed = the oracle model itself: chi2 = sum_k w_k |dV_k|^2,
                     reported as sqrt(chi2 / sum_k w_k) / max|V| (the weighted rms
                     model error, with no noise term to hide it)
    phase_max_abs    a unit point source at the phase centre has the constant
                     spectrum 1 (exact in both precisions), so its visibilities
                     are exp(2 pi i (u dRA + v dDec)) and the difference is the
                     error of the phase factor alone: max_k |V_k - exp(i theta_k)|
    """
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    nthr = max(1, host_info()["usable_cpus"] or 1)
    with ThreadPoolExecutor(nthr) as pool:
        model = oracle_model_threads(p, pool, nthr)
    vmax = float(np.max(np.abs(model)))
    theta = 2.0 * np.pi * (p.u * p.dRA + p.v * p.dDec)
    unit = np.exp(1j * theta)
    N = p.image.shape[0]
    delta = np.zeros((N, N))
    delta[N // 2, N // 2] = 1.0
    out = {"reference": "FP64 oracle on the same float32-rounded inputs",
           "geometry": {"dRA": p.dRA, "dDec": p.dDec, "PA": p.PA}}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
        img, u, v, w = d(p.image), d(p.u), d(p.v), d(p.w)
        vis = ctx.sample_image(img, p.dxy, u, v, p.dRA, p.dDec, p.PA).double().cpu().numpy()
        V = vis[:, 0] + 1j * vis[:, 1]
        dV = np.abs(V - model)
        obs = ctx.register(u, v, d(re_h), d(im_h), w)
        c = ctx.chi2_image(img, p.dxy, obs, p.dRA, p.dDec, p.PA).item()
        c_ref = oracle.chi2(model, re_h, im_h, p.w)
        obs0 = ctx.register(u, v, d(model.real), d(model.imag), w)
        c0 = ctx.chi2_image(img, p.dxy, obs0, p.dRA, p.dDec, p.PA).item()
        vd = ctx.sample_image(d(delta), p.dxy, u, v, p.dRA, p.dDec, p.PA).double().cpu().numpy()
        out[name] = {"vis_normwise": float(np.max(dV) / vmax),
                     "vis_rms": float(np.sqrt(np.mean(dV * dV)) / vmax),
                     "chi2_rel": abs(c - c_ref) / c_ref,
                     "chi2_model_rms": float(np.sqrt(max(c0, 0.0) / np.sum(p.w)) / vmax),
                     "phase_max_abs": float(np.max(np.abs(vd[:, 0] + 1j * vd[:, 1] - unit)))}
        obs.close()
        obs0.close()
    out["gates"] = {"f32": {"vis_normwise": 1e-5, "chi2_rel": 1e-6},
                    "f64": {"vis_normwise": 1e-12, "chi2_rel": 1e-12}}
    return out


def oracle_chi2_of(r, arrays):
    """The FP64 oracle's chi-square of one batched or served request, on the
    request's own float32 arrays (u, v, re, im, w)."""
    import oracle
    u, v, re, im, w = (np.asarray(t.double().cpu().numpy() if hasattr(t, "cpu") else t,
                                  dtype=np.float64) for t in arrays)
    if r.image is not None:
        return oracle.chi2_image(r.image.double().cpu().numpy(), r.dxy, u, v, re, im, w, r.dRA,
                                 r.dDec, r.PA, pb_fwhm=r.pb_fwhm)
    return oracle.chi2_profile(r.intensity.double().cpu().numpy(), r.Rmin, r.dR, r.nxy, r.dxy,
                               u, v, re, im, w, r.dRA, r.dDec, r.PA, r.inc)


# ---------------------------------------------------------------------------
# batched and served throughput (extra measurements at N = 1)
# ---------------------------------------------------------------------------
def _timed(torch, fn, reps, flush=None):
    """Mean device milliseconds of fn() over reps runs (events on the current stream)."""
    total = 0.0
    for _ in range(reps):
        if flush is not None:
            flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        total += a.elapsed_time(b)
    return total / reps


def _single(ctx, r, out=None):
    if r.image is not None:
        return ctx.chi2_image(r.image, r.dxy, r.obs, r.dRA, r.dDec, r.PA, out=out,
                              pb_fwhm=r.pb_fwhm)
    return ctx.chi2_profile(r.intensity, r.Rmin, r.dR, r.nxy, r.dxy, r.obs, r.inc, r.dRA, r.dDec,
                            r.PA, out=out, pb_fwhm=r.pb_fwhm)


def measure_plane(torch, ctx, dev, img, obs, dxy, params, flush_l2, out, steps=200,
                  oracle_chi2=None):
    """chi2_image of the same workload with a primary beam, through the
    full-plane spectrum, and both: L2 flushed before every step, each step
    bracketed by events, plus per-stage times from three calibration steps.
    oracle_chi2(dRA, dDec, PA, pb_fwhm=..., full_plane=...), when given, is
    the FP64 oracle's chi-square of that evaluation: each variant's result at
    the first geometry is stated against it."""
    variants = {k: v for k, v in VARIANTS.items() if k != "plain"}
    stream = torch.cuda.current_stream(dev)
    res = {}
    for name, kw in variants.items():
        for i in range(3):
            ctx.chi2_image(img, dxy, obs, *params[i], out=out, **kw)
        ctx.set_stage_timing(True)
        for i in range(3):
            flush_l2()
            ctx.chi2_image(img, dxy, obs, *params[i], out=out, **kw)
        cal = ctx.stage_times()
        ctx.set_stage_timing(False)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        torch.cuda.synchronize(dev)
        for i in range(steps):
            flush_l2()
            ev[i][0].record(stream)
            ctx.chi2_image(img, dxy, obs, *params[i % len(params)], out=out, **kw)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        res[name] = {"value": 1000.0 / ms, "unit": UNIT, "ms_per_step": ms,
                     "pb_fwhm_rad": kw.get("pb_fwhm", 0.0),
                     "full_plane": bool(kw.get("full_plane", False)),
                     "stages_us_per_step": {STAGES[s]: round(1000 * cal[s][0] / 3, 2)
                                            for s in range(4) if cal[s][1]}}
        if oracle_chi2 is not None:
            got = ctx.chi2_image(img, dxy, obs, *params[0], out=out, **kw).item()
            ref = oracle_chi2(*params[0], pb_fwhm=kw.get("pb_fwhm", 0.0),
                              full_plane=bool(kw.get("full_plane", False)))
            res[name]["chi2_rel_err_vs_oracle"] = abs(got - ref) / abs(ref)
    res["note"] = ("same workload and timing as the headline step; per-stage times are sums "
                   "per step over 3 calibration steps, each launch with about 4 us of event "
                   "overhead; the beam-table launch belongs to the row stage")
    return res


def measure_next(torch, ctx, dev, img, obs, p, params, flush_l2, out, steps=200,
                 oracle_chi2=None):
    """The widened paths at the headline workload: multi-source chi2 (K copies
    of the model, one FFT, K phase terms per point; L2 flushed before every
    step, each step event-timed), registration from baselines in metres with
    one frequency per visibility, and get_image_size on the same coverage (both
    return to the host, so they are wall-clock timed per call).  oracle_chi2,
    when given, states each multi-source result at the first position angle
    against the FP64 oracle (its copies= argument), the chi-square of the
    observation registered from metres against the oracle's at its own
    wavelengths (problem=), and get_image_size against oracle.image_size."""
    stream = torch.cuda.current_stream(dev)
    rng = np.random.default_rng(31)
    arc = math.pi / 648000
    res = {}
    for K in (4, 16):
        dra = [float(x) for x in rng.uniform(-0.5, 0.5, K) * arc]
        ddec = [float(x) for x in rng.uniform(-0.5, 0.5, K) * arc]
        amp = [float(x) for x in rng.uniform(0.2, 1.0, K)]

        def step(i):
            ctx.chi2_image_multi(img, p.dxy, obs, dra, ddec, amp, params[i % len(params)][2],
                                 out=out)
        for i in range(3):
            step(i)
        ctx.set_stage_timing(True)
        for i in range(3):
            flush_l2()
            step(i)
        cal = ctx.stage_times()
        ctx.set_stage_timing(False)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        torch.cuda.synchronize(dev)
        for i in range(steps):
            flush_l2()
            ev[i][0].record(stream)
            step(i)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        res[f"multi_source_K{K}"] = {
            "value": 1000.0 / ms, "unit": UNIT, "ms_per_step": ms, "sources": K,
            "stages_us_per_step": {STAGES[s]: round(1000 * cal[s][0] / 3, 2)
                                   for s in range(4) if cal[s][1]}}
        if oracle_chi2 is not None:
            PA0 = params[0][2]
            got = ctx.chi2_image_multi(img, p.dxy, obs, dra, ddec, amp, PA0, out=out).item()
            ref = oracle_chi2(0.0, 0.0, PA0, copies=list(zip(amp, dra, ddec)))
            res[f"multi_source_K{K}"]["chi2_rel_err_vs_oracle"] = abs(got - ref) / abs(ref)
    # one frequency per visibility around 100 GHz (the coverage's 93 channels
    # span +-3.75 %), baselines in metres = u c / nu
    M = p.u.size
    nu = 100e9 * (1.0 + rng.uniform(-0.0375, 0.0375, M))
    d32 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)  # noqa: E731
    u_m, v_m, nu_d = d32(p.u * 299792458.0 / nu), d32(p.v * 299792458.0 / nu), d32(nu)
    rest = [t.contiguous() for t in obs._tensors[2:]]
    ctx.register_freq(u_m, v_m, nu_d, *rest).close()
    torch.cuda.synchronize(dev)
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        ctx.register_freq(u_m, v_m, nu_d, *rest).close()
    ms_f = 1000.0 * (time.perf_counter() - t0) / reps
    res["freq_registration"] = {
        "ms_per_registration": ms_f, "points": M,
        "note": "u_m, v_m, nu (f32) -> u, v in wavelengths (FP64 product, rounded once), then "
                "the uv extent and its read-back; includes the handle's allocation"}
    if oracle_chi2 is not None:
        # chi2 of the observation registered from metres and frequencies,
        # against the oracle's chi2 at its own wavelengths (uv_from_frequency
        # of the same float32 values, rounded to float32 as the kernel stores
        # them)
        import copy
        import oracle
        obs_f = ctx.register_freq(u_m, v_m, nu_d, *rest)
        got = ctx.chi2_image(img, p.dxy, obs_f, *params[0], out=out).item()
        obs_f.close()
        uw, vw = oracle.uv_from_frequency(u_m.double().cpu().numpy(), v_m.double().cpu().numpy(),
                                          nu_d.double().cpu().numpy())
        pf = copy.copy(p)
        pf.u = uw.astype(np.float32).astype(np.float64)
        pf.v = vw.astype(np.float32).astype(np.float64)
        ref = oracle_chi2(*params[0], problem=pf)
        res["freq_registration"]["chi2_rel_err_vs_oracle"] = abs(got - ref) / abs(ref)
    u_d, v_d = obs._tensors[0], obs._tensors[1]
    ctx.get_image_size(u_d, v_d)
    t0 = time.perf_counter()
    for _ in range(reps):
        nxy, dxy = ctx.get_image_size(u_d, v_d)
    res["image_size"] = {"ms_per_call": 1000.0 * (time.perf_counter() - t0) / reps, "nxy": nxy,
                         "dxy_arcsec": dxy / arc, "points": M,
                         "note": "criterion (iia) of Sect. 3.3 on the 5e6-point coverage"}
    if oracle_chi2 is not None:
        import oracle
        n_ref, dxy_ref = oracle.image_size(p.u, p.v)
        res["image_size"]["oracle"] = {"nxy": int(n_ref), "dxy_rel_err": abs(dxy - dxy_ref) / dxy_ref}
    return res


def launch_shape(ctx, reqs):
    """The float32 launch shape the context keeps for this batch (tuned by its
    first call): every request here runs in the batched kernels."""
    import torch
    (rb, jobs, fold), kept = ctx.batch_shape(torch.float32, len(reqs), max(r.nxy for r in reqs))
    return {"row_blocks_per_sm": rb, "requests_per_launch": jobs, "gather_fold": fold,
            "tuned": kept}


def measure_batched(torch, ctx, dev, flush, reps=3, n_oracle=3):
    """Spectral cube (128 Keplerian channels, nxy in {512, 1024, 2048}, M_c in
    [1e5, 2e6]), 64 ring-profile walkers (nxy 1024, M 1e6 shared) and 16
    walkers of the large single-image case (nxy 4096, M 5e6 shared): one
    gal_chi2_batch per set, its CUDA-graph replay, sequential FP32 single
    calls and sequential FP64 single calls of the same requests."""
    from paper_1709_06999_gb300 import Request, get_fft_radix, synth
    d32 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)  # noqa: E731
    sets = {}
    cube = synth.spectral_cube(n_chan=128, seed=3)
    r32, r64, arr_cube = [], [], []
    for ch in cube:
        t32 = [d32(a) for a in (ch.u, ch.v, ch.noise_re, ch.noise_im, ch.w)]
        arr_cube.append(t32)
        o32 = ctx.register(*t32, z_order=True)
        o64 = ctx.register(*[t.double() for t in t32], z_order=True)
        img = d32(ch.image)
        r32.append(Request(o32, image=img, dxy=ch.dxy, dRA=ch.dRA, dDec=ch.dDec, PA=ch.PA))
        r64.append(Request(o64, image=img.double(), dxy=ch.dxy, dRA=ch.dRA, dDec=ch.dDec,
                           PA=ch.PA))
    sets["cube"] = (r32, r64, "128 Keplerian-disc channels, nxy U{512,1024,2048}, "
                              "M_c U[1e5,2e6] (ALMA-like layout x channel frequency), "
                              "observations registered in Z-order", arr_cube)
    # the same channels, each through its own primary beam: FWHM 1.13 lambda_c / 12 m
    # (channel frequency: line at 100 GHz, channels 0.5 km/s apart, as in the cube)
    b32, b64 = [], []
    for k, (a, b) in enumerate(zip(r32, r64)):
        v_chan = (k - (len(r32) - 1) / 2) * 0.5
        theta = 1.13 * (299792458.0 / (100e9 * (1.0 - v_chan / 299792.458))) / 12.0
        for src, dst in ((a, b32), (b, b64)):
            dst.append(Request(src.obs, image=src.image, dxy=src.dxy, dRA=src.dRA,
                               dDec=src.dDec, PA=src.PA, pb_fwhm=theta))
    sets["cube_beams"] = (b32, b64, "the same 128 channels, each with its primary beam "
                                    "(FWHM 1.13 lambda_c / 12 m, applied in the row FFT)",
                          arr_cube)
    q = synth.profile_problem(nxy=1024, M=1_000_000, nr=8192, seed=1)
    t32 = [d32(a) for a in (q.u, q.v, q.noise_re, q.noise_im, q.w)]
    o32 = ctx.register(*t32, z_order=True)
    o64 = ctx.register(*[t.double() for t in t32], z_order=True)
    w32, w64 = [], []
    for wp in synth.walker_params(64):
        I = d32(synth.ring_profile(8192, q.dR, q.Rmin, wp["r0"], wp["width"], wp["power"]))
        kw = dict(nxy=q.nxy, dxy=q.dxy, Rmin=q.Rmin, dR=q.dR, inc=wp["inc"], dRA=wp["dRA"],
                  dDec=wp["dDec"], PA=wp["PA"])
        w32.append(Request(o32, intensity=I, **kw))
        w64.append(Request(o64, intensity=I.double(), **kw))
    sets["walkers"] = (w32, w64, "64 ring-profile walkers, nxy 1024, nr 8192, one M=1e6 "
                                 "observation shared, registered in Z-order", [t32] * len(w32))
    # 16 MCMC walkers of the large single-image case: distinct models (the
    # large image scaled per walker) and geometries, one observation shared
    lp = synth.large_image_problem()
    lt = [d32(a) for a in (lp.u, lp.v, lp.noise_re, lp.noise_im, lp.w)]
    lo32 = ctx.register(*lt)
    lo64 = ctx.register(*[t.double() for t in lt])
    lrng = np.random.default_rng(17)
    limg = d32(lp.image)
    l32, l64 = [], []
    for k in range(16):
        img_k = limg * float(1.0 + 0.01 * k)
        dRA, dDec = (float(x) for x in lrng.uniform(-0.1, 0.1, 2) * math.pi / 648000)
        PA = float(lrng.uniform(0.0, math.pi))
        l32.append(Request(lo32, image=img_k, dxy=lp.dxy, dRA=dRA, dDec=dDec, PA=PA))
        l64.append(Request(lo64, image=img_k.double(), dxy=lp.dxy, dRA=dRA, dDec=dDec, PA=PA))
    sets["large_walkers"] = (l32, l64, "16 walkers of the large single-image case (nxy 4096, "
                                       "M 5e6 shared): distinct models and geometries, input order",
                             [lt] * len(l32))
    res = {}
    for name, (a32, a64, desc, arrays) in sets.items():
        n = len(a32)
        out = ctx.chi2_batch(a32)                      # first call tunes the launch shape
        seq = torch.stack([_single(ctx, r) for r in a32])
        ref64 = torch.stack([_single(ctx, r) for r in a64])
        torch.cuda.synchronize(dev)
        l0 = ctx.launch_count()
        ms_b = _timed(torch, lambda: ctx.chi2_batch(a32, out=out), reps, flush)
        launches = (ctx.launch_count() - l0) // reps
        g = ctx.capture_batch(a32)
        g.launch()
        ms_g = _timed(torch, g.launch, reps, flush)
        outs = torch.empty(n, dtype=torch.float64, device=dev)
        ms_s = _timed(torch, lambda: [_single(ctx, r, out=outs[k]) for k, r in enumerate(a32)],
                      reps, flush)
        ms_64 = _timed(torch, lambda: [_single(ctx, r, out=outs[k]) for k, r in enumerate(a64)],
                       1, flush)
        rel = ((out - ref64).abs() / ref64.abs()).max().item()
        # against the FP64 oracle: the first n_oracle requests of the set
        got = out.cpu().numpy()
        refs = [oracle_chi2_of(a32[k], arrays[k]) for k in range(n_oracle)]
        rel_oracle = max(abs(got[k] - refs[k]) / abs(refs[k]) for k in range(n_oracle))
        # compulsory bytes of the batch: every request reads its image (4 N^2)
        # or profile (4 nr) once and its observation's five arrays (20 B per
        # point) once; requests sharing an observation each read it
        alg = sum((4.0 * r.nxy * r.nxy if r.image is not None else 4.0 * r.intensity.numel())
                  + 20.0 * r.obs.M for r in a32)
        peak_gbs, peak_kind = peaks()
        res_roof = {"bound": "hbm", "algorithmic_bytes_per_batch": alg,
                    "achieved": alg / (ms_g * 1e-3) / 1e9, "peak": peak_gbs, "unit": "GB/s",
                    "frac": alg / (ms_g * 1e-3) / 1e9 / peak_gbs,
                    "peak_source": f"{peak_kind} hbm_gbs",
                    "note": "whole batch (all passes) from its graph replay time"}
        res[name] = {
            "workload": desc, "requests": n,
            "batched_evals_per_s": 1000.0 * n / ms_b, "graph_evals_per_s": 1000.0 * n / ms_g,
            "single_fp32_evals_per_s": 1000.0 * n / ms_s,
            "plain_fp64_evals_per_s": 1000.0 * n / ms_64,
            "ms_per_batch": ms_b, "launches_per_batch": launches,
            "bitwise_equal_to_single_calls": bool(torch.equal(out, seq)),
            "max_rel_err_vs_fp64_path": rel,
            "max_chi2_rel_err_vs_oracle": rel_oracle,
            "oracle_checked_requests": n_oracle,
            "fft_plans": {str(nx): list(get_fft_radix(dev.index or 0, torch.float32, nx))
                          for nx in sorted({int(r.nxy) for r in a32})},
            "launch_shape": launch_shape(ctx, a32),
            "roofline": res_roof,
        }
        g.close()
    return res


def measure_serving(torch, dev, seconds=2.0, rate=2000.0, seed=21):
    """Poisson arrivals (rate/s) of chi2_image / chi2_profile requests (50/50),
    nxy U{256..4096}, over 16 resident observations with M log-U[1e4, 5e6]:
    the FP32 server (4 slots, batches of <= 16, 150 GB budget) against the
    plain FP64 path (single calls, one at a time, in arrival order)."""
    from paper_1709_06999_gb300 import Context, Request, Server, synth
    rng = np.random.default_rng(seed)
    d32 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)  # noqa: E731
    sizes = (256, 512, 1024, 2048, 4096)
    fov = 4096 * 0.002 * synth.ARCSEC
    srv = Server(dev.index or 0, hbm_budget=150 * 10**9, slots=4, max_batch=16)
    ctx64 = Context(dev.index or 0)
    data32, data64 = [], []
    for _ in range(16):
        m = int(np.exp(rng.uniform(np.log(1e4), np.log(5e6))))
        u, v = synth.alma_like_uv(m, rng)
        w = synth.weights_uniform(m, rng)
        nre, nim = synth.noise(w, rng)
        t = [d32(a) for a in (u, v, nre, nim, w)]
        data32.append(srv.add_data(*t))
        data64.append(ctx64.register(*[x.double() for x in t]))
    imgs = {s: d32(synth.large_image(s, fov / s, rng)) for s in sizes}
    nr = 8192
    dR = 4.5 * synth.ARCSEC * 1.6 / nr
    prof = d32(synth.ring_profile(nr, dR, dR / 2))
    n = int(rate * seconds)
    trace = []
    for _ in range(n):
        k = int(rng.integers(16))
        s = int(sizes[rng.integers(len(sizes))])
        geo = dict(dxy=fov / s, dRA=float(rng.uniform(-0.1, 0.1) * synth.ARCSEC),
                   dDec=float(rng.uniform(-0.1, 0.1) * synth.ARCSEC), PA=float(rng.uniform(0, np.pi)))
        if rng.random() < 0.5:
            trace.append((k, dict(image=True, nxy=s, **geo)))
        else:
            trace.append((k, dict(image=False, nxy=s, inc=float(rng.uniform(0, 1.2)), **geo)))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n))

    def make(k, spec, data, dt):
        kw = {x: spec[x] for x in ("dxy", "dRA", "dDec", "PA")}
        if spec["image"]:
            img = imgs[spec["nxy"]]
            return Request(data[k], image=img if dt == torch.float32 else img.double(), **kw)
        I = prof if dt == torch.float32 else prof.double()
        return Request(data[k], intensity=I, nxy=spec["nxy"], Rmin=dR / 2, dR=dR,
                       inc=spec["inc"], **kw)

    reqs32 = [make(k, sp, data32, torch.float32) for k, sp in trace]

    def serve(reqs, times):
        t0 = time.perf_counter()
        tickets = []
        for r, ta in zip(reqs, times):
            while time.perf_counter() - t0 < ta:
                pass
            tickets.append(srv.submit(r))
        got = [srv.wait(tk) for tk in tickets]
        return np.array([g[1] for g in got]), np.array([g[0] for g in got])

    # warm-up: the first 20% of the trace (every worker grows its workspaces)
    n_warm = max(1, n // 5)
    serve(reqs32[:n_warm], arrivals[:n_warm])
    lat, chi2_served = serve(reqs32, arrivals)
    span = max(float(np.max(arrivals + lat)), float(arrivals[-1]))
    st = srv.stats()
    srv.close()
    # served results against the FP64 oracle: the first request of each kind
    # at the largest and smallest sizes in the trace
    picks = []
    for want in ((True, 4096), (False, 4096), (True, 256), (False, 256)):
        k = next((i for i, (_, sp) in enumerate(trace) if (sp["image"], sp["nxy"]) == want), None)
        if k is not None:
            picks.append(k)
    served_rel = 0.0
    for i in picks:
        r = reqs32[i]
        ref = oracle_chi2_of(r, data32[trace[i][0]]._tensors)
        served_rel = max(served_rel, abs(chi2_served[i] - ref) / abs(ref))
    # plain FP64: one single call at a time, in arrival order
    imgs64 = {s: im.double() for s, im in imgs.items()}
    prof64 = prof.double()
    for s in sizes:
        ctx64.chi2_image(imgs64[s], fov / s, data64[0])
    torch.cuda.synchronize(dev)
    out = torch.empty((), dtype=torch.float64, device=dev)
    lat64 = np.empty(n)
    t0 = time.perf_counter()
    for i, ((k, sp), ta) in enumerate(zip(trace, arrivals)):
        while time.perf_counter() - t0 < ta:
            pass
        if sp["image"]:
            ctx64.chi2_image(imgs64[sp["nxy"]], sp["dxy"], data64[k], sp["dRA"], sp["dDec"],
                             sp["PA"], out=out)
        else:
            ctx64.chi2_profile(prof64, dR / 2, dR, sp["nxy"], sp["dxy"], data64[k], sp["inc"],
                               sp["dRA"], sp["dDec"], sp["PA"], out=out)
        torch.cuda.synchronize(dev)
        lat64[i] = time.perf_counter() - t0 - ta
    span64 = float(np.max(arrivals + lat64))
    ms = lambda x, q: float(np.percentile(x, q) * 1000.0)  # noqa: E731
    return {
        "workload": f"Poisson {rate:.0f} req/s for {seconds:.1f} s, chi2_image/chi2_profile 50/50, "
                    "nxy U{256..4096}, 16 resident observations M log-U[1e4,5e6]",
        "requests": n,
        "fp32_server": {"p50_ms": ms(lat, 50), "p99_ms": ms(lat, 99), "mean_ms": float(lat.mean() * 1e3),
                        "throughput_req_per_s": n / span, "launches": st["launches"],
                        "max_inflight": st["max_inflight"], "peak_hbm_bytes": st["peak_bytes"],
                        "slots": 4, "max_batch": 16, "budget_bytes": 150 * 10**9,
                        "max_chi2_rel_err_vs_oracle": served_rel,
                        "oracle_checked_requests": len(picks)},
        "plain_fp64": {"p50_ms": ms(lat64, 50), "p99_ms": ms(lat64, 99),
                       "mean_ms": float(lat64.mean() * 1e3), "throughput_req_per_s": n / span64},
        "latency": "host clock, submit to result in host memory",
    }


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_1709_06999_gb300 import Context

    p = make_problem(seed=2 + rank)
    ctx = Context(dev.index)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)  # noqa: E731
    img = d(p.image)
    u, v, w = d(p.u), d(p.v), d(p.w)
    # observed data = model (from this library) + noise: inputs for timing only
    model = ctx.sample_image(img, p.dxy, u, v, p.dRA, p.dDec, p.PA)
    re = (model[:, 0] + d(p.noise_re)).contiguous()
    im = (model[:, 1] + d(p.noise_im)).contiguous()
    obs = ctx.register(u, v, re, im, w)
    out = torch.empty((), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    flush_rd = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # a few parameter sets, as successive MCMC steps would use
    prng = np.random.default_rng(11 + rank)
    params = [(float(a), float(b), float(c)) for a, b, c in
              zip(prng.uniform(-0.1, 0.1, 8) * math.pi / 648000,
                  prng.uniform(-0.1, 0.1, 8) * math.pi / 648000, prng.uniform(0, math.pi, 8))]

    opts = VARIANTS[args.variant]

    def step(i):
        dRA, dDec, PA = params[i % len(params)]
        ctx.chi2_image(img, p.dxy, obs, dRA, dDec, PA, out=out, **opts)

    def flush_l2():
        # write a buffer larger than L2 (evicts every line of the workload),
        # then read a second one so that the write-back of those dirty lines
        # happens here and not inside the next timed step
        flush.zero_()
        flush_rd.sum(dtype=torch.int32)

    clk = ClockSampler(dev.index).start()
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize(dev)
    # calibration (untimed): per-stage event times of a few steps (reported
    # as stages_us; events between kernels stop the dependent launches)
    ctx.set_stage_timing(True)
    for i in range(3):
        flush_l2()
        step(i)
    cal = ctx.stage_times()
    ctx.set_stage_timing(False)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    launches0 = ctx.launch_count()
    # The timed region holds exactly K plain steps.  The dominant kernel's own
    # launch time is measured afterwards on separate steps of the same kind
    # (L2 flushed, events around that kernel alone): events between kernels
    # would also stop the dependent launch of the next kernel.
    clk.begin()
    for i in range(args.steps):
        flush_l2()
        ev[i][0].record(stream)
        step(i)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    clk.end()
    clk.stop()
    gpu_launches = ctx.launch_count() - launches0
    # The dominant kernel: each pass's own launch time, measured the same way
    # for all three (L2 flushed, events around that kernel alone, on separate
    # steps after the timed region); the longest is the roofline's kernel.
    # (per step: a stage of more than one launch, as the beam table and the
    # row pass of the beam variants, counts as one)
    stage = {s: (0.0, 0) for s in range(4)}
    n_alone = max(10, min(args.steps, 50))
    for s in (1, 2, 3):
        ctx.set_stage_timing(True, stages=[s])
        for i in range(n_alone):
            flush_l2()
            step(i)
        stage[s] = (ctx.stage_times()[s][0], n_alone)
        ctx.set_stage_timing(False)
    dom = max((1, 2, 3), key=lambda s: stage[s][0] / max(stage[s][1], 1))
    dom_ms, dom_n = stage[dom]
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps
    value = world * 1000.0 / ms_per_step

    # end to end through the C ABI with host buffers: H2D of the step's image
    # from pinned memory, compute, D2H of chi2, synchronise
    img_host = torch.as_tensor(p.image, dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(args.steps, 200))
    chi2_host = torch.empty(e2e_steps, dtype=torch.float64).pin_memory()
    for i in range(2):
        ctx.chi2_image_host_async(img_host, p.dxy, obs, chi2_host, i, *params[i])
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        ctx.chi2_image_host_async(img_host, p.dxy, obs, chi2_host, i, *params[i % len(params)])
    torch.cuda.synchronize(dev)
    e2e_dt = time.perf_counter() - t0
    e2e_value = world * e2e_steps / e2e_dt

    # plain FP64 single-call path on the same workload (context)
    d64 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa: E731
    obs64 = ctx.register(d64(p.u), d64(p.v), re.double(), im.double(), d64(p.w))
    img64 = d64(p.image)
    ctx.chi2_image(img64, p.dxy, obs64, *params[0], out=out)
    torch.cuda.synchronize(dev)
    s64, e64 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n64 = 5
    s64.record(stream)
    for i in range(n64):
        ctx.chi2_image(img64, p.dxy, obs64, *params[i % len(params)], out=out)
    e64.record(stream)
    torch.cuda.synchronize(dev)
    ms64 = s64.elapsed_time(e64) / n64

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    # roofline of the dominant kernel (largest average launch time)
    rho = float(np.sqrt(np.max(p.u ** 2 + p.v ** 2)))
    Kc, nrw = window(rho, NXY * p.dxy, NXY)
    full = bool(opts.get("full_plane", False))
    kernels = dict(KERNELS_FULL if full else KERNELS)
    if "pb_fwhm" in opts and not full:  # the row pass's beam instance
        kernels[1] = "row_fft3_ldg_kernel<1, 1>"
    if full:
        Kc = full_window_columns(Kc, NXY)
    avg = {s: (stage[s][0] / stage[s][1]) for s in (1, 2, 3) if stage[s][1]}
    alg = algorithmic_bytes(dom, NXY, M_UV, Kc, nrw, beam="pb_fwhm" in opts)
    achieved = alg / (avg[dom] * 1e-3) / 1e9
    peak, peak_kind = peaks()
    traffic = measured_traffic(kernels[dom], full)

    base = None
    re_h, im_h = re.double().cpu().numpy(), im.double().cpu().numpy()
    if world == 1 and args.cpu_evals > 0:
        base = cpu_baseline(p, re_h, im_h, evals=args.cpu_evals)
    accuracy = None
    if world == 1 and not args.no_accuracy:
        accuracy = measure_accuracy(torch, ctx, dev, p, re_h, im_h)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nxy": NXY, "M": M_UV, "l2": "flushed before every step (256 MiB write + 256 MiB read)",
                   "kept_window": {"columns": Kc, "rows": nrw}, "parallelism": f"replicas x{world}",
                   "variant": args.variant},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * NXY * NXY,
                "d2h_bytes_per_step": 8,
                "note": "per step: host image (pinned) -> device on a copy stream into one of two "
                        "staging buffers, overlapping the previous step's compute, and chi2 -> "
                        "pinned host; observation resident; one synchronisation after the steps"},
        "gpu_launches": gpu_launches,
        "roofline": {"bound": "hbm", "kernel": kernels[dom], "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes": alg,
                     "avg_launch_us": 1000 * avg[dom]},
        "stages_us": {STAGES[s]: round(1000 * cal[s][0] / cal[s][1], 2)
                      for s in range(4) if cal[s][1]},
        "kernel_launch_us": {STAGES[s]: round(1000 * avg[s], 2) for s in sorted(avg)},
        "stages_note": "stages_us: per-stage event times from 3 untimed calibration steps "
                       "(each with about 4 us of event overhead); kernel_launch_us: each "
                       "pass timed alone on 10-50 further steps after the timed region "
                       "(L2 flushed, events around that pass's launches only, per step); "
                       "the longest is the roofline's kernel",
        "fp64_plain": {"value": 1000.0 / ms64, "unit": UNIT, "ms_per_step": ms64,
                       "note": "same workload through the float64 entry point, single calls"},
        "flops": fft_equivalent(NXY, value),
        "clocks": clk.summary(),
    }
    if base is not None:
        line["cpu_baseline"] = base
    if accuracy is not None:
        line["accuracy"] = accuracy
    if world == 1 and not args.no_extras:
        extras = set(args.extras.split(","))
        check, pool = None, None
        if not args.no_accuracy:
            from concurrent.futures import ThreadPoolExecutor
            nthr = max(1, host_info()["usable_cpus"] or 1)
            pool = ThreadPoolExecutor(nthr)

            def check(dRA, dDec, PA, problem=None, **kw):
                return oracle_chi2_sharded(p if problem is None else problem, re_h, im_h, dRA,
                                           dDec, PA, pool, nthr, **kw)
        if "plane" in extras:
            line["plane"] = measure_plane(torch, ctx, dev, img, obs, p.dxy, params, flush_l2, out,
                                          oracle_chi2=check)
        if "next" in extras:
            line["next"] = measure_next(torch, ctx, dev, img, obs, p, params, flush_l2, out,
                                        oracle_chi2=check)
        if pool is not None:
            pool.shutdown()
        if "batched" in extras:
            line["batched"] = measure_batched(torch, ctx, dev, flush_l2)
        if "serving" in extras:
            line["serving"] = measure_serving(torch, dev)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# one evaluation split over ranks (uv points sharded, one exchange per step)
# ---------------------------------------------------------------------------
def shard_loop(local_chi2, steps: int, world: int, device, group=None, before=None,
               events=None):
    """Run `steps` sharded evaluations.  local_chi2(i) enqueues this rank's
    partial chi-square of step i and returns it as a 0-d float64 tensor on
    `device`; the partials are all-gathered on the device, one double per rank
    per step, into a [steps, world] buffer, and summed in rank order with
    math.fsum once the loop is over.  before(i) runs ahead of each step (the
    L2 flush); events[i] = (start, end) CUDA events bracket step i's partial
    and exchange.  Returns every step's total."""
    import torch
    import torch.distributed as dist
    gathered = torch.zeros((steps, world), dtype=torch.float64, device=device)
    for i in range(steps):
        if before is not None:
            before(i)
        if events is not None:
            events[i][0].record()
        part = local_chi2(i).reshape(1)
        if world > 1:
            dist.all_gather([gathered[i, r:r + 1] for r in range(world)], part, group=group)
        else:
            gathered[i, 0:1].copy_(part)
        if events is not None:
            events[i][1].record()
    return [math.fsum(row) for row in gathered.cpu().tolist()]


def run_shard(args):
    """One chi2_image evaluation of the workload split over the ranks: every
    rank transforms the same image and evaluates its contiguous share of the
    5e6 uv points; one all-gather of one double per rank per step; the total is
    the same on every rank.  Strong scaling: value = whole evaluations per
    second of the job."""
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_1709_06999_gb300 import Context, shard

    p = make_problem(seed=2)   # the same evaluation on every rank
    ctx = Context(dev.index)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)  # noqa: E731
    img = d(p.image)
    u, v, w = d(p.u), d(p.v), d(p.w)
    model = ctx.sample_image(img, p.dxy, u, v, p.dRA, p.dDec, p.PA)
    re = (model[:, 0] + d(p.noise_re)).contiguous()
    im = (model[:, 1] + d(p.noise_im)).contiguous()
    lo, hi = shard.shard_bounds(u.numel(), world, rank)
    obs = ctx.register(u[lo:hi], v[lo:hi], re[lo:hi], im[lo:hi], w[lo:hi])
    partial = torch.empty((), dtype=torch.float64, device=dev)
    prng = np.random.default_rng(11)
    params = [(float(a), float(b), float(c)) for a, b, c in
              zip(prng.uniform(-0.1, 0.1, 8) * math.pi / 648000,
                  prng.uniform(-0.1, 0.1, 8) * math.pi / 648000, prng.uniform(0, math.pi, 8))]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    flush_rd = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def local_chi2(i):
        ctx.chi2_image(img, p.dxy, obs, *params[i % len(params)], out=partial)
        return partial

    def flush_l2(i):
        flush.zero_()
        flush_rd.sum(dtype=torch.int32)

    shard_loop(local_chi2, args.warmup, world, dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clk = ClockSampler(dev.index).start()
    launches0 = ctx.launch_count()
    clk.begin()
    totals = shard_loop(local_chi2, args.steps, world, dev, before=flush_l2, events=ev)
    torch.cuda.synchronize(dev)
    clk.end()
    clk.stop()
    gpu_launches = ctx.launch_count() - launches0
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    # the same evaluation on one rank's GPU over all points: equal to rounding
    full = None
    if rank == 0:
        obs_all = ctx.register(u, v, re, im, w)
        full = ctx.chi2_image(img, p.dxy, obs_all, *params[0]).item()
    if world > 1:
        torch.distributed.barrier()
    if rank == 0:
        line = {
            "metric": METRIC, "value": 1000.0 / ms_per_step, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nxy": NXY, "M": M_UV,
                       "l2": "flushed before every step (256 MiB write + 256 MiB read)",
                       "parallelism": f"uv points sharded x{world}, one all-gather of one "
                                      "double per rank per step", "mode": "shard"},
            "chi2_step0": totals[0], "chi2_one_gpu_all_points": full,
            "rel_diff_vs_one_gpu": abs(totals[0] - full) / abs(full),
            "gpu_launches": gpu_launches, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-evals", type=int, default=3)
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the per-result errors against the FP64 oracle")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the beam/full-plane, batched (cube, walkers) and serving "
                         "measurements")
    ap.add_argument("--extras", default="plane,next,batched,serving",
                    help="comma-separated extra measurements to run after the bench line "
                         "(plane, next, batched, serving)")
    ap.add_argument("--mode", default="replicas", choices=["replicas", "shard"],
                    help="replicas: independent evaluations per rank (weak scaling, the "
                         "headline); shard: one evaluation's uv points split over the ranks "
                         "(strong scaling)")
    ap.add_argument("--variant", default="plain", choices=sorted(VARIANTS),
                    help="options of the timed chi2_image step (plain: the headline line)")
    ap.add_argument("--clock-sampler", nargs=2, metavar=("TARGET", "PERIOD"),
                    help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.clock_sampler:
        return nvml_sample_loop(args.clock_sampler[0], float(args.clock_sampler[1]))
    args.warmup = max(3, args.warmup)   # the timing rules need at least 3 warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "shard":
        return run_shard(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
