"""bench.py on the CPU: the reference arm's JSON line (the FP64 oracle timed
on the host) and the host-side helpers behind the native line's roofline.
No GPU needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_line():
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    line = json.loads(p.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["steps"] == 1 and line["warmup"] == 3
    assert line["unit"] == "evals/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "evals/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["nxy"] == 4096 and line["config"]["M"] == 5_000_000


def test_window_rule():
    # e = rho * S cells: k = floor(e) + 3 cells of margin, Kc = k + 1 columns
    # and rows N/2 - k .. N/2 + k, clipped to the half spectrum
    assert bench.window(57.5, 1.0, 4096) == (61, 121)
    assert bench.window(0.0, 1.0, 64) == (4, 7)
    assert bench.window(100.0, 1.0, 64) == (33, 64)        # whole half spectrum
    assert bench.window(31.0, 1.0, 64) == (33, 64)         # margins clipped
    assert bench.window(float("nan"), 1.0, 64) == (33, 64)


def test_full_window_columns():
    assert bench.full_window_columns(61, 4096) == 121       # u from -60 to 60
    assert bench.full_window_columns(33, 64) == 64          # node range -32 .. 31
    assert bench.full_window_columns(2, 64) == 3


def test_algorithmic_bytes():
    N, M, Kc, nrw = 4096, 5_000_000, 61, 121
    assert bench.algorithmic_bytes(1, N, M, Kc, nrw) == 4 * N * N + 8 * N * Kc
    assert bench.algorithmic_bytes(1, N, M, Kc, nrw, beam=True) == 4 * N * N + 8 * N * Kc + 8 * N
    assert bench.algorithmic_bytes(2, N, M, Kc, nrw) == 8 * N * Kc + 8 * nrw * Kc
    # the headline gather: 20 B per point plus the window once
    assert bench.algorithmic_bytes(3, N, M, Kc, nrw) == 100_059_048


def test_cpu_baseline_fields(monkeypatch):
    import time
    monkeypatch.setattr(bench, "oracle_eval", lambda p, re, im: time.sleep(0.01))
    monkeypatch.setattr(bench, "oracle_eval_threads",
                        lambda p, re, im, pool, n: time.sleep(0.005))
    b = bench.cpu_baseline(None, None, None, 3)
    assert b["kind"] == "oracle" and b["unit"] == "evals/s"
    assert b["cores"] == b["host"]["usable_cpus"] >= 1
    s = b["seconds_per_eval"]
    assert 0.004 < s["min"] <= s["median"] < 1.0
    assert abs(b["value"] - 1.0 / s["median"]) < 1e-9
    one = b["single_thread"]
    assert one["cores"] == 1 and one["evals"] == 3
    assert 0.009 < one["seconds_per_eval"]["min"] <= one["seconds_per_eval"]["median"] < 1.0
    assert set(b["host"]) == {"cpu_model", "nproc", "usable_cpus"}


def test_host_info():
    h = bench.host_info()
    assert h["nproc"] >= 1 and 1 <= h["usable_cpus"] <= h["nproc"]
    assert h["cpu_model"] is None or isinstance(h["cpu_model"], str)


def test_clock_samples_summary():
    t0 = 1000.0
    lines = [f"{t0 - 0.01} 1980 2070 300.0 1",       # before the region, idle
             f"{t0 + 0.0002} 2070 2070 700.5 0",
             f"{t0 + 0.0007} 2055 2070 900.0 4",      # sw_power_cap
             "garbage line",
             f"{t0 + 0.05} 2070 2070 200.0 1"]        # after the region
    s = bench.parse_clock_samples(lines, t0, t0 + 0.001)
    assert s["samples"] == 2 and s["window"] == "timed region"
    assert s["sm_mhz"] == 2062.5 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["power_w_max"] == 900.0
    # a region shorter than the sampling period: the neighbouring samples stand in
    s = bench.parse_clock_samples(lines, t0 + 0.001, t0 + 0.0011)
    assert s["samples"] == 2 and s["window"].startswith("nearest")
    # hardware slowdown bits are reported by name
    s = bench.parse_clock_samples([f"{t0} 1500 2070 1400.0 {0x8 | 0x40}"], t0, t0)
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    assert bench.parse_clock_samples([], 0, 1)["reasons"] == ["unavailable"]


def test_fft_equivalent():
    f = bench.fft_equivalent(4096, 1000.0)
    assert abs(f["fft_gflop_per_eval"] - 2.5 * 4096 ** 2 * 24 / 1e9) < 1e-12
    assert abs(f["fft_equivalent_tflop_per_s"] - f["fft_gflop_per_eval"]) < 1e-12


def test_sharded_oracle_chi2_is_the_oracle():
    """The bench states the beam, full-plane and multi-source results against
    oracle_chi2_sharded: it must be the oracle's own chi-square of that
    evaluation (chi2_image with pb_fwhm / full_plane, chi2_image_multi), the
    sharding changing only the last bits of the sum."""
    import math
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    from paper_1709_06999_gb300 import synth
    p = synth.small_image_problem(nxy=64, M=5003, seed=3)
    re, im = p.noise_re + 0.1, p.noise_im - 0.2
    fwhm = 0.4 * 64 * p.dxy
    with ThreadPoolExecutor(3) as pool:
        for kw in ({}, {"pb_fwhm": fwhm}, {"full_plane": True},
                   {"pb_fwhm": fwhm, "full_plane": True}):
            got = bench.oracle_chi2_sharded(p, re, im, p.dRA, p.dDec, p.PA, pool, 3, **kw)
            ref = oracle.chi2_image(p.image, p.dxy, p.u, p.v, re, im, p.w, p.dRA, p.dDec, p.PA,
                                    **kw)
            assert math.isclose(got, ref, rel_tol=1e-14), (kw, got, ref)
        copies = [(0.7, 1e-7, -2e-7), (0.3, -3e-7, 1e-7), (1.1, 0.0, 2e-7)]
        got = bench.oracle_chi2_sharded(p, re, im, 0.0, 0.0, p.PA, pool, 3, copies=copies)
        amp, dra, ddec = (list(c) for c in zip(*copies))
        ref = oracle.chi2_image_multi(p.image, p.dxy, p.u, p.v, re, im, p.w, dra, ddec, amp, p.PA)
        assert math.isclose(got, ref, rel_tol=1e-14), (got, ref)
        # a different beam or offset moves it: the check is not blind
        off = bench.oracle_chi2_sharded(p, re, im, p.dRA, p.dDec, p.PA, pool, 3,
                                        pb_fwhm=0.5 * fwhm)
        assert not math.isclose(off, ref, rel_tol=1e-6)
