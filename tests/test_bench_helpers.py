"""Host arithmetic of bench.py (CPU only): flop conventions, the profile flop
count of a variable band, the oracle sample's flop count, the roofline
fractions and the launch accounting of the refinement loop."""
import importlib.util
import os
import types

import numpy as np

import synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
bench = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(bench)


def _profile_brute(a):
    n = a.shape[0]
    lo = [next((j for j in range(i) if a[i, j] != 0.0), i) for i in range(n)]
    up = [next((i for i in range(j) if a[i, j] != 0.0), j) for j in range(n)]
    work = rs = cs = 0.0
    for k in range(n):
        r = sum(1 for i in range(k + 1, n) if lo[i] <= k)
        c = sum(1 for j in range(k + 1, n) if up[j] <= k)
        work += 2.0 * r * c
        rs += r
        cs += c
    return work, rs, cs


def test_profile_work_matches_brute_force():
    from oracle_pins import variable_profile_dd
    ab, kl, ku = synthetic.laplacian_disc_band(9)
    assert bench.profile_work(ab, kl, ku) == _profile_brute(synthetic.band_to_dense(ab, kl, ku))
    a = variable_profile_dd(90, 11, 7, 5)
    assert bench.profile_work(synthetic.dense_to_band(a, 11, 7), 11, 7) == _profile_brute(a)
    # a uniform band is its own profile: 2 kl ku per step away from the edges
    ab, kl, ku = synthetic.laplacian_band(12)
    w, _, _ = bench.profile_work(ab, kl, ku)
    n = ab.shape[0]
    assert w <= 2.0 * n * kl * ku and w >= 2.0 * (n - 2 * kl) * kl * ku


def test_flop_conventions():
    n, r = 1000, 32
    assert bench.nominal_flops(n, r) == 2.0 * n ** 3 / 3.0 + 2.0 * n * n * r
    # the oracle's first k elimination steps: m divisions and m^2 multiply-adds at step k (m = n-k-1)
    for n in (1, 2, 7, 50):
        full = 2.0 * n ** 3 / 3.0 - n * n / 2.0 - n / 6.0  # the LU count 2n^3/3 - n^2/2 - n/6
        assert abs(bench.oracle_sample_flops(n, n) - full) <= 1e-9 * max(1.0, full)
        count = sum((n - k - 1) + 2 * (n - k - 1) ** 2 for k in range(min(n, 3)))
        assert bench.oracle_sample_flops(n, min(n, 3)) == count
    assert bench.whole_job_gflops(4, 2.0e12, 1000.0) == 8000.0


def test_roofline_fractions():
    args = types.SimpleNamespace(tc_used=True, n=1000)
    peaks = {"bf16_tflops_sustained": 1000.0, "hbm_gbs": 5000.0}
    r = bench.roofline_for("lowp_gemm", 2.0, 1.0e12, 4, peaks, args)
    assert r["bound"] == "tensor" and abs(r["achieved"] - 500.0) < 1e-9 and abs(r["frac"] - 0.5) < 1e-12
    assert r["avg_launch_ms"] == 0.5
    # residual: A (8 n^2 bytes) read once per launch that evaluated a residual
    r = bench.roofline_for("residual", 1.0, 0.0, 11, peaks, args, active=3)
    assert r["bound"] == "hbm" and r["launches"] == 3
    assert abs(r["achieved"] - 3 * 8.0 * 1000 ** 2 / 1e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 5000.0) < 1e-12
    assert bench.roofline_for("panel", 0.0, 1.0, 0, peaks, args) is None
    # launches that did work in a refinement loop of `iters` corrections
    assert bench.active_launches("residual", {"iters": 2}) == 3
    assert bench.active_launches("trsv", {"iters": 2}) == 6
    assert bench.active_launches("panel", {"iters": 2}) is None


def _fake_smi(tmp_path, line, delay="0.05"):
    """A stand-in nvidia-smi that prints `line` every `delay` seconds until killed."""
    d = tmp_path / "bin"
    d.mkdir()
    f = d / "nvidia-smi"
    f.write_text(f"#!/bin/sh\nwhile true; do echo '{line}'; sleep {delay}; done\n")
    f.chmod(0o755)
    return str(d)


def test_clock_sampler_reads_clocks_and_reasons(tmp_path, monkeypatch):
    path = _fake_smi(tmp_path, "2070, 2070, 900.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active")
    monkeypatch.setenv("PATH", path + os.pathsep + os.environ.get("PATH", ""))
    s = bench.ClockSampler(0)
    s.start()
    assert s.lines, "start() returns once the first sample is in"
    import time
    time.sleep(0.2)
    c = s.stop()
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] >= 2 and c["interval_ms"] == bench.ClockSampler.INTERVAL_MS


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    empty = tmp_path / "empty"
    empty.mkdir()
    monkeypatch.setenv("PATH", str(empty))
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
