"""Host-side measurement helpers of bench.py, on the CPU: the periodogram-peak frequency the
transient study reports beside eq:st's zero-crossing count, and the weighted L2 error of the
velocity magnitude against L0 that the fixed-error check reports."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import fd, qtt_ops as Q, step as S, tt  # noqa: E402


def test_periodogram_peak_recovers_a_sine_frequency_under_noise():
    """A lift-like signal sin(2 pi f t) + mean + high-frequency noise over 30 time units: the
    peak frequency is within 1e-3 of f (the zero-crossing count is not, the noise adding
    crossings)."""
    dt, f = 1e-2, 0.1637
    t = dt * np.arange(3000)
    g = np.random.default_rng(3)
    clean = 0.3 + 0.6 * np.sin(2 * np.pi * f * t + 0.4)
    noisy = clean + 0.05 * np.sin(2 * np.pi * 7.3 * t) + 0.02 * g.standard_normal(t.size)
    assert abs(bench.periodogram_peak(clean, dt) - f) < 1e-3
    assert abs(bench.periodogram_peak(noisy, dt) - f) < 1e-3
    assert abs(fd.strouhal(t, clean - 0.3) - f) < 1e-3
    assert abs(fd.strouhal(t, noisy - 0.3) - f) > 1e-2


def test_l0_errors_on_oracle_steps():
    """l0_errors: the GPU inputs replaced by the oracle's own first step give identical errors
    for 'GPU' and oracle (ratio 1, distance 0), and a step's error against L0 from the same
    encoded state is small at full rank (the QTT step at full rank equals L0)."""
    cfg = dict(bench.WORKLOAD)
    cfg.update(n_eta=3, n_xi=3, chi=8, apply="sketch", poisson_warm="previous",
               mom=(6, 1e-12, 400, 1e-12, 0.1), poi=(12, 1e-12, 600, 1e-12, 0.1))
    ops, (u, v, p), o = bench.oracle_start(cfg)
    un, vn, pn, _ = S.step(ops, u, v, p, o)
    r = bench.l0_errors(cfg, [tt.full(un), tt.full(vn)], (un, vn, pn), [tt.full(un), tt.full(vn)], 1)
    assert r["first_step"]["ratio"] == 1.0 and r["first_step"]["gpu_vs_oracle_L1"] == 0.0
    assert r["first_step"]["ok"]
    assert r["first_step"]["gpu"] < 1e-9          # 2^6 cells at chi = 8: full rank, equals L0
    assert r["after_timed_window"]["gpu"] == r["first_step"]["gpu"]
    assert r["L0_fd_s_per_step"] > 0.0 and r["L0_cores"] >= 1
