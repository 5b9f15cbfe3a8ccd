"""Transient-flow reference for the Strouhal-versus-chi study of Sec. IV.A.2 (vortex shedding
behind the non-rotating cylinder), at a reduced grid: the full-grid FD oracle (L0) at Re = 100
on 2^6 x 2^7 cells (R = 32, dt = 1e-2), started from the seeded synthetic wake state
(paper_2507_05222_gb300.inputs.wake_field, seed 7; its asymmetric packets trigger the
shedding in place of App. G's perturbation), integrated to t = 60.  Writes the Strouhal number
of the lift (eq:st, zero crossings of C_L over t in [30, 60], and the periodogram's peak), the mean drag and the lift
amplitude over that window to tests/golden/transient_re100_fd.txt, which
bench.py --transient-sweep compares the QTT runs with.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

    python -m oracle.transient_run
"""
from __future__ import annotations

import argparse
import os

import numpy as np

from . import fd

N_ETA, N_XI, R, RE, DT, SEED = 6, 7, 32.0, 100.0, 1e-2, 7
T_END, T_WINDOW = 60.0, 30.0


def run(t_end: float = T_END, t_window: float = T_WINDOW):
    from paper_2507_05222_gb300 import inputs
    g = fd.Grid(N_ETA, N_XI, R)
    case = fd.Case(g, RE, DT)
    s = fd.FDSolver(case)
    u0, v0 = inputs.wake_field(N_ETA, N_XI, SEED)
    u, v = u0.ravel(), v0.ravel()
    ts, cds, cls = [], [], []
    for k in range(int(round(t_end / DT))):
        u, v, p, _, _ = s.step(u, v)
        cd, cl = fd.forces(case, u, v, p)
        ts.append((k + 1) * DT); cds.append(cd); cls.append(cl)
    ts, cds, cls = np.asarray(ts), np.asarray(cds), np.asarray(cls)
    w = ts >= t_window
    return dict(st=fd.strouhal(ts[w], cls[w]), st_spectral=spectral_st(cls[w], DT), cd_mean=float(np.mean(cds[w])),
                cl_amp=float(np.ptp(cls[w])), cl_end=float(cls[-1]))


def spectral_st(cl, dt):
    """Frequency of the largest peak of the (Hann-windowed) periodogram of C_L, refined by a
    parabola through the log-power of the peak bin and its neighbours (D = U = 1, so this is a
    Strouhal number); unlike the zero-crossing count it is not moved by high-frequency noise."""
    x = np.asarray(cl) - np.mean(cl)
    pw = np.abs(np.fft.rfft(x * np.hanning(len(x)))) ** 2
    k = int(np.argmax(pw[1:]) + 1)
    off = 0.0
    if 1 <= k < len(pw) - 1 and min(pw[k - 1], pw[k], pw[k + 1]) > 0:
        a, b, c = np.log(pw[k - 1]), np.log(pw[k]), np.log(pw[k + 1])
        off = 0.5 * (a - c) / (a - 2 * b + c)
    return float((k + off) / (len(x) * dt))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(__file__), "..", "tests", "golden",
                                                  "transient_re100_fd.txt"))
    args = ap.parse_args()
    r = run()
    with open(args.out, "w") as f:
        f.write(f"# FD oracle (L0), vortex shedding: Re = {RE:g}, 2^{N_ETA} x 2^{N_XI} cells, R = {R:g}, dt = {DT:g}, "
                f"wake_field seed {SEED} start, t = {T_END:g}; statistics over t >= {T_WINDOW:g}\n")
        f.write("# Written by: python -m oracle.transient_run\n")
        for k in ("st", "st_spectral", "cd_mean", "cl_amp", "cl_end"):
            f.write(f"{k} {r[k]:.12e}\n")
    print(r)


if __name__ == "__main__":
    main()
