"""Long run of the full-grid FD oracle (L0) for the rotating-cylinder sanity pin: Re = 100,
wall rotation rate 1 (eq:rot_bc), grid G1 (2^8 x 2^8 cells, outer diameter 32 D, App. E),
dt = 2e-3 -- the configuration of the FD row of Table II (Sec. IV.B).  It integrates from a
uniform flow with a small seeded perturbation, records C_L and C_D every 10 steps and, from the
last `--window` time units, the mean lift (over whole periods) and the Strouhal number (eq:st).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): the result is written to
tests/golden/table2_fd.txt, which tests/test_oracle.py compares with Table II.

    python -m oracle.table2_run --time 160 --window 60
"""
from __future__ import annotations

import argparse
import os
import time

import numpy as np

from . import fd


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--time", type=float, default=160.0, help="convective time units to integrate")
    ap.add_argument("--window", type=float, default=60.0, help="trailing time units used for C_L and St")
    ap.add_argument("--out", default=os.path.join(os.path.dirname(__file__), "..", "tests", "golden", "table2_fd.txt"))
    args = ap.parse_args()
    g = fd.Grid(8, 8, 32.0)
    case = fd.Case(g, 100.0, 2e-3, rot=1.0)
    s = fd.FDSolver(case)
    rng = np.random.Generator(np.random.PCG64(2024))
    u = 1.0 + 1e-3 * rng.standard_normal((g.N_eta, g.N_xi))
    v = 1e-3 * rng.standard_normal((g.N_eta, g.N_xi))
    nsteps = int(round(args.time / case.dt))
    t_rec, cl_rec, cd_rec = [], [], []
    t0 = time.time()
    for k in range(1, nsteps + 1):
        u, v, p, _, _ = s.step(u, v)
        if k % 10 == 0:
            cd, cl = fd.forces(case, u, v, p)
            t_rec.append(k * case.dt)
            cl_rec.append(cl)
            cd_rec.append(cd)
        if k % 5000 == 0:
            print(f"t = {k * case.dt:.1f}  C_L = {cl_rec[-1]:.4f}  C_D = {cd_rec[-1]:.4f}  ({time.time() - t0:.0f} s)",
                  flush=True)
    t = np.asarray(t_rec); cl = np.asarray(cl_rec); cd = np.asarray(cd_rec)
    w = t >= t[-1] - args.window
    st = fd.strouhal(t[w], cl[w])
    c = cl[w] - np.mean(cl[w])
    up = np.nonzero((c[:-1] < 0) & (c[1:] >= 0))[0]
    lo, hi = up[0], up[-1]                      # whole periods between the first and last crossing
    cl_mean = float(np.mean(cl[w][lo:hi]))
    cd_mean = float(np.mean(cd[w][lo:hi]))
    with open(args.out, "w") as f:
        f.write("# FD oracle (L0), rotating cylinder: Re = 100, rotation rate 1, grid 2^8 x 2^8, R = 32,\n")
        f.write(f"# dt = 2e-3, {args.time:g} time units from uniform flow + 1e-3 seeded noise; means over whole\n")
        f.write(f"# lift periods of the last {args.window:g} time units.  Written by: python -m oracle.table2_run "
                f"--time {args.time:g} --window {args.window:g}\n")
        f.write("# Table II (Sec. IV.B), FD row, for comparison: mean C_L 2.4908, St 0.1663\n")
        f.write(f"mean_cl {cl_mean:.6f}\nst {st:.6f}\nmean_cd {cd_mean:.6f}\n")
    print(f"mean C_L {cl_mean:.5f}  St {st:.5f}  mean C_D {cd_mean:.5f}")


if __name__ == "__main__":
    main()
