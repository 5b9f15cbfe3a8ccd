"""Steady-flow reference for the chi sweep of Sec. IV.A.1 (steady Re = 20), at a reduced grid:
the full-grid FD oracle (L0) at Re = 20 on 2^6 x 2^7 cells (R = 32, dt = 1e-2, uniform start)
integrated to t = 50, where C_D has settled to 1.5e-5 of its steady value.  Writes C_D, C_L,
the kinetic energy 1/2 mean |v|^2 over the nodes and the velocity magnitude |v| on the grid
(row-major, eta first) to tests/golden/steady_re20_fd.txt, which bench.py --steady-sweep
compares the QTT runs with.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

    python -m oracle.steady_run
"""
from __future__ import annotations

import argparse
import os

import numpy as np

from . import fd

N_ETA, N_XI, R, RE, DT = 6, 7, 32.0, 20.0, 1e-2


def run(time_units: float):
    g = fd.Grid(N_ETA, N_XI, R)
    case = fd.Case(g, RE, DT)
    s = fd.FDSolver(case)
    u = np.ones((g.N_eta, g.N_xi))
    v = np.zeros((g.N_eta, g.N_xi))
    p = np.zeros_like(u)
    for _ in range(int(round(time_units / DT))):
        u, v, p, _, _ = s.step(u, v)
    cd, cl = fd.forces(case, u, v, p)
    shape = (g.N_eta, g.N_xi)
    return np.reshape(u, shape), np.reshape(v, shape), np.reshape(p, shape), float(cd), float(cl)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--time", type=float, default=50.0)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(__file__), "..", "tests", "golden",
                                                  "steady_re20_fd.txt"))
    args = ap.parse_args()
    u, v, p, cd, cl = run(args.time)
    mag = np.sqrt(u * u + v * v)
    with open(args.out, "w") as f:
        f.write(f"# FD oracle (L0), steady cylinder flow: Re = {RE:g}, 2^{N_ETA} x 2^{N_XI} cells, R = {R:g}, "
                f"dt = {DT:g}, uniform start, t = {args.time:g}\n")
        f.write(f"# Written by: python -m oracle.steady_run --time {args.time:g}\n")
        f.write(f"cd {cd:.12e}\ncl {cl:.12e}\nekin {0.5 * float(np.mean(mag * mag)):.12e}\n")
        f.write(f"shape {mag.shape[0]} {mag.shape[1]}\n")
        for row in mag:
            f.write(" ".join(f"{x:.12e}" for x in row) + "\n")
    print(f"C_D {cd:.8f}  C_L {cl:.2e}")


if __name__ == "__main__":
    main()
