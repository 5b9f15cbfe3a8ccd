"""L1 oracle: one QTT fractional step (Sec. III.C) from the L1 algebra, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The step (same sequence as the CUDA library, written independently):

1. convective derivatives, each an MPO-MPS product rounded to chi (Sec. II.A.2):
   dxu = round(D_x u), dzu = round(D_z u), dxv = round(D_x v), dzv = round(D_z v);
2. explicit right-hand sides (eq:intermediate_vel_eq), one variational fit each
   (Table I), warm-started from u (v):
   rhs_u = u - dt [u (.) (dxu + bcx_u) + v (.) (dzu + bcz_u)],  rhs_v likewise;
3. implicit momentum solves by ALS with the |J|-weighted SPD operator
   H = |J| (I - dt/Re Lap_h):  H u* = |J| (.) rhs_u + dt/Re |J| bcLap_u  (warm start u);
4. pressure Poisson by ALS (eq:Poisson with the Jacobian weighting of Sec. III.C):
   (-|J| Lap_h^p) p = -|J| (.) (D_x u* + D_z v* + bc_div) / dt   (warm start p^m);
   both solves sweep under the true-residual stop rule of ``tt.als`` (options ``SolveOpts``);
5. projection, one fit each (warm start u*, v*):  u = u* - dt D_x^p p,  v = v* - dt D_z^p p.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import tt
from .qtt_ops import Ops


@dataclass
class SolveOpts:
    """Options of one ALS solve (stop rule of ``tt.als``)."""
    max_sweeps: int
    rel_tol: float
    cg_max_iter: int
    cg_tol: float = 1e-2
    stall: float = 0.1


@dataclass
class StepOpts:
    chi: int
    fit_sweeps: int = 1
    mom: SolveOpts = field(default_factory=lambda: SolveOpts(6, 1e-8, 100))
    poi: SolveOpts = field(default_factory=lambda: SolveOpts(12, 1e-10, 500))
    # Poisson warm start: "previous" (p^m, the reading of Sec. III.C) or "extrapolated"
    # (2 p^m - p^(m-1), fitted at the bonds of p^m from p^m with fit_sweeps sweeps)
    poisson_warm: str = "previous"


def _nz(terms):
    return [t for t in terms if all(x is not None for x in t[2:])]


def step(ops: Ops, u, v, p, o: StepOpts, p_prev=None):
    """One fractional step; p_prev (the pressure of the step before; None right after the state
    was set, when the Poisson solve starts from p) feeds the extrapolated warm start."""
    dt, Re = ops.dt, ops.Re
    chi = o.chi
    dxu = tt.round_tt(tt.mpo_mps(ops.Dx, u), chi)
    dzu = tt.round_tt(tt.mpo_mps(ops.Dz, u), chi)
    dxv = tt.round_tt(tt.mpo_mps(ops.Dx, v), chi)
    dzv = tt.round_tt(tt.mpo_mps(ops.Dz, v), chi)
    rhs_u = tt.fit(_nz([("vec", 1.0, u), ("had", -dt, u, dxu), ("had", -dt, u, ops.bcx_u),
                        ("had", -dt, v, dzu), ("had", -dt, v, ops.bcz_u)]), u, o.fit_sweeps)
    rhs_v = tt.fit(_nz([("vec", 1.0, v), ("had", -dt, u, dxv), ("had", -dt, u, ops.bcx_v),
                        ("had", -dt, v, dzv), ("had", -dt, v, ops.bcz_v)]), v, o.fit_sweeps)
    k = dt / Re
    m, q = o.mom, o.poi
    us, iu = tt.als(ops.H, _nz([("mpo", 1.0, ops.Jdiag, rhs_u), ("vec", k, ops.JbcLap_u)]), u,
                    m.max_sweeps, m.cg_max_iter, m.cg_tol, m.rel_tol, m.stall)
    vs, iv = tt.als(ops.H, _nz([("mpo", 1.0, ops.Jdiag, rhs_v), ("vec", k, ops.JbcLap_v)]), v,
                    m.max_sweeps, m.cg_max_iter, m.cg_tol, m.rel_tol, m.stall)
    p0 = p
    if o.poisson_warm == "extrapolated" and p_prev is not None:
        p0 = tt.fit([("vec", 2.0, p), ("vec", -1.0, p_prev)], p, o.fit_sweeps)
    pn, ip = tt.als(ops.Ap, _nz([("mpo", 1.0, ops.Px, us), ("mpo", 1.0, ops.Pz, vs),
                                 ("vec", 1.0, ops.bcdiv_w)]), p0, q.max_sweeps, q.cg_max_iter, q.cg_tol,
                    q.rel_tol, q.stall)
    un = tt.fit([("vec", 1.0, us), ("mpo", -dt, ops.Dxp, pn)], us, o.fit_sweeps)
    vn = tt.fit([("vec", 1.0, vs), ("mpo", -dt, ops.Dzp, pn)], vs, o.fit_sweeps)
    info = dict(u=iu, v=iv, p=ip, cg_u=iu["cg_iters"], cg_v=iv["cg_iters"], cg_p=ip["cg_iters"])
    return un, vn, pn, info


def padded(cores, chi: int, seed_cores):
    """Embed an MPS into the bond profile min(2^k, 2^(n-k), chi): the missing rows and
    columns of each core are filled from ``seed_cores`` (small seeded noise drawn by the
    caller), the existing block is kept.  Used for warm starts of lower rank."""
    out = []
    for c, s in zip(cores, seed_cores):
        r0, d, r1 = s.shape
        x = s.copy()
        a, b = min(r0, c.shape[0]), min(r1, c.shape[2])
        x[:a, :, :b] = c[:a, :, :b]
        out.append(x)
    return out
