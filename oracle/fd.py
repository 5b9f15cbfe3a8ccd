"""L0 oracle: the classical full-grid finite-difference fractional step, in FP64.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg do.

What it computes (cited by section / equation of arXiv:2507.05222):

* the log-polar O-grid of App. E (eq:mesh) with the interior nodes of eq:defetaxi,
  eta_i = (i+1) d_eta, xi_j = j d_xi, d_eta = 1/(N_eta+1), d_xi = 1/N_xi, ghost rows
  i = -1 (the cylinder wall) and i = N_eta (the far field);
* analytic metric terms of that mapping and the curvilinear derivatives of
  eq:curviliner-deriavtive and the seven-term Laplacian (App. A);
* second-order central stencils (App. A), periodic in xi;
* ghost-point boundary conditions (Sec. III.A, eq:bound): Dirichlet velocity at both
  ghost rows, Neumann pressure at the wall (ghost p_{-1} = p_0), Dirichlet p = 0 at the
  far field;
* one Chorin step (Sec. III.C, eq:intermediate_vel_eq, eq:Poisson and the correction)
  with sparse direct solves;
* lift and drag from the wall stress (App. F, eq:liftdrag) and the Strouhal number
  from lift zero crossings (eq:st).

Readings where the paper is silent or garbled: the wall is ghost row i=-1 (App. E); the
metric terms are analytic; the Neumann pressure ghost is p_{-1}=p_0; the wall stress uses
the outward cylinder normal and ds = (D/2) 2 pi d_xi.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


@dataclass
class Grid:
    n_eta: int
    n_xi: int
    R: float          # D_outer / D  (App. E)
    D: float = 1.0

    @property
    def N_eta(self) -> int:
        return 2 ** self.n_eta

    @property
    def N_xi(self) -> int:
        return 2 ** self.n_xi

    @property
    def deta(self) -> float:
        return 1.0 / (self.N_eta + 1)

    @property
    def dxi(self) -> float:
        return 1.0 / self.N_xi

    @property
    def lnR(self) -> float:
        return float(np.log(self.R))

    def eta(self, i):
        """eta at row i (i = -1 .. N_eta allowed), eq:discretization_unit_square."""
        return (np.asarray(i, dtype=np.float64) + 1.0) * self.deta

    def r(self, i):
        """Radius of row i: (D/2) R^eta (App. E, eq:mesh)."""
        return 0.5 * self.D * self.R ** self.eta(i)

    def theta(self, j):
        return 2.0 * np.pi * np.asarray(j, dtype=np.float64) * self.dxi

    def nodes(self, ghosts: bool = False):
        """(r, theta) arrays of shape (rows, N_xi); rows include the two ghost rows if asked."""
        i = np.arange(-1, self.N_eta + 1) if ghosts else np.arange(self.N_eta)
        j = np.arange(self.N_xi)
        return np.meshgrid(self.r(i), self.theta(j), indexing="ij")

    def xz(self, ghosts: bool = False):
        rr, th = self.nodes(ghosts)
        return rr * np.cos(th), rr * np.sin(th)

    def h_min(self) -> float:
        """Smallest of the first normal spacing and the wall arc length (Sec. IV, h_min)."""
        normal = self.r(0) - self.r(-1)
        arc = 2.0 * np.pi * self.r(-1) * self.dxi
        return float(min(normal, arc))


def metrics(g: Grid, ghosts: bool = False) -> dict:
    """Analytic metric terms of x = r cos(2 pi xi), z = r sin(2 pi xi), r = (D/2) R^eta.

    Returns the partial derivatives of the mapping, J, g11, g22, g12 (App. A) and the
    coefficients of d/dx, d/dz (eq:curviliner-deriavtive) and of the seven-term
    Laplacian, all at nodes (ghost rows included if asked).
    """
    rr, th = g.nodes(ghosts)
    lnR = g.lnR
    x_xi = -2.0 * np.pi * rr * np.sin(th)
    z_xi = 2.0 * np.pi * rr * np.cos(th)
    x_eta = lnR * rr * np.cos(th)
    z_eta = lnR * rr * np.sin(th)
    J = x_xi * z_eta - x_eta * z_xi
    g11 = x_xi ** 2 + z_xi ** 2
    g22 = x_eta ** 2 + z_eta ** 2
    g12 = x_xi * x_eta + z_xi * z_eta
    out = dict(J=J, g11=g11, g22=g22, g12=g12,
               cx_xi=z_eta / J, cx_eta=-z_xi / J,      # d/dx = (z_eta d_xi - z_xi d_eta)/J
               cz_xi=-x_eta / J, cz_eta=x_xi / J)      # d/dz = (-x_eta d_xi + x_xi d_eta)/J
    # Seven-term Laplacian coefficients (App. A).  For this mapping g22/J = -lnR/(2 pi)
    # and g11/J = -2 pi/lnR are constants and g12 = 0, so the derivatives of the g/J
    # ratios vanish identically; they are written out as the closed-form zeros.
    zero = np.zeros_like(J)
    out.update(L_xi=zero, L_xixi=(g22 / J) / J, L_eta=zero, L_etaeta=(g11 / J) / J,
               L_xieta=-2.0 * (g12 / J) / J)
    return out


# --------------------------------------------------------------------------------------
# Stencils on the extended grid (ghost rows included) and ghost elimination
# --------------------------------------------------------------------------------------

def _ext_index(g: Grid, i, j):
    """Flat index in the extended layout: rows i = -1..N_eta, row-major."""
    return (np.asarray(i) + 1) * g.N_xi + (np.asarray(j) % g.N_xi)


def _int_index(g: Grid, i, j):
    return np.asarray(i) * g.N_xi + (np.asarray(j) % g.N_xi)


def stencil(g: Grid, kind: str) -> sp.csr_matrix:
    """Central second-order stencil (App. A) mapping extended-grid values to interior rows.

    kind in {"xi", "eta", "xixi", "etaeta", "xieta"}.  xi is periodic.
    """
    Ne, Nx = g.N_eta, g.N_xi
    ii, jj = np.meshgrid(np.arange(Ne), np.arange(Nx), indexing="ij")
    ii = ii.ravel(); jj = jj.ravel()
    row = _int_index(g, ii, jj)
    de, dx = g.deta, g.dxi
    if kind == "xi":
        taps = [(0, +1, 1 / (2 * dx)), (0, -1, -1 / (2 * dx))]
    elif kind == "eta":
        taps = [(+1, 0, 1 / (2 * de)), (-1, 0, -1 / (2 * de))]
    elif kind == "xixi":
        taps = [(0, +1, 1 / dx ** 2), (0, 0, -2 / dx ** 2), (0, -1, 1 / dx ** 2)]
    elif kind == "etaeta":
        taps = [(+1, 0, 1 / de ** 2), (0, 0, -2 / de ** 2), (-1, 0, 1 / de ** 2)]
    elif kind == "xieta":
        c = 1 / (4 * dx * de)
        taps = [(+1, +1, c), (+1, -1, -c), (-1, +1, -c), (-1, -1, c)]
    else:
        raise ValueError(kind)
    rows, cols, vals = [], [], []
    for di, dj, w in taps:
        rows.append(row)
        cols.append(_ext_index(g, ii + di, jj + dj))
        vals.append(np.full(row.shape, w))
    n_ext = (Ne + 2) * Nx
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(Ne * Nx, n_ext))


def lift(g: Grid, wall: str, far: str):
    """Affine ghost rule f_ext = A f + c(ghost values), as (A, C_wall, C_far).

    wall/far in {"dirichlet", "neumann"}.  Dirichlet: ghost = prescribed value (enters
    through c).  Neumann at the wall: ghost p_{-1} = p_0 (first-order image of the
    interior row, the wall sitting at the ghost node).
    """
    Ne, Nx = g.N_eta, g.N_xi
    n_ext, n_int = (Ne + 2) * Nx, Ne * Nx
    j = np.arange(Nx)
    rows = [_ext_index(g, np.repeat(np.arange(Ne), Nx), np.tile(j, Ne))]
    cols = [np.arange(n_int)]
    if wall == "neumann":
        rows.append(_ext_index(g, -1, j)); cols.append(_int_index(g, 0, j))
    elif wall != "dirichlet":
        raise ValueError(wall)
    if far == "neumann":
        rows.append(_ext_index(g, Ne, j)); cols.append(_int_index(g, Ne - 1, j))
    elif far != "dirichlet":
        raise ValueError(far)
    r = np.concatenate(rows); c = np.concatenate(cols)
    A = sp.csr_matrix((np.ones(r.shape), (r, c)), shape=(n_ext, n_int))
    Cw = sp.csr_matrix((np.ones(Nx), (_ext_index(g, -1, j), j)), shape=(n_ext, Nx))
    Cf = sp.csr_matrix((np.ones(Nx), (_ext_index(g, Ne, j), j)), shape=(n_ext, Nx))
    if wall == "neumann":
        Cw = Cw * 0.0
    if far == "neumann":
        Cf = Cf * 0.0
    return A, Cw, Cf


def operators(g: Grid, bc: str):
    """Curvilinear operators for a field with boundary rule ``bc``.

    bc = "velocity": Dirichlet ghosts at both ends (values supplied per call).
    bc = "pressure": Neumann wall (p_{-1} = p_0), Dirichlet far field p = 0.
    Returns dict name -> (M, Bw, Bf) with op(f) = M f + Bw g_wall + Bf g_far.
    """
    m = metrics(g)
    wall, far = ("dirichlet", "dirichlet") if bc == "velocity" else ("neumann", "dirichlet")
    A, Cw, Cf = lift(g, wall, far)
    S = {k: stencil(g, k) for k in ("xi", "eta", "xixi", "etaeta", "xieta")}

    def diag(a):
        return sp.diags(np.ravel(a))

    ext_ops = {
        "Dx": diag(m["cx_xi"]) @ S["xi"] + diag(m["cx_eta"]) @ S["eta"],
        "Dz": diag(m["cz_xi"]) @ S["xi"] + diag(m["cz_eta"]) @ S["eta"],
        "Lap": (diag(m["L_xi"]) @ S["xi"] + diag(m["L_xixi"]) @ S["xixi"]
                + diag(m["L_eta"]) @ S["eta"] + diag(m["L_etaeta"]) @ S["etaeta"]
                + diag(m["L_xieta"]) @ S["xieta"]),
    }
    return {k: ((E @ A).tocsr(), (E @ Cw).tocsr(), (E @ Cf).tocsr()) for k, E in ext_ops.items()}


def apply_op(op, f, g_wall=None, g_far=None):
    M, Bw, Bf = op
    out = M @ np.ravel(f)
    if g_wall is not None:
        out = out + Bw @ np.broadcast_to(g_wall, (Bw.shape[1],))
    if g_far is not None:
        out = out + Bf @ np.broadcast_to(g_far, (Bf.shape[1],))
    return out


# --------------------------------------------------------------------------------------
# Case and the Chorin step
# --------------------------------------------------------------------------------------

@dataclass
class Case:
    grid: Grid
    Re: float
    dt: float
    rot: float = 0.0          # wall rotation rate (eq:rot_bc); 0 = stationary cylinder
    u_inf: float = 1.0

    def wall_velocity(self):
        """Wall ghost values (u_Gamma, v_Gamma) per xi node, eq:rot_bc."""
        th = self.grid.theta(np.arange(self.grid.N_xi))
        return self.rot * np.sin(th), -self.rot * np.cos(th)

    def far_velocity(self):
        Nx = self.grid.N_xi
        return np.full(Nx, self.u_inf), np.zeros(Nx)


class PeriodicXiSolver:
    """Direct solve of M x = b for a grid operator M that is invariant under shifts along the
    periodic xi direction (the coefficients of the momentum operator and of the pressure
    Laplacian depend on eta only: J, g11/J, g22/J of App. A's analytic metric, g12 = 0), with
    couplings to xi neighbours s in {-1, 0, +1} only.  M is block-circulant: with
    B_s[i, i'] = M[(i, j), (i', j + s)], the discrete Fourier transform along xi turns it into
    one tridiagonal eta system per mode m, sum_s B_s exp(2 pi i s m / N_xi), solved by a banded
    LU; this is the same linear system as the sparse solve, in O(N log N)."""

    def __init__(self, M: sp.spmatrix, g: Grid):
        Ne, Nx = g.N_eta, g.N_xi
        M = M.tocsr()
        self.Ne, self.Nx = Ne, Nx
        B = {s: np.zeros((Ne, Ne)) for s in (-1, 0, 1)}
        rows = np.arange(Ne) * Nx                      # (i, j = 0)
        sub = M[rows]
        coo = sub.tocoo()
        for r, c, v in zip(coo.row, coo.col, coo.data):
            ip, jp = divmod(int(c), Nx)
            s = jp if jp <= Nx // 2 else jp - Nx
            if s not in B:
                raise ValueError("operator couples xi neighbours beyond +-1")
            B[s][r, ip] += v
        for s_, Bs in B.items():
            off = Bs - np.diag(np.diag(Bs)) - np.diag(np.diag(Bs, 1), 1) - np.diag(np.diag(Bs, -1), -1)
            if np.abs(off).max() > 0:
                raise ValueError("eta coupling beyond the tridiagonal band")
        w = np.exp(2j * np.pi * np.arange(Nx) / Nx)      # mode m: shift s contributes w_m^s
        self.ab = np.zeros((Nx, 3, Ne), dtype=complex)   # solve_banded layout per mode
        for s_, Bs in B.items():
            f = (w ** s_)[:, None]
            self.ab[:, 0, 1:] += f * np.diag(Bs, 1)
            self.ab[:, 1, :] += f * np.diag(Bs)
            self.ab[:, 2, :-1] += f * np.diag(Bs, -1)

    def solve(self, b):
        from scipy.linalg import solve_banded
        bh = np.fft.fft(np.reshape(b, (self.Ne, self.Nx)), axis=1)
        xh = np.empty_like(bh)
        for k in range(self.Nx):
            xh[:, k] = solve_banded((1, 1), self.ab[k], bh[:, k])
        return np.real(np.fft.ifft(xh, axis=1)).ravel()


class FDSolver:
    """Full-grid fractional step (Sec. III.C) with cached direct solvers of the momentum and
    pressure systems: sparse LU (direct="lu") or the exact Fourier-in-xi, tridiagonal-in-eta
    solve of the same matrices (direct="fft", for grids where a sparse LU would not fit)."""

    def __init__(self, case: Case, direct: str = "lu"):
        self.case = case
        g = case.grid
        self.vel = operators(g, "velocity")
        self.pre = operators(g, "pressure")
        n = g.N_eta * g.N_xi
        I = sp.identity(n, format="csc")
        self.H = (I - (case.dt / case.Re) * self.vel["Lap"][0]).tocsc()
        self.Lp = self.pre["Lap"][0].tocsc()
        if direct == "lu":
            self._Hlu = spla.splu(self.H)
            self._Plu = spla.splu(self.Lp)
        elif direct == "fft":
            self._Hlu = PeriodicXiSolver(self.H, g)
            self._Plu = PeriodicXiSolver(self.Lp, g)
        else:
            raise ValueError(direct)

    def grad_div(self, u, v):
        c = self.case
        uw, vw = c.wall_velocity()
        uf, vf = c.far_velocity()
        return (apply_op(self.vel["Dx"], u, uw, uf) + apply_op(self.vel["Dz"], v, vw, vf))

    def step(self, u, v, p=None):
        """One step: returns (u_new, v_new, p_new, u_star, v_star), all flattened."""
        c = self.case
        u = np.ravel(u); v = np.ravel(v)
        uw, vw = c.wall_velocity()
        uf, vf = c.far_velocity()
        Dxu = apply_op(self.vel["Dx"], u, uw, uf)
        Dzu = apply_op(self.vel["Dz"], u, uw, uf)
        Dxv = apply_op(self.vel["Dx"], v, vw, vf)
        Dzv = apply_op(self.vel["Dz"], v, vw, vf)
        # eq:intermediate_vel_eq: (1 - dt/Re Lap) v* = v - dt (v.grad) v, the ghost part of
        # Lap v* moved to the right-hand side.
        k = c.dt / c.Re
        Lap_u_bc = apply_op(self.vel["Lap"], np.zeros_like(u), uw, uf)
        Lap_v_bc = apply_op(self.vel["Lap"], np.zeros_like(v), vw, vf)
        rhs_u = u - c.dt * (u * Dxu + v * Dzu) + k * Lap_u_bc
        rhs_v = v - c.dt * (u * Dxv + v * Dzv) + k * Lap_v_bc
        us = self._Hlu.solve(rhs_u)
        vs = self._Hlu.solve(rhs_v)
        # eq:Poisson: Lap p = div(v*)/dt (pressure ghosts: Neumann wall, p = 0 outside).
        b = (apply_op(self.vel["Dx"], us, uw, uf) + apply_op(self.vel["Dz"], vs, vw, vf)) / c.dt
        p_new = self._Plu.solve(b)
        un = us - c.dt * apply_op(self.pre["Dx"], p_new)
        vn = vs - c.dt * apply_op(self.pre["Dz"], p_new)
        return un, vn, p_new, us, vs


# --------------------------------------------------------------------------------------
# Diagnostics
# --------------------------------------------------------------------------------------

def forces(case: Case, u, v, p):
    """(C_D, C_L) from the wall stress (App. F, eq:liftdrag).

    Wall derivatives: one-sided second order in eta from the wall ghost row and rows
    0, 1; central in xi along the wall.  p on the wall = p_0 (Neumann ghost).  Stress
    sigma = -(p + 2/(3 Re) div v) I + (1/Re)(grad v + grad v^T); traction sigma . n with
    the unit normal n = (cos th, sin th) pointing from the cylinder into the fluid;
    ds = (D/2) 2 pi d_xi.  C = 2 F (rho = U = D = 1).
    """
    g = case.grid
    Nx = g.N_xi
    u = np.reshape(u, (g.N_eta, Nx)); v = np.reshape(v, (g.N_eta, Nx)); p = np.reshape(p, (g.N_eta, Nx))
    uw, vw = case.wall_velocity()
    th = g.theta(np.arange(Nx))
    rw = g.r(-1)
    lnR = g.lnR

    def d_eta(fw, f0, f1):
        return (-3.0 * fw + 4.0 * f0 - f1) / (2.0 * g.deta)

    def d_xi(fw):
        return (np.roll(fw, -1) - np.roll(fw, 1)) / (2.0 * g.dxi)

    cx_xi = -np.sin(th) / (2 * np.pi * rw); cx_eta = np.cos(th) / (lnR * rw)
    cz_xi = np.cos(th) / (2 * np.pi * rw); cz_eta = np.sin(th) / (lnR * rw)
    ue, ux = d_eta(uw, u[0], u[1]), d_xi(uw)
    ve, vx = d_eta(vw, v[0], v[1]), d_xi(vw)
    du_dx = cx_xi * ux + cx_eta * ue
    du_dz = cz_xi * ux + cz_eta * ue
    dv_dx = cx_xi * vx + cx_eta * ve
    dv_dz = cz_xi * vx + cz_eta * ve
    div = du_dx + dv_dz
    Re = case.Re
    iso = -(p[0] + 2.0 / (3.0 * Re) * div)
    sxx = iso + 2.0 / Re * du_dx
    szz = iso + 2.0 / Re * dv_dz
    sxz = (du_dz + dv_dx) / Re
    nx, nz = np.cos(th), np.sin(th)
    ds = 0.5 * g.D * 2.0 * np.pi * g.dxi
    Fd = np.sum(sxx * nx + sxz * nz) * ds
    Fl = np.sum(sxz * nx + szz * nz) * ds
    return 2.0 * Fd, 2.0 * Fl


def strouhal(t, cl):
    """St = 1/T from upward zero crossings of C_L (eq:st with D = U = 1), linear interpolation."""
    t = np.asarray(t, dtype=np.float64); cl = np.asarray(cl, dtype=np.float64)
    c = cl - np.mean(cl)
    idx = np.nonzero((c[:-1] < 0) & (c[1:] >= 0))[0]
    if len(idx) < 2:
        return float("nan")
    tc = t[idx] - c[idx] * (t[idx + 1] - t[idx]) / (c[idx + 1] - c[idx])
    return float(1.0 / np.mean(np.diff(tc)))


def weighted_l2(g: Grid, s):
    """||s||_L2 = sqrt(d_xi d_eta sum |s|^2 |J|) (Sec. IV, weighted L2 norm, |J| reading)."""
    J = metrics(g)["J"]
    return float(np.sqrt(g.dxi * g.deta * np.sum(np.abs(np.reshape(s, J.shape)) ** 2 * np.abs(J))))
