"""L1 oracle: analytic QTT construction of the grid fields, metric terms and the
curvilinear finite-difference operators (Sec. III.B.3, App. A, App. E), in NumPy FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Bit layout: a 2-D field f(i, j) on the (2^n_eta x 2^n_xi) interior grid is a vector
over n = n_eta + n_xi bits (Sec. III.B.1).  ``sequential`` places the eta bits of i
first and then the xi bits of j (r = i_b U j_b); ``interleaved`` alternates i and j bits
level by level.  Within each index the first bit is the most significant (App. D).

Construction (Sec. III.B.3 with the analytic metric of App. E):
* 1-D shift MPOs (carry automata) give the central stencils; xi is periodic, eta keeps
  only interior neighbours (the ghost part goes into boundary vectors);
* metric coefficients are exact low-rank MPS: exponentials in eta have rank 1, sin/cos
  in xi rank 2;
* D_x = diag(c_x_xi) D_xi + diag(c_x_eta) D_eta, etc.; products diag(c) D are MPO-MPO
  products; every operator is rounded at sigma < 1e-14 sigma_1 (Sec. III.B.3).
"""
from __future__ import annotations

import numpy as np

from . import tt

OP_EPS = 1e-14


def layout(n_eta: int, n_xi: int, ordering: str):
    """List of (axis, level) per core: axis 0 = eta (i), 1 = xi (j); level 0 = MSB."""
    if ordering == "sequential":
        return [(0, l) for l in range(n_eta)] + [(1, l) for l in range(n_xi)]
    if ordering == "interleaved":
        out = []
        for l in range(max(n_eta, n_xi)):
            if l < n_eta:
                out.append((0, l))
            if l < n_xi:
                out.append((1, l))
        return out
    raise ValueError(ordering)


def field_to_vec(f2d, ordering: str) -> np.ndarray:
    """Reorder a (2^n_eta, 2^n_xi) array into the QTT vector index q (first core = MSB)."""
    Ne, Nx = f2d.shape
    ne, nx = int(np.log2(Ne)), int(np.log2(Nx))
    lay = layout(ne, nx, ordering)
    n = ne + nx
    q = np.arange(2 ** n)
    i = np.zeros_like(q); j = np.zeros_like(q)
    for p, (ax, l) in enumerate(lay):
        bit = (q >> (n - 1 - p)) & 1
        if ax == 0:
            i |= bit << (ne - 1 - l)
        else:
            j |= bit << (nx - 1 - l)
    return np.asarray(f2d)[i, j]


def vec_to_field(v, n_eta: int, n_xi: int, ordering: str) -> np.ndarray:
    lay = layout(n_eta, n_xi, ordering)
    n = n_eta + n_xi
    q = np.arange(2 ** n)
    i = np.zeros_like(q); j = np.zeros_like(q)
    for p, (ax, l) in enumerate(lay):
        bit = (q >> (n - 1 - p)) & 1
        if ax == 0:
            i |= bit << (n_eta - 1 - l)
        else:
            j |= bit << (n_xi - 1 - l)
    out = np.zeros((2 ** n_eta, 2 ** n_xi))
    out[i, j] = np.asarray(v)
    return out


# ---------------------------------------------------------------- 1-D building blocks

def mps1_exp(nb: int, C: float, lam: float):
    """C exp(lam q), q = 0..2^nb-1: rank 1, core k holds exp(lam s 2^(nb-1-k))."""
    cores = []
    for k in range(nb):
        c = np.array([1.0, np.exp(lam * 2.0 ** (nb - 1 - k))]).reshape(1, 2, 1)
        cores.append(c)
    cores[0] = cores[0] * C
    return cores


def mps1_trig(nb: int, omega: float, phase: float, kind: str, amp: float = 1.0):
    """amp cos(omega q + phase) or amp sin(...): rank 2 through the angle-addition rule.

    [cos(a+b), sin(a+b)] = [cos a, sin a] [[cos b, sin b], [-sin b, cos b]].
    """
    def rot(b):
        return np.array([[np.cos(b), np.sin(b)], [-np.sin(b), np.cos(b)]])
    cores = []
    for k in range(nb):
        c = np.zeros((2, 2, 2))
        for s in range(2):
            c[:, s, :] = rot(omega * s * 2.0 ** (nb - 1 - k))
        cores.append(c)
    first = np.array([np.cos(phase), np.sin(phase)]) * amp
    cores[0] = np.einsum("a,asb->sb", first, cores[0])[None]
    last = np.array([1.0, 0.0]) if kind == "cos" else np.array([0.0, 1.0])
    cores[-1] = np.einsum("asb,b->as", cores[-1], last)[:, :, None]
    return cores


def mps1_const(nb: int, C: float = 1.0):
    return mps1_exp(nb, C, 0.0)


def mps1_indicator(nb: int, q: int):
    """e_q: 1 at index q, 0 elsewhere (rank 1)."""
    cores = []
    for k in range(nb):
        bit = (q >> (nb - 1 - k)) & 1
        c = np.zeros((1, 2, 1)); c[0, bit, 0] = 1.0
        cores.append(c)
    return cores


def mpo1_identity(nb: int):
    return [np.eye(2).reshape(1, 2, 2, 1) for _ in range(nb)]


def mpo1_shift(nb: int, step: int, periodic: bool):
    """(S f)_q = f_{q+step}, step = +1 or -1, as a carry automaton (bond 2).

    Bond index = carry (borrow for step = -1).  The LSB core (last) receives carry 1;
    the MSB core (first) keeps only carry-out 0 when not periodic, both when periodic.
    """
    cores = []
    for k in range(nb):
        W = np.zeros((2, 2, 2, 2))   # (carry_out (left), out bit, in bit, carry_in (right))
        for o in range(2):
            for c in range(2):
                if step > 0:
                    t = o + c
                    q, cout = t % 2, t // 2
                else:
                    t = o - c
                    q, cout = t % 2, 1 if t < 0 else 0
                W[cout, o, q, c] = 1.0
        cores.append(W)
    left = np.array([1.0, 1.0]) if periodic else np.array([1.0, 0.0])
    right = np.array([0.0, 1.0])
    cores[0] = np.einsum("a,asrb->srb", left, cores[0])[None]
    cores[-1] = np.einsum("asrb,b->asr", cores[-1], right)[..., None]
    return cores


def mpo1_diag_indicator(nb: int, q: int):
    return tt.diag_mpo(mps1_indicator(nb, q))


def lin_mpo(terms):
    """sum coef * M as one MPO (direct sums, unrounded)."""
    out = None
    for coef, M in terms:
        if out is None:
            out = [c.copy() for c in M]
            out[0] = out[0] * coef
        else:
            out = tt.mpo_direct_sum(1.0, out, coef, M)
    return out


# ---------------------------------------------------------------- 2-D assembly

def combine_mps(f_eta, f_xi, n_eta, n_xi, ordering):
    """f(i) g(j) as one 2-D MPS in the given bit layout (bond = product of the 1-D bonds)."""
    lay = layout(n_eta, n_xi, ordering)
    pos = [0, 0]
    be, bx = 1, 1  # current right bonds of each 1-D train
    out = []
    for ax, l in lay:
        if ax == 0:
            A = f_eta[l]
            c = np.einsum("asb,xy->axsby", A, np.eye(bx))
            c = c.reshape(A.shape[0] * bx, 2, A.shape[2] * bx)
            be = A.shape[2]
        else:
            A = f_xi[l]
            c = np.einsum("xy,asb->xasyb", np.eye(be), A)
            c = c.reshape(be * A.shape[0], 2, be * A.shape[2])
            bx = A.shape[2]
        out.append(c)
    return out


def combine_mpo(M_eta, M_xi, n_eta, n_xi, ordering):
    """M_eta (x) M_xi acting on (i, j) in the given bit layout."""
    lay = layout(n_eta, n_xi, ordering)
    be, bx = 1, 1
    out = []
    for ax, l in lay:
        if ax == 0:
            A = M_eta[l]
            c = np.einsum("asrb,xy->axsrby", A, np.eye(bx))
            c = c.reshape(A.shape[0] * bx, 2, 2, A.shape[3] * bx)
            be = A.shape[3]
        else:
            A = M_xi[l]
            c = np.einsum("xy,asrb->xasryb", np.eye(be), A)
            c = c.reshape(be * A.shape[0], 2, 2, be * A.shape[3])
            bx = A.shape[3]
        out.append(c)
    return out


class Ops:
    """All operators and boundary vectors of one cylinder case (Sec. III, App. A, App. E)."""

    def __init__(self, n_eta, n_xi, R, Re, dt, ordering="interleaved", D=1.0, rot=0.0, u_inf=1.0):
        self.n_eta, self.n_xi, self.R, self.Re, self.dt = n_eta, n_xi, R, Re, dt
        self.ordering, self.D, self.rot, self.u_inf = ordering, D, rot, u_inf
        ne, nx = n_eta, n_xi
        Ne, Nx = 2 ** ne, 2 ** nx
        self.deta = de = 1.0 / (Ne + 1)
        self.dxi = dx = 1.0 / Nx
        lnR = np.log(R)
        om = 2 * np.pi * dx

        def m2(fe, fx):
            return combine_mps(fe, fx, ne, nx, ordering)

        def o2(Me, Mx):
            return combine_mpo(Me, Mx, ne, nx, ordering)

        Ie, Ix = mpo1_identity(ne), mpo1_identity(nx)
        # 1/r_i = (2/D) R^{-(i+1) d_eta}, r_i^2 = (D/2)^2 R^{2 (i+1) d_eta}
        inv_r = mps1_exp(ne, (2.0 / D) * R ** (-de), -lnR * de)
        r2 = mps1_exp(ne, (D / 2) ** 2 * R ** (2 * de), 2 * lnR * de)
        sin_x = mps1_trig(nx, om, 0.0, "sin")
        cos_x = mps1_trig(nx, om, 0.0, "cos")
        one_e, one_x = mps1_const(ne), mps1_const(nx)
        # metric coefficients (analytic, App. A with App. E's mapping)
        cx_xi = m2(tt.scale(inv_r, -1.0 / (2 * np.pi)), sin_x)
        cx_eta = m2(tt.scale(inv_r, 1.0 / lnR), cos_x)
        cz_xi = m2(tt.scale(inv_r, 1.0 / (2 * np.pi)), cos_x)
        cz_eta = m2(tt.scale(inv_r, 1.0 / lnR), sin_x)
        self.absJ = m2(tt.scale(r2, 2 * np.pi * lnR), one_x)       # |J| = 2 pi lnR r^2
        # stencils
        Sxp, Sxm = mpo1_shift(nx, +1, True), mpo1_shift(nx, -1, True)
        Sep, Sem = mpo1_shift(ne, +1, False), mpo1_shift(ne, -1, False)
        d_xi = o2(Ie, lin_mpo([(1 / (2 * dx), Sxp), (-1 / (2 * dx), Sxm)]))
        d_eta = o2(lin_mpo([(1 / (2 * de), Sep), (-1 / (2 * de), Sem)]), Ix)
        dd_xi = o2(Ie, lin_mpo([(1 / dx ** 2, Sxp), (-2 / dx ** 2, Ix), (1 / dx ** 2, Sxm)]))
        dd_eta = o2(lin_mpo([(1 / de ** 2, Sep), (-2 / de ** 2, Ie), (1 / de ** 2, Sem)]), Ix)
        E0 = o2(mpo1_diag_indicator(ne, 0), Ix)                      # rows i = 0
        d_eta_p = lin_mpo([(1.0, d_eta), (-1 / (2 * de), E0)])       # Neumann ghost p_{-1} = p_0
        dd_eta_p = lin_mpo([(1.0, dd_eta), (1 / de ** 2, E0)])
        rnd = lambda M: tt.round_mpo(M, 10 ** 9, OP_EPS)
        D = lambda c: tt.diag_mpo(c)
        self.Dx = rnd(lin_mpo([(1.0, tt.mpo_mpo(D(cx_xi), d_xi)), (1.0, tt.mpo_mpo(D(cx_eta), d_eta))]))
        self.Dz = rnd(lin_mpo([(1.0, tt.mpo_mpo(D(cz_xi), d_xi)), (1.0, tt.mpo_mpo(D(cz_eta), d_eta))]))
        self.Dxp = rnd(lin_mpo([(1.0, tt.mpo_mpo(D(cx_xi), d_xi)), (1.0, tt.mpo_mpo(D(cx_eta), d_eta_p))]))
        self.Dzp = rnd(lin_mpo([(1.0, tt.mpo_mpo(D(cz_xi), d_xi)), (1.0, tt.mpo_mpo(D(cz_eta), d_eta_p))]))
        # |J| Lap_h = (lnR / 2 pi) d_xixi + (2 pi / lnR) d_etaeta  (g12 = 0, g/J constant)
        aX, aE = lnR / (2 * np.pi), 2 * np.pi / lnR
        k = dt / Re
        self.H = rnd(lin_mpo([(1.0, D(self.absJ)), (-k * aX, dd_xi), (-k * aE, dd_eta)]))
        self.Ap = rnd(lin_mpo([(-aX, dd_xi), (-aE, dd_eta_p)]))
        self.Jdiag = D(self.absJ)
        self.Px = rnd(tt.mpo_mpo(D(tt.scale(self.absJ, -1.0 / dt)), self.Dx))
        self.Pz = rnd(tt.mpo_mpo(D(tt.scale(self.absJ, -1.0 / dt)), self.Dz))
        # ghost (boundary) vectors, Sec. III.A: op(f) = M f + bc(f)
        uw_amp, vw_amp = rot, -rot      # u_G = rot sin(theta), v_G = -rot cos(theta) (eq:rot_bc)
        e0, eN = mps1_indicator(ne, 0), mps1_indicator(ne, Ne - 1)

        def bc_eta(wall, far, scale_w, scale_f):
            """e_0 (x) wall(j) * scale_w + e_{N-1} (x) far(j) * scale_f, or None if zero."""
            parts = []
            if wall is not None:
                parts.append(m2(tt.scale(e0, scale_w), wall))
            if far is not None:
                parts.append(m2(tt.scale(eN, scale_f), far))
            if not parts:
                return None
            out = parts[0]
            for p in parts[1:]:
                out = tt.direct_sum(1.0, out, 1.0, p)
            return tt.round_tt(out, 10 ** 9, OP_EPS)

        u_wall = mps1_trig(nx, om, 0.0, "sin", uw_amp) if rot != 0.0 else None
        v_wall = mps1_trig(nx, om, 0.0, "cos", vw_amp) if rot != 0.0 else None
        u_far = mps1_const(nx, u_inf) if u_inf != 0.0 else None
        v_far = None
        self.wall = (u_wall, v_wall)

        def had(a, b):
            if a is None or b is None:
                return None
            return tt.round_tt(tt.hadamard_exact(a, b), 10 ** 9, OP_EPS)

        def add(a, b):
            if a is None:
                return b
            if b is None:
                return a
            return tt.round_tt(tt.direct_sum(1.0, a, 1.0, b), 10 ** 9, OP_EPS)

        def bc_first(w, f):
            return bc_eta(w, f, -1 / (2 * de), 1 / (2 * de))

        def bc_second(w, f):
            return bc_eta(w, f, 1 / de ** 2, 1 / de ** 2)

        self.bcx_u = had(cx_eta, bc_first(u_wall, u_far))
        self.bcz_u = had(cz_eta, bc_first(u_wall, u_far))
        self.bcx_v = had(cx_eta, bc_first(v_wall, v_far))
        self.bcz_v = had(cz_eta, bc_first(v_wall, v_far))
        # |J| * ghost part of Lap_h = (2 pi / lnR) * eta-ghost part of d_etaeta
        bl_u, bl_v = bc_second(u_wall, u_far), bc_second(v_wall, v_far)
        self.JbcLap_u = None if bl_u is None else tt.scale(bl_u, aE)
        self.JbcLap_v = None if bl_v is None else tt.scale(bl_v, aE)
        bdiv = add(self.bcx_u, self.bcz_v)
        self.bcdiv_w = had(tt.scale(self.absJ, -1.0 / dt), bdiv)
        self.fields = dict(cx_xi=cx_xi, cx_eta=cx_eta, cz_xi=cz_xi, cz_eta=cz_eta, inv_r=inv_r)

    def encode(self, f2d, chi, eps=0.0):
        n = self.n_eta + self.n_xi
        return tt.tt_svd(field_to_vec(f2d, self.ordering), n, 2, chi, eps)

    def decode(self, cores):
        return vec_to_field(tt.full(cores), self.n_eta, self.n_xi, self.ordering)
