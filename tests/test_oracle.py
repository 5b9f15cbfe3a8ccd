"""Pins of the FP64 oracle against what arXiv:2507.05222 and the mathematics fix.

Each test names the passage (section / equation / appendix) it pins.  No expected value
here comes from the CUDA path.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fd, tt, qtt_ops as Q, step as S
from paper_2507_05222_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def perm(ne, nx, ordering):
    n = ne + nx
    return np.array([Q.field_to_vec(e.reshape(2 ** ne, 2 ** nx), ordering) for e in np.eye(2 ** n)]).T


# ------------------------------------------------------------------ App. D worked example

def load_appD():
    cores = [np.zeros((1, 2, 2)), np.zeros((2, 2, 2)), np.zeros((2, 2, 1))]
    with open(os.path.join(GOLDEN, "appD_cores.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, a, s, b, v = line.split()
            cores[int(k)][int(a), int(s), int(b)] = float(v)
    return cores


def test_appD_reconstruction_msb_first():
    """App. D: the printed cores give t = 1..8 only with the first core as the MSB."""
    assert np.array_equal(tt.full(load_appD()), np.arange(1.0, 9.0))


def test_appD_tt_svd_rank_and_roundtrip():
    """App. D: t = (1..8) has TT ranks (2, 2) and TT-SVD reproduces it exactly."""
    t = np.arange(1.0, 9.0)
    c = tt.tt_svd(t, 3, 2, chi=8, eps=1e-12)
    assert tt.bonds(c) == [1, 2, 2, 1]
    assert np.allclose(tt.full(c), t, rtol=0, atol=1e-13)


# ------------------------------------------------------------------ exact low ranks (Sec. II, III.B.1)

@pytest.mark.parametrize("kind,rank", [("exp", 1), ("const", 1), ("sin", 2), ("cos", 2), ("lin", 2)])
def test_analytic_ranks(kind, rank):
    """Exponentials rank 1, constants rank 1, sin/cos and linear ramps rank 2 (Sec. II, III.B.1)."""
    n = 10
    q = np.arange(2 ** n, dtype=np.float64)
    f = {"exp": np.exp(0.013 * q), "const": np.full(q.shape, 3.0),
         "sin": np.sin(0.37 * q + 0.2), "cos": np.cos(2 * np.pi * q / 2 ** n), "lin": 2.0 + 0.5 * q}[kind]
    c = tt.tt_svd(f, n, 2, chi=64, eps=1e-12)
    assert max(tt.bonds(c)) == rank
    assert np.allclose(tt.full(c), f, atol=1e-10 * np.abs(f).max())


@pytest.mark.parametrize("kind", ["exp", "sin", "cos", "const", "ind0", "indN"])
def test_analytic_mps_builders(kind):
    """The direct O(log N) cores of Sec. III.B.1 equal the sampled functions."""
    nb = 7
    q = np.arange(2 ** nb, dtype=np.float64)
    if kind == "exp":
        c, f = Q.mps1_exp(nb, 1.7, -0.05), 1.7 * np.exp(-0.05 * q)
    elif kind == "sin":
        c, f = Q.mps1_trig(nb, 0.3, 0.4, "sin", 2.0), 2.0 * np.sin(0.3 * q + 0.4)
    elif kind == "cos":
        c, f = Q.mps1_trig(nb, 0.3, 0.4, "cos"), np.cos(0.3 * q + 0.4)
    elif kind == "const":
        c, f = Q.mps1_const(nb, 2.5), np.full(q.shape, 2.5)
    elif kind == "ind0":
        c, f = Q.mps1_indicator(nb, 0), (q == 0).astype(float)
    else:
        c, f = Q.mps1_indicator(nb, 2 ** nb - 1), (q == 2 ** nb - 1).astype(float)
    assert np.allclose(tt.full(c), f, atol=1e-13 * max(1.0, np.abs(f).max()))


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("step", [1, -1])
def test_shift_mpo_brute_force(periodic, step):
    """Carry-automaton shift MPOs equal the shift matrices (Kazeev-type, Sec. III.B.3)."""
    nb = 5
    N = 2 ** nb
    M = tt.full_mpo(Q.mpo1_shift(nb, step, periodic))
    ref = np.zeros((N, N))
    for i in range(N):
        j = i + step
        if 0 <= j < N:
            ref[i, j] = 1.0
        elif periodic:
            ref[i, j % N] = 1.0
    assert np.array_equal(M, ref)


# ------------------------------------------------------------------ NVPS (Sec. IV)

@pytest.mark.parametrize("n,chi,frac,tol", [(17, 20, 0.058, 0.001), (17, 35, 0.15, 0.005),
                                            (17, 50, 0.25, 0.015), (17, 40, 0.18, 0.005),
                                            (16, 40, 0.30, 0.02), (16, 80, 0.87, 0.005)])
def test_nvps_fractions(n, chi, frac, tol):
    """NVPS_TT = 2 sum alpha_{k-1} alpha_k with alpha_k = min(2^k, 2^(n-k), chi) (eq:simpleMPS,
    Sec. IV) reproduces the printed compression ratios: 5.8 %, ~15 %, ~1/4, 18 %, ~30 %, 87 %."""
    b = inputs.bond_profile(n, chi)
    nv = 2 * sum(b[k] * b[k + 1] for k in range(n))
    assert abs(nv / 2 ** n - frac) <= tol
    if (n, chi) == (17, 20):
        assert nv == 7560


# ------------------------------------------------------------------ grid (App. E) and operators (App. A)

@pytest.mark.parametrize("ne,nx,h", [(8, 8, 6.78e-3), (8, 9, 6.14e-3), (9, 9, 3.39e-3)])
def test_hmin_grids(ne, nx, h):
    """h_min of G1/G2/G3 with D_outer = 32 D (Sec. IV, App. E)."""
    assert abs(fd.Grid(ne, nx, 32.0).h_min() - h) < 0.006 * h


def test_jacobian_closed_form():
    """J = -2 pi lnR r^2 < 0, g12 = 0, g22/J and g11/J constant (App. A with App. E)."""
    g = fd.Grid(4, 5, 40.0)
    m = fd.metrics(g)
    rr, _ = g.nodes()
    assert np.allclose(m["J"], -2 * np.pi * g.lnR * rr ** 2, rtol=1e-14)
    assert np.abs(m["g12"]).max() < 1e-12 * np.abs(m["g11"]).max()
    assert np.allclose(m["g22"] / m["J"], -g.lnR / (2 * np.pi), rtol=1e-13)
    assert np.allclose(m["g11"] / m["J"], -2 * np.pi / g.lnR, rtol=1e-13)


def test_curvilinear_first_derivatives_closed_form():
    """Central differences with the analytic metric: D_x x = a sin^2 + b cos^2,
    D_x z = (b - a) sin cos, D_z z = a cos^2 + b sin^2 (App. A stencils, eq:curviliner-deriavtive)."""
    g = fd.Grid(4, 5, 40.0)
    ops = fd.operators(g, "velocity")
    x, z = g.xz(); xg, zg = g.xz(ghosts=True)
    th = g.theta(np.arange(g.N_xi))[None, :]
    a = np.sin(2 * np.pi * g.dxi) / (2 * np.pi * g.dxi)
    b = np.sinh(g.lnR * g.deta) / (g.lnR * g.deta)
    Dxx = fd.apply_op(ops["Dx"], x, xg[0], xg[-1]).reshape(x.shape)
    Dxz = fd.apply_op(ops["Dx"], z, zg[0], zg[-1]).reshape(x.shape)
    Dzz = fd.apply_op(ops["Dz"], z, zg[0], zg[-1]).reshape(x.shape)
    Dzx = fd.apply_op(ops["Dz"], x, xg[0], xg[-1]).reshape(x.shape)
    assert np.abs(Dxx - (a * np.sin(th) ** 2 + b * np.cos(th) ** 2)).max() < 1e-13
    assert np.abs(Dxz - (b - a) * np.sin(th) * np.cos(th)).max() < 1e-13
    assert np.abs(Dzz - (a * np.cos(th) ** 2 + b * np.sin(th) ** 2)).max() < 1e-13
    assert np.abs(Dzx - (b - a) * np.sin(th) * np.cos(th)).max() < 1e-13


def test_laplacian_closed_form():
    """Lap_h applied to x = r cos(theta) (harmonic) gives the exact discrete value
    (x / r^2) [(2cos(w) - 2)/(4 pi^2 dxi^2) + (2cosh(lnR deta) - 2)/(lnR^2 deta^2)],
    and Lap_h ln r = 0 exactly (seven-term Laplacian of App. A, analytic metric)."""
    g = fd.Grid(4, 5, 40.0)
    ops = fd.operators(g, "velocity")
    x, _ = g.xz(); xg, _ = g.xz(ghosts=True)
    rr, _ = g.nodes(); rg, _ = g.nodes(ghosts=True)
    w = 2 * np.pi * g.dxi
    lam = (2 * np.cos(w) - 2) / (4 * np.pi ** 2 * g.dxi ** 2) + \
          (2 * np.cosh(g.lnR * g.deta) - 2) / (g.lnR ** 2 * g.deta ** 2)
    L = fd.apply_op(ops["Lap"], x, xg[0], xg[-1]).reshape(x.shape)
    assert np.allclose(L, x / rr ** 2 * lam, rtol=1e-10, atol=1e-10)
    lr = np.log(rr); lrg = np.log(rg)
    L2 = fd.apply_op(ops["Lap"], lr, lrg[0], lrg[-1])
    assert np.abs(L2).max() < 1e-9


@pytest.mark.parametrize("bc", ["velocity", "pressure"])
def test_weighted_operators_symmetric(bc):
    """|J| Lap_h is symmetric (and -|J| Lap_h^p positive definite): the reading that makes
    the ALS systems SPD (Sec. III.C, J-weighted cost)."""
    g = fd.Grid(4, 4, 40.0)
    ops = fd.operators(g, bc)
    JL = sp.diags(np.abs(fd.metrics(g)["J"]).ravel()) @ ops["Lap"][0]
    A = JL.toarray()
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(-A).min() > 0


@pytest.mark.parametrize("ordering", ["interleaved", "sequential"])
def test_qtt_operators_equal_sparse_fd(ordering):
    """Dense reconstruction of every QTT operator and boundary vector equals the sparse FD
    matrix / ghost vector of L0 (Sec. III.B.3, App. A), with a rotating wall (eq:rot_bc)."""
    ne, nx = 3, 4
    ops = Q.Ops(ne, nx, 40.0, 100.0, 2e-3, ordering, rot=0.7)
    g = fd.Grid(ne, nx, 40.0)
    case = fd.Case(g, 100.0, 2e-3, rot=0.7)
    vel, pre = fd.operators(g, "velocity"), fd.operators(g, "pressure")
    P = perm(ne, nx, ordering)
    J = np.abs(fd.metrics(g)["J"]).ravel()

    def rel(M, Sm):
        a = tt.full_mpo(M); b = P @ Sm.toarray() @ P.T
        return np.abs(a - b).max() / np.abs(b).max()

    assert rel(ops.Dx, vel["Dx"][0]) < 1e-13
    assert rel(ops.Dz, vel["Dz"][0]) < 1e-13
    assert rel(ops.Dxp, pre["Dx"][0]) < 1e-13
    assert rel(ops.Dzp, pre["Dz"][0]) < 1e-13
    I = sp.identity(J.size)
    assert rel(ops.H, sp.diags(J) @ (I - 2e-3 / 100.0 * vel["Lap"][0])) < 1e-13
    assert rel(ops.Ap, -sp.diags(J) @ pre["Lap"][0]) < 1e-13
    assert rel(ops.Px, -sp.diags(J) @ vel["Dx"][0] / 2e-3) < 1e-13
    uw, vw = case.wall_velocity(); uf, vf = case.far_velocity()
    z = np.zeros(J.size)
    for vec, ref in [(ops.bcx_u, fd.apply_op(vel["Dx"], z, uw, uf)),
                     (ops.bcz_u, fd.apply_op(vel["Dz"], z, uw, uf)),
                     (ops.bcx_v, fd.apply_op(vel["Dx"], z, vw, vf)),
                     (ops.bcz_v, fd.apply_op(vel["Dz"], z, vw, vf)),
                     (ops.JbcLap_u, J * fd.apply_op(vel["Lap"], z, uw, uf)),
                     (ops.JbcLap_v, J * fd.apply_op(vel["Lap"], z, vw, vf))]:
        assert np.abs(tt.full(vec) - P @ ref).max() < 1e-13 * np.abs(ref).max()
    bdiv = fd.apply_op(vel["Dx"], z, uw, uf) + fd.apply_op(vel["Dz"], z, vw, vf)
    assert np.abs(tt.full(ops.bcdiv_w) - P @ (-J * bdiv / 2e-3)).max() < 1e-13 * np.abs(J * bdiv / 2e-3).max()


def test_operator_bonds_small_and_compressive():
    """The curvilinear operators stay low-rank (Sec. IV.C: operator NVPS far below 5N)."""
    ops = Q.Ops(7, 7, 40.0, 200.0, 8e-4, "interleaved")
    for M in (ops.Dx, ops.Dz, ops.H, ops.Ap):
        assert max(tt.bonds(M)) <= 12
    nv = sum(c.size for c in ops.Dx)
    assert nv < 5 * 2 ** 14 / 10


def test_field_layouts_roundtrip():
    """Bit layouts (Sec. III.B.1; interleaved alternative): sequential is the row-major
    reshape, and both orderings round-trip."""
    f = np.arange(8 * 16, dtype=float).reshape(8, 16)
    assert np.array_equal(Q.field_to_vec(f, "sequential"), f.ravel())
    for o in ("sequential", "interleaved"):
        assert np.array_equal(Q.vec_to_field(Q.field_to_vec(f, o), 3, 4, o), f)


# ------------------------------------------------------------------ TT algebra (Sec. II.A)

def test_round_tt_equals_dense_tt_svd():
    """TT-rounding (QR + SVD sweeps) equals the right-to-left TT-SVD of the dense tensor."""
    n, chi = 9, 6
    x = inputs.random_cores(n, 12, seed=5)
    ref = tt.tt_svd(tt.full(x), n, 2, chi, pre_bonds=tt.bonds(x))
    got = tt.round_tt(x, chi)
    assert tt.bonds(got) == tt.bonds(ref)
    assert np.allclose(tt.full(got), tt.full(ref), atol=1e-12 * np.abs(tt.full(ref)).max())


def test_round_tt_error_bound_and_canonical():
    """||x - round(x)||^2 <= sum of discarded sigma^2 over all cuts (Oseledets 2011, cited
    Sec. II.A), the result is right-canonical (Sec. II), and chi >= rank is exact."""
    n, chi = 10, 5
    x = inputs.random_cores(n, 16, seed=7)
    xd = tt.full(x)
    y = tt.round_tt(x, chi)
    # discarded weights cut by cut (right-to-left, on the sequentially truncated tensor)
    disc = 0.0
    cur = xd.reshape(-1, 1); rk = 1
    for k in range(n, 1, -1):
        U, Sg, Vt = np.linalg.svd(cur.reshape(2 ** (k - 1), 2 * rk), full_matrices=False)
        b = min(chi, len(Sg))
        disc += np.sum(Sg[b:] ** 2)
        cur = U[:, :b] * Sg[:b]; rk = b
    err2 = np.sum((tt.full(y) - xd) ** 2)
    assert err2 <= disc * (1 + 1e-10) + 1e-20
    for c in y[1:]:
        m = c.reshape(c.shape[0], -1)
        assert np.allclose(m @ m.T, np.eye(c.shape[0]), atol=1e-12)
    z = tt.round_tt(x, 10 ** 6)
    assert np.allclose(tt.full(z), xd, atol=1e-12 * np.abs(xd).max())


def test_rounding_eps_threshold():
    """Operator rounding keeps sigma > eps sigma_1 only (Sec. III.B.3, 1e-14)."""
    a = Q.mps1_trig(8, 0.1, 0.0, "sin")
    b = Q.mps1_trig(8, 0.1, 0.0, "cos")
    s = tt.direct_sum(1.0, a, 1.0, b)               # bond 4, true rank 2
    r = tt.round_tt(s, 100, 1e-14)
    assert max(tt.bonds(r)) == 2


def test_direct_sum_mpo_mps_hadamard_dense():
    """Sec. II.A.1-3 against dense brute force."""
    n = 8
    a = inputs.random_cores(n, 4, seed=1); b = inputs.random_cores(n, 3, seed=2)
    M = inputs.random_mpo_cores(n, 3, seed=3)
    ad, bd, Md = tt.full(a), tt.full(b), tt.full_mpo(M)
    assert np.allclose(tt.full(tt.direct_sum(0.5, a, -2.0, b)), 0.5 * ad - 2.0 * bd, atol=1e-12)
    assert np.allclose(tt.full(tt.mpo_mps(M, a)), Md @ ad, atol=1e-10)
    assert np.allclose(tt.full(tt.hadamard_exact(a, b)), ad * bd, atol=1e-10)
    assert np.allclose(tt.full_mpo(tt.diag_mpo(a)), np.diag(ad), atol=1e-12)
    M2 = inputs.random_mpo_cores(n, 2, seed=4)
    assert np.allclose(tt.full_mpo(tt.mpo_mpo(M, M2)), Md @ tt.full_mpo(M2), atol=1e-9)
    assert np.isclose(tt.dot(a, b), ad @ bd, rtol=1e-12)


def test_round_discarded_norm_is_the_rounding_error():
    """The discarded norm of a canonical TT-SVD sweep equals ||x - round(x)||: the truncation
    errors of different cuts are orthogonal (the left part is orthonormal at every cut), so the
    TT-SVD bound of Sec. II's rounding holds with equality."""
    x = inputs.random_cores(10, 16, seed=5)
    for chi in (4, 8, 12, 32):
        info = {}
        y = tt.round_tt(x, chi, info=info)
        err = np.linalg.norm(tt.full(x) - tt.full(y))
        assert abs(info["discarded_norm"] - err) <= 1e-12 * np.linalg.norm(tt.full(x))
    info = {}
    tt.round_tt(x, 64, info=info)
    assert info["discarded_norm"] == 0.0


def test_fit_exact_when_representable():
    """Variational fit (Table I) is exact when the target has rank <= chi: Hadamard of
    rank-2 sin and rank-1 exp fields, plus an MPO term and a plain term."""
    n = 9
    a = Q.mps1_trig(n, 0.21, 0.3, "sin")
    b = Q.mps1_exp(n, 1.0, 0.004)
    c = inputs.random_cores(n, 3, seed=11)
    M = Q.lin_mpo([(1.0, Q.mpo1_shift(n, 1, True)), (-1.0, Q.mpo1_shift(n, -1, True))])
    terms = [("had", 2.0, a, b), ("vec", 0.5, c), ("mpo", -1.0, M, a)]
    target = tt.terms_full(terms)
    assert max(tt.bonds(tt.tt_svd(target, n, 2, 100, 1e-12))) == 9
    init = inputs.random_cores(n, 16, seed=12)
    got = tt.fit(terms, init, sweeps=2)
    assert np.allclose(tt.full(got), target, atol=1e-11 * np.abs(target).max())


def test_hadamard_round_quality():
    """Zip-up + fit gives an approximation no worse than 2x the TT-SVD truncation of the
    exact product (the fit minimises the same distance; Table I)."""
    n, chi = 10, 8
    a = inputs.random_cores(n, 6, seed=21); b = inputs.random_cores(n, 5, seed=22)
    exact = tt.full(a) * tt.full(b)
    best = tt.full(tt.round_tt(tt.hadamard_exact(a, b), chi))
    got = tt.full(tt.hadamard_round(a, b, chi, sweeps=3))
    e_best = np.linalg.norm(best - exact); e_got = np.linalg.norm(got - exact)
    assert e_got <= 2.0 * e_best


def test_cg_solves_spd():
    """CG and diagonally preconditioned CG reach the direct solution of an SPD system; on a
    badly scaled matrix the preconditioned one needs far fewer iterations."""
    g = inputs.rng(3)
    A = g.standard_normal((30, 30)); A = A @ A.T + 30 * np.eye(30)
    b = g.standard_normal(30)
    x, it = tt.cg(lambda v: A @ v, b, np.zeros(30), 200, 1e-14)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10)
    Dm = np.diag(np.logspace(0, 4, 30))
    B = Dm @ A @ Dm
    x0, it0 = tt.cg(lambda v: B @ v, b, np.zeros(30), 2000, 1e-13)
    x1, it1 = tt.cg(lambda v: B @ v, b, np.zeros(30), 2000, 1e-13, dinv=1.0 / np.diag(B))
    ref = np.linalg.solve(B, b)
    assert np.allclose(x1, ref, rtol=1e-8) and it1 < it0 / 3


def test_local_diag_is_the_diagonal_of_the_local_matrix():
    """The ALS preconditioner's diagonal equals the diagonal of the assembled local matrix
    (Fig. 5: M_eff = L (x) W (x) R contracted over the operator bonds)."""
    g = inputs.rng(4)
    L = g.standard_normal((5, 3, 5)); W = g.standard_normal((3, 2, 2, 4)); R = g.standard_normal((6, 4, 6))
    M = np.einsum("cwa,wstv,evb->cseatb", L, W, R).reshape(5 * 2 * 6, 5 * 2 * 6)
    assert np.allclose(tt.local_diag(L, W, R).ravel(), np.diag(M), rtol=1e-13, atol=0)


def test_als_full_rank_equals_sparse_solve():
    """Single-site ALS (Sec. II.A.4) at full bond dimension reaches the sparse direct
    solution of the J-weighted Poisson problem (Sec. III.C) and stops on the residual."""
    ne, nx = 3, 4
    ops = Q.Ops(ne, nx, 40.0, 100.0, 2e-3, "interleaved")
    n = ne + nx
    rhs = inputs.random_cores(n, 4, seed=31)
    x0 = inputs.random_cores(n, 16, seed=32, scale=0.1)
    x, info = tt.als(ops.Ap, [("vec", 1.0, rhs)], x0, max_sweeps=8, cg_max_iter=300, cg_tol=1e-3,
                     rel_tol=1e-12, stall=0.0)
    A = tt.full_mpo(ops.Ap)
    ref = spla.spsolve(sp.csr_matrix(A), tt.full(rhs))
    assert info["status"] == tt.CONVERGED and info["rel_residual"] <= 1e-12
    assert info["sweeps"] == len(info["history"]) - 1 and info["sweeps"] <= 8
    assert np.allclose(tt.full(x), ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_residual_is_entrywise_and_resolves_rounding_level():
    """The ALS stop test's residual ||A x - b|| / ||b|| equals the dense matrix-vector value, and
    for the exact solution it is at rounding level (~1e-15), far below the ~1e-8 floor of the
    expanded form ||Ax||^2 - 2 <b, Ax> + ||b||^2 (which cancels)."""
    ne, nx = 3, 4
    ops = Q.Ops(ne, nx, 40.0, 100.0, 2e-3, "interleaved")
    n = ne + nx
    x = inputs.random_cores(n, 16, seed=33)
    b = inputs.random_cores(n, 4, seed=34)
    bd = tt.full(b)
    A = tt.full_mpo(ops.Ap)
    want = np.linalg.norm(A @ tt.full(x) - bd) / np.linalg.norm(bd)
    assert abs(tt.residual(ops.Ap, x, bd, np.linalg.norm(bd)) - want) <= 1e-13 * want
    xs = np.linalg.solve(A, bd)
    xe = tt.tt_svd(xs, n, 2, 64)
    r = tt.residual(ops.Ap, xe, bd, np.linalg.norm(bd))
    assert r < 1e-13
    y = tt.mpo_mps(ops.Ap, xe)
    expanded = tt.dot(y, y) - 2 * tt.dot(b, y) + tt.dot(b, b)
    assert np.sqrt(abs(expanded)) / np.linalg.norm(bd) > 10 * r


def test_als_stop_rule_stalls_at_the_rank_floor():
    """At a bond below the solution's rank the ALS residual levels off (the truncation bounds it
    from below): the solve ends STALLED once a sweep gains less than the stall fraction; the energy
    1/2 <x, A x> - <b, x> never rises (every local CG step minimises it); max_sweeps ends an
    unfinished solve as MAX_SWEEPS; a solve that starts at the solution takes no sweep."""
    ne = nx = 4
    ops = Q.Ops(ne, nx, 40.0, 100.0, 2e-3, "interleaved")
    n = ne + nx
    rhs = inputs.random_cores(n, 16, seed=35)
    x0 = inputs.random_cores(n, 4, seed=36, scale=0.1)
    x, info = tt.als(ops.Ap, [("vec", 1.0, rhs)], x0, max_sweeps=30, cg_max_iter=500, cg_tol=1e-3,
                     rel_tol=1e-12, stall=0.05)
    h = info["history"]
    assert info["status"] == tt.STALLED
    assert h[-1] > 0.95 * h[-2] and all(b <= 0.95 * a for a, b in zip(h[:-2], h[1:-1]))
    assert info["rel_residual"] == h[-1] > 1e-6
    bd = tt.full(rhs)
    A = tt.full_mpo(ops.Ap)
    energy = []
    for s in range(1, 6):
        xs, _ = tt.als(ops.Ap, [("vec", 1.0, rhs)], x0, max_sweeps=s, cg_max_iter=500, cg_tol=1e-3,
                       rel_tol=0.0, stall=0.0)
        f = tt.full(xs)
        energy.append(0.5 * f @ (A @ f) - bd @ f)
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(energy, energy[1:]))
    _, info = tt.als(ops.Ap, [("vec", 1.0, rhs)], x0, max_sweeps=2, cg_max_iter=500, cg_tol=1e-3,
                     rel_tol=1e-14, stall=0.0)
    assert info["status"] == tt.MAX_SWEEPS and info["sweeps"] == 2
    xe = tt.tt_svd(np.linalg.solve(A, bd), n, 2, 256)
    _, info = tt.als(ops.Ap, [("vec", 1.0, rhs)], xe, max_sweeps=5, cg_max_iter=10, cg_tol=1e-3,
                     rel_tol=1e-10, stall=0.1)
    assert info["status"] == tt.CONVERGED and info["sweeps"] == 0 and info["cg_iters"] == 0


# ------------------------------------------------------------------ L0 step and diagnostics

def test_l0_poisson_and_projection_identity():
    """Sec. III.C: the pressure solves Lap_h p = div_h(v*)/dt exactly, and the corrected field
    satisfies the collocated-grid identity div_h(v+) = dt (Lap_h - D_x D_x^p - D_z D_z^p) p
    (grad_h . grad_h != Lap_h, so div_h(v+) is not machine zero)."""
    g = fd.Grid(5, 5, 40.0)
    case = fd.Case(g, 100.0, 2e-3)
    s = fd.FDSolver(case)
    u0 = 1.0 + inputs.gaussian_field(5, 5, 1, 1e-2)
    v0 = inputs.gaussian_field(5, 5, 2, 1e-2)
    un, vn, p, us, vs = s.step(u0, v0)
    b = s.grad_div(us, vs) / case.dt
    assert np.linalg.norm(s.Lp @ p - b) <= 1e-10 * np.linalg.norm(b)
    lhs = s.grad_div(un, vn)
    rhs = case.dt * (s.Lp @ p - s.vel["Dx"][0] @ (s.pre["Dx"][0] @ p) - s.vel["Dz"][0] @ (s.pre["Dz"][0] @ p))
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(lhs).max()


def test_l0_projection_second_order_in_interior():
    """For a smooth divergent field the projected divergence away from the boundary rows
    falls at (at least) second order under refinement: the wide-minus-compact stencil
    difference is O(h^2) (App. A stencils)."""
    ratios = []
    for n in (6, 7, 8):
        g = fd.Grid(n, n, 40.0)
        case = fd.Case(g, 100.0, 2e-3, u_inf=0.0)
        s = fd.FDSolver(case)
        x, z = g.xz()
        bump = np.exp(-((x - 3.0) ** 2 + (z - 1.0) ** 2) / 2.0)
        us, vs = (x - 3.0) * bump, 0.5 * (z - 1.0) * bump
        d0 = s.grad_div(us, vs)
        p = s._Plu.solve(d0 / case.dt)
        un = us.ravel() - case.dt * (s.pre["Dx"][0] @ p)
        vn = vs.ravel() - case.dt * (s.pre["Dz"][0] @ p)
        d1 = s.grad_div(un, vn).reshape(x.shape)
        k = 2 ** n // 8
        ratios.append(np.abs(d1[k:-k]).max() / np.abs(d0).max())
    assert ratios[1] < ratios[0] / 3.5 and ratios[2] < ratios[1] / 3.5


def test_forces_closed_forms():
    """App. F / eq:liftdrag: constant pressure gives no force; p_0 = cos(theta) with no flow
    gives C_D = -pi D (sum of cos^2 over the wall nodes), C_L = 0."""
    g = fd.Grid(4, 6, 40.0)
    case = fd.Case(g, 100.0, 2e-3)
    shape = (g.N_eta, g.N_xi)
    z = np.zeros(shape)
    cd, cl = fd.forces(case, z, z, np.full(shape, 3.0))
    assert abs(cd) < 1e-12 and abs(cl) < 1e-12
    th = g.theta(np.arange(g.N_xi))
    p = np.tile(np.cos(th), (g.N_eta, 1))
    cd, cl = fd.forces(case, z, z, p)
    assert abs(cd + np.pi * g.D) < 1e-12 and abs(cl) < 1e-12
    p = np.tile(np.sin(th), (g.N_eta, 1))
    cd, cl = fd.forces(case, z, z, p)
    assert abs(cl + np.pi * g.D) < 1e-12 and abs(cd) < 1e-12


def test_forces_viscous_closed_form():
    """App. F / eq:liftdrag, viscous part: for u = c (r - r_w), v = 0 (zero on the wall, no
    pressure) the wall stress sigma = -(2/(3Re)) div v I + (1/Re)(grad v + grad v^T) has
    traction t_x = (c/Re)((4/3) cos^2 + sin^2) on the outward normal, so C_D = 2 (7/3) pi c r_w / Re
    and C_L = 0; the same field in v gives that C_L and C_D = 0.  The one-sided second-order wall
    derivative converges to it at second order (a wrong factor, sign or a dropped divergence
    term changes the limit by 15-60 %)."""
    Re, c = 100.0, 0.7
    errs = []
    for n in (6, 7, 8):
        g = fd.Grid(n, 6, 40.0)
        case = fd.Case(g, Re, 2e-3)
        rr, _ = g.nodes()
        rw = g.r(-1)
        f = c * (rr - rw)
        z = np.zeros_like(f)
        want = 2 * (7 / 3) * np.pi * c * rw / Re
        cd, cl = fd.forces(case, f, z, z)
        cd2, cl2 = fd.forces(case, z, f, z)
        assert abs(cl) < 1e-15 and abs(cd2) < 1e-15
        assert abs(cl2 - cd) <= 1e-14 * abs(cd)
        errs.append(abs(cd / want - 1))
    assert errs[0] < 2e-3 and errs[1] < errs[0] / 3.5 and errs[2] < errs[1] / 3.5


def test_strouhal_from_zero_crossings():
    """eq:st: St = f D / U from the lift oscillation."""
    t = np.arange(0, 50, 0.013)
    cl = 0.3 + np.sin(2 * np.pi * 0.1937 * t + 0.4)
    assert abs(fd.strouhal(t, cl) - 0.1937) < 1e-4


@pytest.mark.parametrize("ordering", ["interleaved", "sequential"])
def test_l1_step_equals_l0_at_full_rank(ordering):
    """Whole step: with chi at full rank the QTT step (L1) equals the FD step (L0)."""
    ne = nx = 3
    R, Re, dt, chi = 40.0, 100.0, 2e-3, 8
    ops = Q.Ops(ne, nx, R, Re, dt, ordering)
    g = fd.Grid(ne, nx, R)
    L0 = fd.FDSolver(fd.Case(g, Re, dt))
    u0 = 1.0 + inputs.gaussian_field(ne, nx, 1, 1e-3)
    v0 = inputs.gaussian_field(ne, nx, 2, 1e-3)
    u, v = ops.encode(u0, chi), ops.encode(v0, chi)
    p = S.padded([np.zeros((1, 2, 1))] * (ne + nx), chi, inputs.random_cores(ne + nx, chi, 3, scale=1e-8))
    o = S.StepOpts(chi=chi, fit_sweeps=2, mom=S.SolveOpts(6, 1e-14, 200, 1e-3, 0.0),
                   poi=S.SolveOpts(8, 1e-13, 300, 1e-3, 0.0))
    un, vn, pn, info = S.step(ops, u, v, p, o)
    for k in "uvp":
        assert info[k]["status"] == tt.CONVERGED
    uf, vf, pf, _, _ = L0.step(u0, v0)
    for a, b in ((un, uf), (vn, vf), (pn, pf)):
        b = b.reshape(2 ** ne, 2 ** nx)
        assert np.abs(ops.decode(a) - b).max() <= 1e-10 * np.abs(b).max()


def test_extrapolated_warm_start_fit_and_step():
    """The extrapolated Poisson warm start: at full rank the fit reproduces 2 p^m - p^(m-1)
    exactly, and the step's answer does not depend on the warm start (solves converged)."""
    ne = nx = 3
    ops = Q.Ops(ne, nx, 40.0, 100.0, 2e-3, "interleaved")
    g = inputs.rng(31)
    p = ops.encode(g.standard_normal((2 ** ne, 2 ** nx)), 8)
    q = ops.encode(g.standard_normal((2 ** ne, 2 ** nx)), 8)
    f = tt.fit([("vec", 2.0, p), ("vec", -1.0, q)], p, 1)
    assert np.allclose(tt.full(f), 2 * tt.full(p) - tt.full(q), rtol=1e-12, atol=1e-12)
    u = ops.encode(1.0 + inputs.gaussian_field(ne, nx, 1, 1e-2), 8)
    v = ops.encode(inputs.gaussian_field(ne, nx, 2, 1e-2), 8)
    tight = dict(chi=8, fit_sweeps=2, mom=S.SolveOpts(20, 1e-13, 300, 1e-6, 0.0),
                 poi=S.SolveOpts(30, 1e-13, 500, 1e-6, 0.0))
    a = S.step(ops, u, v, p, S.StepOpts(**tight))
    b = S.step(ops, u, v, p, S.StepOpts(**tight, poisson_warm="extrapolated"), p_prev=q)
    for x, y in zip(a[:3], b[:3]):
        assert np.linalg.norm(tt.full(x) - tt.full(y)) <= 1e-9 * np.linalg.norm(tt.full(x))


def test_table2_rotating_cylinder_fd_sanity():
    """Table II (Sec. IV.B), FD row: rotating cylinder at Re = 100, rotation rate 1, grid G1,
    R = 32, dt = 2e-3 gives a mean lift coefficient 2.4908 and St 0.1663.  The L0 oracle's long
    run (tests/golden/table2_fd.txt, written by `python -m oracle.table2_run --time 160
    --window 60`) must reproduce both within 1 %: this pins the force read-out (pressure and
    viscous wall stress, App. F) and the Strouhal estimate on a developed periodic flow."""
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "table2_fd.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    assert abs(vals["mean_cl"] - 2.4908) <= 0.01 * 2.4908
    assert abs(vals["st"] - 0.1663) <= 0.01 * 0.1663
    assert vals["mean_cd"] > 0.0


@pytest.mark.parametrize("ne,nx,rot", [(3, 4, 0.0), (4, 5, 0.7), (5, 3, 1.3)])
def test_fft_direct_solver_equals_sparse_lu(ne, nx, rot):
    """The Fourier-in-xi, tridiagonal-in-eta solve of L0 (for grids too large for a sparse LU)
    is the same linear algebra as the sparse LU: the momentum and pressure systems on random
    right-hand sides, and a whole L0 step, agree to rounding (the block-circulant structure
    holds because the analytic metric depends on eta only)."""
    case = fd.Case(fd.Grid(ne, nx, 40.0), Re=100.0, dt=2e-3, rot=rot)
    lu, ff = fd.FDSolver(case, "lu"), fd.FDSolver(case, "fft")
    g = inputs.rng(ne * 10 + nx)
    n = case.grid.N_eta * case.grid.N_xi
    for M, a, b in ((lu.H, lu._Hlu, ff._Hlu), (lu.Lp, lu._Plu, ff._Plu)):
        rhs = g.standard_normal(n)
        x1, x2 = a.solve(rhs), b.solve(rhs)
        assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x1)
        assert np.linalg.norm(M @ x2 - rhs) <= 1e-11 * np.linalg.norm(rhs)
    u = 1.0 + 1e-2 * g.standard_normal(n)
    v = 1e-2 * g.standard_normal(n)
    for r1, r2 in zip(lu.step(u, v), ff.step(u, v)):
        assert np.linalg.norm(r1 - r2) <= 1e-12 * np.linalg.norm(r1)


def test_fft_direct_solver_rejects_coupling_beyond_neighbours():
    """A matrix coupling xi nodes two apart is not of the solver's form and is refused."""
    gr = fd.Grid(2, 3, 40.0)
    n = gr.N_eta * gr.N_xi
    M = sp.identity(n, format="csr") + sp.csr_matrix((np.ones(1), ([0], [2])), shape=(n, n))
    with pytest.raises(ValueError):
        fd.PeriodicXiSolver(M, gr)
