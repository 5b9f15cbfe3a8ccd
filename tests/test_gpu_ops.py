"""GPU parity of the TT operations (C ABI) against the FP64 oracle, element by element on
reconstructed vectors.  Tolerance: relative 1e-10 in FP64 (the figure the hot path is held
to); cases are chosen so that no truncation falls inside a near-degenerate singular-value
pair (where the TT-SVD itself is not unique)."""
import numpy as np
import pytest

from oracle import tt, qtt_ops as Q
from paper_2507_05222_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2507_05222_gb300 import qtt
    return qtt.Context(0)


def rel(a, b):
    a = np.asarray(a).ravel(); b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def up(ctx, cores):
    from paper_2507_05222_gb300 import qtt
    return qtt.MPS.from_cores(ctx, cores)


def down(ctx, x):
    from paper_2507_05222_gb300 import qtt
    return qtt.qtt_decode(ctx, x)


def test_mps_roundtrip_and_decode(ctx):
    x = inputs.random_cores(7, 5, seed=1)
    g = up(ctx, x)
    back = g.cores()
    for a, b in zip(back, x):
        assert np.array_equal(a, b)
    assert rel(down(ctx, g), tt.full(x)) < 1e-14


@pytest.mark.parametrize("n,chi", [(10, 32), (10, 7), (11, 4), (1, 1), (2, 1)])
def test_encode(ctx, n, chi):
    from paper_2507_05222_gb300 import qtt
    v = inputs.dense_vector(n, seed=n + chi)
    ref = tt.tt_svd(v, n, 2, chi)
    g = qtt.qtt_encode(ctx, v, n, chi)
    assert g.bonds() == tt.bonds(ref)
    assert rel(down(ctx, g), tt.full(ref)) < TOL


def test_encode_smooth_field_low_rank(ctx):
    """Rank-2 trig field encodes to rank 2 under a threshold (Sec. III.B.1)."""
    from paper_2507_05222_gb300 import qtt
    n = 12
    q = np.arange(2 ** n)
    f = np.sin(2 * np.pi * q / 2 ** n * 3 + 0.2)
    g = qtt.qtt_encode(ctx, f, n, 64, rel_tol=1e-10)
    assert max(g.bonds()) == 2
    assert rel(down(ctx, g), f) < 1e-12


@pytest.mark.parametrize("n,bond,chi", [(10, 12, 5), (9, 16, 16), (8, 6, 3), (12, 10, 8)])
def test_round(ctx, n, bond, chi):
    from paper_2507_05222_gb300 import qtt
    x = inputs.random_cores(n, bond, seed=3 * n + bond)
    ref = tt.round_tt(x, chi)
    g = qtt.qtt_round(ctx, up(ctx, x), chi)
    assert g.bonds() == tt.bonds(ref)
    assert rel(down(ctx, g), tt.full(ref)) < TOL
    # right-canonical output (Sec. II); the eigenvectors of the tiniest Gram eigenvalues are
    # orthonormal to ~1e-11 after refinement
    for c in g.cores()[1:]:
        m = c.reshape(c.shape[0], -1)
        assert np.abs(m @ m.T - np.eye(c.shape[0])).max() < 1e-10


def test_round_eps_threshold(ctx):
    from paper_2507_05222_gb300 import qtt
    a = Q.mps1_trig(9, 0.1, 0.0, "sin"); b = Q.mps1_trig(9, 0.1, 0.3, "cos")
    s = tt.direct_sum(1.0, a, 2.0, b)
    g = qtt.qtt_round(ctx, up(ctx, s), 100, rel_tol=1e-14)
    assert max(g.bonds()) == 2
    assert rel(down(ctx, g), tt.full(s)) < 1e-13


@pytest.mark.parametrize("n,ba,bb,chi", [(10, 8, 6, 8), (9, 4, 4, 16), (12, 10, 9, 6)])
def test_axpby(ctx, n, ba, bb, chi):
    from paper_2507_05222_gb300 import qtt
    x = inputs.random_cores(n, ba, seed=10 + n); y = inputs.random_cores(n, bb, seed=20 + n)
    ref = tt.round_tt(tt.direct_sum(0.7, x, -1.3, y), chi)
    g = qtt.mps_axpby_round(ctx, 0.7, up(ctx, x), -1.3, up(ctx, y), chi)
    assert g.bonds() == tt.bonds(ref)
    assert rel(down(ctx, g), tt.full(ref)) < TOL


@pytest.mark.parametrize("n,bx,w,chi", [(9, 6, 3, 6), (10, 8, 4, 32), (8, 5, 2, 4)])
def test_apply_random(ctx, n, bx, w, chi):
    from paper_2507_05222_gb300 import qtt
    x = inputs.random_cores(n, bx, seed=30 + n)
    M = inputs.random_mpo_cores(n, w, seed=40 + n)
    ref = tt.round_tt(tt.mpo_mps(M, x), chi)
    g = qtt.mpo_apply_round(ctx, qtt.MPO.from_cores(ctx, M), up(ctx, x), chi)
    assert g.bonds() == tt.bonds(ref)
    assert rel(down(ctx, g), tt.full(ref)) < TOL


def test_round_info_discarded_norm(ctx):
    """qtt_round_info: the discarded norm of every rounding entry point equals the oracle's
    TT-SVD value (which equals the true rounding error), and norm and max bond are the result's.
    Gram (rel_tol = 0) and thresholded QR + SVD paths both; -1 for the Hadamard fit."""
    from paper_2507_05222_gb300 import qtt
    x = inputs.random_cores(10, 16, seed=5)
    y = inputs.random_cores(10, 8, seed=6)
    M = inputs.random_mpo_cores(10, 3, seed=7)
    cases = [
        (lambda info: qtt.qtt_round(ctx, up(ctx, x), 6, out_info=info), tt.full(x), x, 6),
        (lambda info: qtt.mps_axpby_round(ctx, 0.7, up(ctx, x), -1.3, up(ctx, y), 10, out_info=info),
         tt.full(tt.direct_sum(0.7, x, -1.3, y)), tt.direct_sum(0.7, x, -1.3, y), 10),
        (lambda info: qtt.mpo_apply_round(ctx, qtt.MPO.from_cores(ctx, M), up(ctx, x), 12, out_info=info),
         tt.full(tt.mpo_mps(M, x)), tt.mpo_mps(M, x), 12),
        (lambda info: qtt.qtt_encode(ctx, tt.full(x), 10, 8, out_info=info), tt.full(x), x, 8),
    ]
    for call, exact, cores, chi in cases:
        info = {}
        g = call(info)
        ref = {}
        r = tt.round_tt(cores, chi, info=ref)
        assert abs(info["discarded_norm"] - ref["discarded_norm"]) <= 1e-9 * np.linalg.norm(exact)
        assert abs(info["discarded_norm"] - np.linalg.norm(exact - down(ctx, g))) <= 1e-9 * np.linalg.norm(exact)
        assert abs(info["norm"] - np.linalg.norm(tt.full(r))) <= 1e-12 * np.linalg.norm(tt.full(r))
        assert info["max_bond"] == max(tt.bonds(r))
    info = {}
    a = Q.mps1_trig(9, 0.1, 0.0, "sin"); b = Q.mps1_trig(9, 0.1, 0.3, "cos")
    s = tt.direct_sum(1.0, a, 2.0, b)
    qtt.qtt_round(ctx, up(ctx, s), 100, rel_tol=1e-14, out_info=info)
    assert info["max_bond"] == 2 and info["discarded_norm"] <= 1e-13 * np.linalg.norm(tt.full(s))
    info = {}
    qtt.mps_hadamard_round(ctx, up(ctx, y), up(ctx, y), 8, out_info=info)
    assert info["discarded_norm"] == -1.0


@pytest.mark.parametrize("ordering", ["interleaved", "sequential"])
def test_apply_fd_operator_exact(ctx, ordering):
    """Curvilinear D_x of a smooth field without truncation equals the dense product."""
    from paper_2507_05222_gb300 import qtt
    ne, nx = 4, 5
    ops = Q.Ops(ne, nx, 40.0, 100.0, 2e-3, ordering)
    f = inputs.gaussian_field(ne, nx, 5, 1.0)
    x = ops.encode(f, 64)
    g = qtt.mpo_apply_round(ctx, qtt.MPO.from_cores(ctx, ops.Dx), up(ctx, x), 512)
    assert rel(down(ctx, g), tt.full_mpo(ops.Dx) @ tt.full(x)) < TOL


@pytest.mark.parametrize("n,ba,bb,chi", [(8, 4, 3, 6), (10, 5, 5, 8)])
def test_hadamard_fit(ctx, n, ba, bb, chi):
    from paper_2507_05222_gb300 import qtt
    a = inputs.random_cores(n, ba, seed=50 + n); b = inputs.random_cores(n, bb, seed=60 + n)
    ref = tt.hadamard_round(a, b, chi, sweeps=2)
    g = qtt.mps_hadamard_round(ctx, up(ctx, a), up(ctx, b), chi, sweeps=2)
    assert g.bonds() == tt.bonds(ref)
    assert rel(down(ctx, g), tt.full(ref)) < TOL


def test_hadamard_exact_low_rank(ctx):
    """sin (.) exp has rank 2: the fit reproduces the pointwise product (Sec. II.A.3)."""
    from paper_2507_05222_gb300 import qtt
    n = 11
    a = Q.mps1_trig(n, 0.013, 0.3, "sin"); b = Q.mps1_exp(n, 1.0, 0.001)
    g = qtt.mps_hadamard_round(ctx, up(ctx, a), up(ctx, b), 4, sweeps=2)
    assert rel(down(ctx, g), tt.full(a) * tt.full(b)) < 1e-12


def test_dot(ctx):
    from paper_2507_05222_gb300 import qtt
    a = inputs.random_cores(11, 7, seed=70); b = inputs.random_cores(11, 5, seed=71)
    v = qtt.mps_dot(ctx, up(ctx, a), up(ctx, b))
    ref = float(tt.full(a) @ tt.full(b))
    assert abs(v - ref) <= 1e-12 * np.linalg.norm(tt.full(a)) * np.linalg.norm(tt.full(b))


@pytest.fixture(params=[0, 1, 2, 3], ids=["cg_default", "cg_per_stage", "cg_one_kernel_fp64",
                                          "cg_one_kernel_tensor_cores"])
def cg_mode(ctx, request):
    ctx.set_cg_mode(request.param)
    yield request.param
    ctx.set_cg_mode(0)


def test_poisson_solve_matches_oracle_als(ctx, cg_mode):
    """ALS (Sec. II.A.4) under the true-residual stop rule, same options as the oracle: the same
    sweep count, status and CG count, the residual to 1e-8 of itself, the solution at 1e-10."""
    from paper_2507_05222_gb300 import qtt
    ne, nx = 4, 4
    ops = Q.Ops(ne, nx, 40.0, 100.0, 2e-3, "interleaved")
    n = ne + nx
    b = inputs.random_cores(n, 4, seed=80)
    x0 = inputs.random_cores(n, 8, seed=81, scale=0.1)
    opts = (8, 1e-10, 300, 1e-10, 0.1)
    ref, ir = tt.als(ops.Ap, [("vec", 1.0, b)], x0, *opts[:1], opts[2], opts[3], opts[1], opts[4])
    g = up(ctx, x0)
    gi = qtt.poisson_solve(ctx, qtt.MPO.from_cores(ctx, ops.Ap), up(ctx, b), g, *opts)
    assert (gi["sweeps"], gi["status"]) == (ir["sweeps"], ir["status"])
    assert abs(gi["cg_iters"] - ir["cg_iters"]) <= 2
    assert abs(gi["rel_residual"] - ir["rel_residual"]) <= 1e-3 * ir["rel_residual"] + 1e-13
    assert gi["rc"] == (0 if ir["status"] == tt.CONVERGED else -4)
    assert rel(down(ctx, g), tt.full(ref)) < TOL


def test_poisson_solve_full_rank_exact(ctx, cg_mode):
    """At full bond dimension the ALS solution equals the dense solve (J-weighted Poisson) and the
    solve stops as converged on its true residual."""
    from paper_2507_05222_gb300 import qtt
    ne, nx = 3, 4
    ops = Q.Ops(ne, nx, 40.0, 100.0, 2e-3, "interleaved")
    n = ne + nx
    b = inputs.random_cores(n, 4, seed=82)
    x0 = inputs.random_cores(n, 16, seed=83, scale=0.1)
    g = up(ctx, x0)
    gi = qtt.poisson_solve(ctx, qtt.MPO.from_cores(ctx, ops.Ap), up(ctx, b), g, 10, 1e-12, 300, 1e-3, 0.0)
    ref = np.linalg.solve(tt.full_mpo(ops.Ap), tt.full(b))
    assert gi["status"] == 0 and gi["rc"] == 0 and gi["rel_residual"] <= 1e-12
    A = tt.full_mpo(ops.Ap)
    x = down(ctx, g)
    assert abs(gi["rel_residual"] - np.linalg.norm(A @ x - tt.full(b)) / np.linalg.norm(tt.full(b))) < 1e-14
    assert rel(x, ref) < 1e-10


def test_poisson_solve_statuses(ctx):
    """Stop-rule outcomes through the C ABI: out of sweeps returns QTT_ERR_NOT_CONVERGED with the
    last iterate (equal to the oracle's after the same sweeps); a stall at the bond's floor
    likewise; a start at the solution takes no sweep; max_sweeps = 0 returns the warm start."""
    from paper_2507_05222_gb300 import qtt
    ne = nx = 4
    ops = Q.Ops(ne, nx, 40.0, 100.0, 2e-3, "interleaved")
    n = ne + nx
    rhs = inputs.random_cores(n, 16, seed=35)
    x0 = inputs.random_cores(n, 4, seed=36, scale=0.1)
    A = qtt.MPO.from_cores(ctx, ops.Ap)
    g = up(ctx, x0)
    gi = qtt.poisson_solve(ctx, A, up(ctx, rhs), g, 2, 1e-14, 500, 1e-10, 0.0)
    ref, ir = tt.als(ops.Ap, [("vec", 1.0, rhs)], x0, 2, 500, 1e-10, 1e-14, 0.0)
    assert gi["rc"] == -4 and gi["status"] == 2 == ir["status"] and gi["sweeps"] == 2
    assert rel(down(ctx, g), tt.full(ref)) < TOL
    with pytest.raises(qtt.QttError) as e:
        qtt.poisson_solve(ctx, A, up(ctx, rhs), up(ctx, x0), 2, 1e-14, 500, 1e-3, 0.0, check=True)
    assert e.value.code == -4
    g = up(ctx, x0)
    gi = qtt.poisson_solve(ctx, A, up(ctx, rhs), g, 30, 1e-12, 500, 1e-10, 0.05)
    ref, ir = tt.als(ops.Ap, [("vec", 1.0, rhs)], x0, 30, 500, 1e-10, 1e-12, 0.05)
    assert gi["status"] == 1 == ir["status"] and gi["sweeps"] == ir["sweeps"] and gi["rc"] == -4
    assert rel(down(ctx, g), tt.full(ref)) < TOL
    xe = tt.tt_svd(np.linalg.solve(tt.full_mpo(ops.Ap), tt.full(rhs)), n, 2, 256)
    g = up(ctx, xe)
    gi = qtt.poisson_solve(ctx, A, up(ctx, rhs), g, 5, 1e-10, 10, 1e-3, 0.1)
    assert gi["status"] == 0 and gi["sweeps"] == 0 and gi["cg_iters"] == 0 and gi["rc"] == 0
    g = up(ctx, x0)
    gi = qtt.poisson_solve(ctx, A, up(ctx, rhs), g, 0, 1e-10, 10, 1e-3, 0.1)
    assert gi["status"] == 2 and gi["sweeps"] == 0 and rel(down(ctx, g), tt.full(x0)) < 1e-14


def test_poisson_solve_tensor_core_cg_equals_fp64(ctx):
    """ALS local solves at bonds 64 (n = 12, the middle sites hold 64 x 2 x 64 cores): the
    cooperative CG with both contractions as digit-split tensor-core products (mode 3) against
    the same kernel structure on the FP64 pipe (mode 2), the per-stage kernels (mode 1) and the
    default mix (mode 0: tensor cores at the full-bond sites), each solve run to its true-residual
    stop rule: the same sweep counts and statuses, solutions within 1e-10."""
    from paper_2507_05222_gb300 import qtt
    ne, nx = 6, 6
    ops = Q.Ops(ne, nx, 40.0, 100.0, 2e-3, "interleaved")
    n = ne + nx
    b = inputs.random_cores(n, 16, seed=84)
    x0 = inputs.random_cores(n, 64, seed=85, scale=0.1)
    out = []
    try:
        for mode in (3, 2, 1, 0):
            ctx.set_cg_mode(mode)
            g = up(ctx, x0)
            gi = qtt.poisson_solve(ctx, qtt.MPO.from_cores(ctx, ops.Ap), up(ctx, b), g, 8, 1e-11, 600, 1e-10, 0.1)
            out.append((down(ctx, g), gi))
    finally:
        ctx.set_cg_mode(0)
    (x_tc, i_tc), (x_64, i_64), (x_ps, i_ps), (x_d, i_d) = out
    assert rel(x_64, x_ps) < 1e-10
    assert rel(x_tc, x_64) < 1e-10
    assert rel(x_d, x_64) < 1e-10
    for i in (i_tc, i_ps, i_d):
        assert (i["sweeps"], i["status"]) == (i_64["sweeps"], i_64["status"])
        assert abs(i["rel_residual"] - i_64["rel_residual"]) <= 1e-3 * i_64["rel_residual"] + 1e-12


def test_field_reorder(ctx):
    from paper_2507_05222_gb300 import qtt
    f = np.arange(8 * 32, dtype=float).reshape(8, 32)
    for o in ("sequential", "interleaved"):
        v = qtt.qtt_field_to_vector(ctx, f, o)
        assert np.array_equal(v, Q.field_to_vec(f, o))
        assert np.array_equal(qtt.qtt_vector_to_field(ctx, v, 3, 5, o), f)


def test_argument_errors(ctx):
    from paper_2507_05222_gb300 import qtt
    x = up(ctx, inputs.random_cores(6, 3, seed=1))
    y = up(ctx, inputs.random_cores(7, 3, seed=2))
    with pytest.raises(qtt.QttError) as e:
        qtt.mps_axpby_round(ctx, 1.0, x, 1.0, y, 4)
    assert e.value.code == -1
    with pytest.raises(qtt.QttError):
        qtt.qtt_round(ctx, x, 0)


def test_apply_round_of_a_near_zero_train(ctx):
    """MPO-MPS product of a field held at zero inside the chi bond profile by 1e-8 padding (norm
    ~1e-80, the start of a flow at rest): the Gram matrices are ~1e-160 and must still give the
    oracle's product to 1e-10 (they vanished in the FP32 stage before the eigensolver scaled
    its input)."""
    from paper_2507_05222_gb300 import qtt
    ne, nx, chi = 5, 5, 16
    ops = Q.Ops(ne, nx, 32.0, 20.0, 1e-2, "sequential")
    cores = inputs.random_cores(ne + nx, chi, 4, scale=1e-8)
    for c in cores:
        c[0, :, 0] = 0.0
    ref = tt.full(tt.round_tt(tt.mpo_mps(ops.Dx, cores), chi))
    assert 0.0 < np.linalg.norm(ref) < 1e-60
    y = qtt.mpo_apply_round(ctx, qtt.MPO.from_cores(ctx, ops.Dx), qtt.MPS.from_cores(ctx, cores), chi)
    d = qtt.qtt_decode(ctx, y)
    assert np.linalg.norm(d - ref) <= 1e-10 * np.linalg.norm(ref)
