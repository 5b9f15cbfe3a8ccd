"""GPU parity of the cylinder case (operators, boundary vectors), the fractional step and the
forces against the FP64 oracle (L1 QTT step, L0 FD step), through the C ABI."""
import numpy as np
import pytest

from oracle import fd, tt, qtt_ops as Q, step as S
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


def make_state(ctx, ops, ne, nx, chi, seed=1, amp=1e-3):
    from paper_2507_05222_gb300 import qtt
    u0 = 1.0 + inputs.gaussian_field(ne, nx, seed, amp)
    v0 = inputs.gaussian_field(ne, nx, seed + 1, amp)
    u, v = ops.encode(u0, chi), ops.encode(v0, chi)
    p = S.padded([np.zeros((1, 2, 1))] * (ne + nx), chi, inputs.random_cores(ne + nx, chi, seed + 2, scale=1e-8))
    return (u, v, p), (qtt.MPS.from_cores(ctx, u), qtt.MPS.from_cores(ctx, v), qtt.MPS.from_cores(ctx, p)), (u0, v0)


@pytest.mark.parametrize("ordering,ne,nx,rot", [("interleaved", 3, 3, 0.0), ("sequential", 3, 4, 0.7),
                                               ("interleaved", 4, 3, 1.3)])
def test_case_operators_and_vectors(ctx, ordering, ne, nx, rot):
    """Sec. III.B.3 / App. A: every operator and boundary vector equals the oracle's."""
    from paper_2507_05222_gb300 import qtt
    R, Re, dt = 40.0, 100.0, 2e-3
    case = qtt.Case(ctx, ne, nx, R, Re, dt, 8, ordering, rot=rot)
    ops = Q.Ops(ne, nx, R, Re, dt, ordering, rot=rot)
    ref_ops = [ops.Dx, ops.Dz, ops.Dxp, ops.Dzp, ops.H, ops.Ap, ops.Px, ops.Pz]
    for w, M in enumerate(ref_ops):
        g = case.operator(w).cores()
        assert rel(tt.full_mpo(g), tt.full_mpo(M)) < 1e-13, w
        assert max(tt.bonds(g)) <= max(tt.bonds(M)) + 2
    ref_vec = [ops.bcx_u, ops.bcz_u, ops.bcx_v, ops.bcz_v, ops.JbcLap_u, ops.JbcLap_v, ops.bcdiv_w, ops.absJ]
    for w, x in enumerate(ref_vec):
        g = case.vector(w)
        if x is None:
            assert g is None, w
        else:
            assert rel(qtt.qtt_decode(ctx, g), tt.full(x)) < 1e-13, w


# Solve options with the local CG solves converged far below the parity bar (cg_tol 1e-10 of
# the global residual): the GPU and the oracle then differ in rounding only.  With the step's
# default cg_tol = 1e-2 a local CG stop that moves by one iteration on a last-digit difference
# moves the step by ~cg_tol x residual, which the full-size test below measures.
TIGHT_MOM = (6, 1e-10, 300, 1e-10, 0.1)
TIGHT_POI = (12, 1e-10, 600, 1e-10, 0.1)


def same_solves(info, oi, rtol=1e-3):
    """The GPU step's three solves took the oracle's sweep counts and stop decisions.  A solve
    that stalled or ran out of sweeps reports the residual of its last iterate, which must equal
    the oracle's to rtol of itself; a converged solve's residual is only known to be below its
    tolerance (both are).  CG counts agree to 5 % (a local CG stop can move by one iteration on a
    last-digit difference, at every site)."""
    for k in "uvp":
        g, o = info[k], oi[k]
        assert (g["sweeps"], g["status"]) == (o["sweeps"], o["status"]), (k, g, o)
        if g["status"] != 0:
            assert abs(g["rel_residual"] - o["rel_residual"]) <= rtol * o["rel_residual"], (k, g, o)
        assert abs(g["cg_iters"] - o["cg_iters"]) <= 0.05 * o["cg_iters"] + 4 * max(1, g["sweeps"]), (k, g, o)


def step_opts(chi, qtt, tight=True):
    mom, poi = (TIGHT_MOM, TIGHT_POI) if tight else (qtt.MOM_DEFAULT, qtt.POI_DEFAULT)
    return S.StepOpts(chi=chi, fit_sweeps=1, mom=S.SolveOpts(*mom), poi=S.SolveOpts(*poi))


@pytest.mark.parametrize("ordering,ne,nx,chi", [("interleaved", 3, 3, 8), ("sequential", 3, 3, 8),
                                               ("interleaved", 4, 4, 8)])
def test_one_step_matches_oracle(ctx, ordering, ne, nx, chi):
    """Sec. III.C: one fractional step equals the oracle's L1 step (same algorithm, solves swept
    to the true-residual stop rule)."""
    from paper_2507_05222_gb300 import qtt
    R, Re, dt = 40.0, 100.0, 2e-3
    ops = Q.Ops(ne, nx, R, Re, dt, ordering)
    (u, v, p), (gu, gv, gp), _ = make_state(ctx, ops, ne, nx, chi)
    case = qtt.Case(ctx, ne, nx, R, Re, dt, chi, ordering, mom=TIGHT_MOM, poi=TIGHT_POI)
    case.set_state(gu, gv, gp)
    info = case.fractional_step(1, with_forces=False, check=False)
    un, vn, pn, oi = S.step(ops, u, v, p, step_opts(chi, qtt))
    same_solves(info[0], oi)
    assert info[0]["finite"] == 1
    su, sv, sp = case.get_state()
    for g, r in ((su, un), (sv, vn), (sp, pn)):
        assert rel(qtt.qtt_decode(ctx, g), tt.full(r)) < TOL


def test_full_rank_steps_match_fd(ctx):
    """With chi at full rank and converged solves the GPU step equals the FD step (L0)."""
    from paper_2507_05222_gb300 import qtt
    ne = nx = 3
    R, Re, dt, chi = 40.0, 100.0, 2e-3, 8
    ops = Q.Ops(ne, nx, R, Re, dt, "interleaved")
    _, (gu, gv, gp), (u0, v0) = make_state(ctx, ops, ne, nx, chi)
    case = qtt.Case(ctx, ne, nx, R, Re, dt, chi, "interleaved", fit_sweeps=2, mom=(6, 1e-14, 200, 1e-3, 0.0),
                    poi=(8, 1e-13, 300, 1e-3, 0.0))
    case.set_state(gu, gv, gp)
    L0 = fd.FDSolver(fd.Case(fd.Grid(ne, nx, R), Re, dt))
    u, v = u0, v0
    for _ in range(3):
        info = case.fractional_step(1)
        assert all(info[0][k]["status"] == 0 for k in "uvp")
        u, v, p, _, _ = L0.step(u, v)
    su, sv, sp = case.get_state()
    for g, r in ((su, u), (sv, v), (sp, p)):
        r2 = Q.field_to_vec(np.reshape(r, (2 ** ne, 2 ** nx)), "interleaved")
        assert rel(qtt.qtt_decode(ctx, g), r2) < 1e-10


def test_forces_match_fd(ctx):
    """App. F: C_D, C_L of the GPU state equal the FD diagnostics on the decoded fields."""
    from paper_2507_05222_gb300 import qtt
    ne, nx = 4, 5
    R, Re, dt, chi = 40.0, 100.0, 2e-3, 16
    ops = Q.Ops(ne, nx, R, Re, dt, "interleaved", rot=0.8)
    _, (gu, gv, gp), _ = make_state(ctx, ops, ne, nx, chi, amp=1e-1)
    case = qtt.Case(ctx, ne, nx, R, Re, dt, chi, "interleaved", rot=0.8)
    case.set_state(gu, gv, gp)
    cd, cl = case.forces()
    su, sv, sp = case.get_state()
    f = [Q.vec_to_field(qtt.qtt_decode(ctx, g), ne, nx, "interleaved") for g in (su, sv, sp)]
    rcd, rcl = fd.forces(fd.Case(fd.Grid(ne, nx, R), Re, dt, rot=0.8), *f)
    assert abs(cd - rcd) <= 1e-10 * max(1.0, abs(rcd))
    assert abs(cl - rcl) <= 1e-10 * max(1.0, abs(rcl))


def wake_state(ops, ne, nx, chi, seed):
    u0, v0 = inputs.wake_field(ne, nx, seed)
    u, v = ops.encode(u0, chi), ops.encode(v0, chi)
    p = S.padded([np.zeros((1, 2, 1))] * (ne + nx), chi, inputs.random_cores(ne + nx, chi, seed + 2, scale=1e-8))
    return u, v, p


@pytest.mark.parametrize("seed", list(range(10)))
def test_multi_step_truncated_parity(ctx, seed):
    """Config 1 with truncation active: 12 bits (2^6 x 2^6 cells), chi = 16, ten steps from a
    seeded smooth wake state (a decaying spectrum, so no rounding cut falls inside a degenerate
    singular pair), solves under the step's stop rule with local CG converged to 1e-10 of the
    residual.  After every step each solve takes the oracle's sweeps and stop decision, and each
    field equals the oracle's to 1e-10 or, where the trajectory has amplified rounding beyond
    that (the truncated step amplifies a 2^-50 change ~1e5-fold over ten steps for some seeds),
    to ten times the oracle's own spread under a 2^-50 change of its initial pressure."""
    from paper_2507_05222_gb300 import qtt
    ne = nx = 6
    R, Re, dt, chi = 40.0, 100.0, 2e-3, 16
    ops = Q.Ops(ne, nx, R, Re, dt, "interleaved")
    u, v, p = wake_state(ops, ne, nx, chi, seed)
    q = (u, v, [c * (1.0 + 2.0 ** -50) for c in p])
    case = qtt.Case(ctx, ne, nx, R, Re, dt, chi, "interleaved", mom=TIGHT_MOM, poi=TIGHT_POI)
    case.set_state(*(qtt.MPS.from_cores(ctx, x) for x in (u, v, p)))
    o = step_opts(chi, qtt)
    for s in range(10):
        info = case.fractional_step(1, check=False)
        u, v, p, oi = S.step(ops, u, v, p, o)
        q = S.step(ops, *q, o)[:3]
        same_solves(info[0], oi)
        for k, g, r, r2 in zip("uvp", case.get_state(), (u, v, p), q):
            spread = rel(tt.full(r2), tt.full(r))
            d = rel(qtt.qtt_decode(ctx, g), tt.full(r))
            assert d < max(TOL, 10.0 * spread), (s, seed, k, d, spread)


def test_full_rank_12bit_step_matches_fd(ctx):
    """Config 1 at full rank: 12 bits with chi = 64 (= 2^6, no truncation anywhere), solves run to
    1e-14 or 30 sweeps (the FP64 floor of the Poisson residual is ~1e-13 here): three GPU steps
    equal three full-grid FD steps (L0), u and v to 1e-10; p, the solution of the Poisson problem
    (SPD, condition kappa ~1e4), to kappa times its relative residual (at least 1e-10)."""
    from paper_2507_05222_gb300 import qtt
    ne = nx = 6
    R, Re, dt, chi = 40.0, 100.0, 2e-3, 64
    ops = Q.Ops(ne, nx, R, Re, dt, "interleaved")
    u0 = 1.0 + inputs.gaussian_field(ne, nx, 3, 1e-3)
    v0 = inputs.gaussian_field(ne, nx, 4, 1e-3)
    p = S.padded([np.zeros((1, 2, 1))] * (ne + nx), chi, inputs.random_cores(ne + nx, chi, 5, scale=1e-8))
    case = qtt.Case(ctx, ne, nx, R, Re, dt, chi, "interleaved", fit_sweeps=2, mom=(30, 1e-14, 500, 1e-6, 0.0),
                    poi=(30, 1e-14, 800, 1e-6, 0.0))
    case.set_state(qtt.MPS.from_cores(ctx, ops.encode(u0, chi)), qtt.MPS.from_cores(ctx, ops.encode(v0, chi)),
                   qtt.MPS.from_cores(ctx, p))
    L0 = fd.FDSolver(fd.Case(fd.Grid(ne, nx, R), Re, dt))
    u, v = u0, v0
    for _ in range(3):
        info = case.fractional_step(1, check=False)
        for k in "uvp":
            assert info[0][k]["status"] in (0, 2) and info[0][k]["rel_residual"] < 1e-12, info[0][k]
        u, v, pf, _, _ = L0.step(u, v)
    lam = np.linalg.eigvalsh(tt.full_mpo(ops.Ap))
    kappa = lam[-1] / lam[0]
    bound_p = max(1e-10, kappa * info[0]["p"]["rel_residual"])
    for k, g, r in zip("uvp", case.get_state(), (u, v, pf)):
        r2 = Q.field_to_vec(np.reshape(r, (2 ** ne, 2 ** nx)), "interleaved")
        assert rel(qtt.qtt_decode(ctx, g), r2) < (bound_p if k == "p" else 1e-10), (k, kappa, bound_p)


def test_graph_replay_equals_eager(ctx):
    """The captured-graph step (default; the ALS sweep loops are conditional WHILE nodes whose
    trip counts the device decides) and kernel-by-kernel launching (the host reads the loop flag)
    give identical states and solve records (same kernels, deterministic reductions), also after
    set_state re-captures."""
    from paper_2507_05222_gb300 import qtt
    ne = nx = 5
    R, Re, dt, chi = 40.0, 100.0, 2e-3, 16
    ops = Q.Ops(ne, nx, R, Re, dt, "interleaved")
    _, (gu, gv, gp), _ = make_state(ctx, ops, ne, nx, chi)
    out = []
    for graph in (True, False, True):
        case = qtt.Case(ctx, ne, nx, R, Re, dt, chi, "interleaved")
        case.use_graph(graph)
        case.set_state(gu, gv, gp)
        info = case.fractional_step(3, with_forces=True, check=False)
        out.append(([qtt.qtt_decode(ctx, x) for x in case.get_state()], info))
    for (a, ia), (b, ib) in ((out[0], out[1]), (out[2], out[1])):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        assert ia == ib


@pytest.mark.parametrize("ne,nx,chi", [(5, 5, 16), (6, 6, 64)])
def test_cg_one_kernel_equals_per_stage(ctx, ne, nx, chi):
    """The local CG solves as one cooperative kernel give the per-stage kernels' iterates up to
    rounding order: the same sweep counts and stop decisions, states within the oracle parity
    bar (1e-10) after one step.  At chi = 64 the grid runs several work items per CTA in both
    contraction stages (the momentum solves run on half the SMs)."""
    from paper_2507_05222_gb300 import qtt
    R, Re, dt = 40.0, 100.0, 2e-3
    ops = Q.Ops(ne, nx, R, Re, dt, "interleaved")
    _, (gu, gv, gp), _ = make_state(ctx, ops, ne, nx, chi)
    out = []
    try:
        for mode in (0, 1):
            ctx.set_cg_mode(mode)
            case = qtt.Case(ctx, ne, nx, R, Re, dt, chi, "interleaved", mom=TIGHT_MOM, poi=TIGHT_POI)
            case.set_state(gu, gv, gp)
            info = case.fractional_step(1, with_forces=False, check=False)
            out.append(([qtt.qtt_decode(ctx, x) for x in case.get_state()], info))
    finally:
        ctx.set_cg_mode(0)
    (a, ia), (b, ib) = out
    for x, y in zip(a, b):
        assert rel(x, y) < TOL
    for k in "uvp":
        assert (ia[0][k]["sweeps"], ia[0][k]["status"]) == (ib[0][k]["sweeps"], ib[0][k]["status"])


def test_tensor_core_products_equal_fp64_pipe(ctx):
    """A step whose large contractions (chi = 64: 4096 x 128 x 64 environment products) run on
    the tensor cores by digit splitting equals the same step with every product on the FP64
    pipe, within the oracle parity bar after one step, with the same sweep counts."""
    from paper_2507_05222_gb300 import qtt
    ne = nx = 6
    R, Re, dt, chi = 40.0, 100.0, 2e-3, 64
    ops = Q.Ops(ne, nx, R, Re, dt, "interleaved")
    _, (gu, gv, gp), _ = make_state(ctx, ops, ne, nx, chi)
    out = []
    try:
        for mode in (0, 1):
            ctx.set_gemm_mode(mode)
            case = qtt.Case(ctx, ne, nx, R, Re, dt, chi, "interleaved", mom=TIGHT_MOM, poi=TIGHT_POI)
            case.set_state(gu, gv, gp)
            info = case.fractional_step(1, with_forces=False, check=False)
            out.append(([qtt.qtt_decode(ctx, x) for x in case.get_state()], info))
    finally:
        ctx.set_gemm_mode(0)
    (a, ia), (b, ib) = out
    for x, y in zip(a, b):
        assert rel(x, y) < TOL
    for k in "uvp":
        assert (ia[0][k]["sweeps"], ia[0][k]["status"]) == (ib[0][k]["sweeps"], ib[0][k]["status"])


def smooth_field(ne, nx, seed, amp, modes):
    """A field with a decaying QTT spectrum: modes products of a sine in xi and a cosine in eta
    (QTT rank <= 4 each) with amplitudes 2^(-k/2) and seeded phases, so that truncation to chi is
    active but the kept and discarded singular values stay apart (unlike i.i.d. noise, whose flat
    spectrum makes the chi-truncation non-unique)."""
    g = inputs.rng(seed)
    i = (np.arange(2 ** ne) + 0.5) / 2 ** ne
    j = np.arange(2 ** nx) / 2 ** nx
    f = np.zeros((2 ** ne, 2 ** nx))
    for k in range(1, modes + 1):
        ph, ps = g.uniform(0, 2 * np.pi, 2)
        f += 2.0 ** (-k / 2) * np.outer(np.cos(np.pi * k * i + ps), np.sin(2 * np.pi * k * j + ph))
    return amp * f


def headline_state(ctx, chi=64):
    from paper_2507_05222_gb300 import qtt
    ne = nx = 10
    ops = Q.Ops(ne, nx, 40.0, 200.0, 8e-4, "interleaved")
    u0 = 1.0 + smooth_field(ne, nx, 11, 1e-2, 24)
    v0 = smooth_field(ne, nx, 12, 1e-2, 24)
    u, v = ops.encode(u0, chi), ops.encode(v0, chi)
    p = S.padded([np.zeros((1, 2, 1))] * (ne + nx), chi, inputs.random_cores(ne + nx, chi, 13, scale=1e-8))
    return ops, (u, v, p)


def test_headline_operations_match_oracle(ctx):
    """The operations of the step at the timed size (2^20 cells, chi = 64), each against the
    oracle on the same input: MPO·MPS products with rounding, the Hadamard fit, and a
    momentum-operator ALS solve under the stop rule.  The products are held to the Gram-rounding
    limit: this state keeps singular values down to ~1e-14 sigma_1 in its bonds, and directions
    with sigma below sqrt(eps) sigma_1 are not resolved by a Gram eigenproblem, which leaves ~1e-8
    of the product (measured 5e-8 with tensor-core contractions, 1e-8 on the FP64 pipe).  The
    sketched rounding of the same products is held to 1e-10 in both product modes."""
    from paper_2507_05222_gb300 import qtt
    ops, (u, v, p) = headline_state(ctx)
    gu, gv = qtt.MPS.from_cores(ctx, u), qtt.MPS.from_cores(ctx, v)
    for M, x, gx in ((ops.Dx, u, gu), (ops.Dz, v, gv)):
        ref = tt.full(tt.round_tt(tt.mpo_mps(M, x), 64))
        g = qtt.mpo_apply_round(ctx, qtt.MPO.from_cores(ctx, M), gx, 64)
        assert rel(qtt.qtt_decode(ctx, g), ref) < 1e-6
        # the sketched rounding (no squared singular values) at the 1e-10 bar, with the
        # contractions on the tensor cores (digit split) and on the FP64 pipe
        try:
            for mode in (0, 1):
                ctx.set_gemm_mode(mode)
                g = qtt.mpo_apply_round(ctx, qtt.MPO.from_cores(ctx, M), gx, 64, apply="sketch")
                err = rel(qtt.qtt_decode(ctx, g), ref)
                print(f"sketched product, gemm mode {mode}: {err:.2e}")
                assert err < 1e-10
        finally:
            ctx.set_gemm_mode(0)
    ref = tt.full(tt.hadamard_round(u, v, 64, sweeps=2))
    g = qtt.mps_hadamard_round(ctx, gu, gv, 64, sweeps=2)
    assert rel(qtt.qtt_decode(ctx, g), ref) < 1e-11
    opts = (3, 1e-10, 300, 1e-10, 0.1)
    xr, ir = tt.als(ops.H, [("vec", 1.0, u)], u, opts[0], opts[2], opts[3], opts[1], opts[4])
    g = qtt.MPS.from_cores(ctx, u)
    gi = qtt.poisson_solve(ctx, qtt.MPO.from_cores(ctx, ops.H), qtt.MPS.from_cores(ctx, u), g, *opts)
    assert (gi["sweeps"], gi["status"]) == (ir["sweeps"], ir["status"])
    assert abs(gi["rel_residual"] - ir["rel_residual"]) <= 1e-3 * ir["rel_residual"]
    assert rel(qtt.qtt_decode(ctx, g), tt.full(xr)) < 1e-10


def test_headline_step_matches_oracle(ctx):
    """One step of the timed workload (2^20 cells as 10 + 10 interleaved bits, chi = 64, Re = 200,
    dt = 8e-4, R = 40, the seeded wake state and the solve options bench.py times, local CG to
    1e-2 of the global residual) through the captured CUDA graph bench.py replays, against the
    oracle's step on the same state.  Every solve runs to its stop rule; the step's sensitivity is
    measured here as the change of the oracle's own step under a 2^-50 relative change of the
    initial pressure (~1e-8 to 2e-7 per field: a local CG stop moving by one iteration moves the
    step by ~cg_tol x residual).  The GPU may differ from the oracle by at most ten times that
    spread (at least 1e-10); every solve takes the oracle's sweep count and stop decision, with
    the residuals of stalled solves within 3 % of the oracle's."""
    from paper_2507_05222_gb300 import qtt
    ne = nx = 10
    chi = 64
    ops = Q.Ops(ne, nx, 40.0, 200.0, 8e-4, "interleaved")
    u, v, p = wake_state(ops, ne, nx, chi, 7)
    o = step_opts(chi, qtt, tight=False)
    ref = S.step(ops, u, v, p, o)
    pert = S.step(ops, u, v, [c * (1.0 + 2.0 ** -50) for c in p], o)
    for apply in ("gram", "sketch"):
        case = qtt.Case(ctx, ne, nx, 40.0, 200.0, 8e-4, chi, "interleaved", apply=apply)
        case.use_graph(True)
        case.set_state(*(qtt.MPS.from_cores(ctx, x) for x in (u, v, p)))
        info = case.fractional_step(1, with_forces=True, check=False)
        same_solves(info[0], ref[3], rtol=3e-2)
        spreads, diffs = [], []
        for g, r, q in zip(case.get_state(), ref[:3], pert[:3]):
            full_r = tt.full(r)
            spreads.append(rel(tt.full(q), full_r))
            diffs.append(rel(qtt.qtt_decode(ctx, g), full_r))
        print(apply, "GPU - oracle:", diffs, "oracle spread:", spreads)
        for d_, s_ in zip(diffs, spreads):
            assert d_ <= max(10.0 * s_, 1e-10)
        assert max(diffs) < 2e-6
        assert info[0]["finite"] == 1 and np.isfinite(info[0]["cd"]) and np.isfinite(info[0]["cl"])


@pytest.mark.parametrize("seed", [0, 1])
def test_extrapolated_warm_start_steps_match_oracle(ctx, seed):
    """Three truncated steps (12 bits, chi = 16) with the extrapolated Poisson warm start
    (2 p^m - p^(m-1) fitted from p^m): every solve takes the oracle's sweeps and stop decision
    and each field equals the oracle's to 1e-10 or ten times the oracle's own spread under a
    2^-50 change of its initial pressure."""
    from paper_2507_05222_gb300 import qtt
    ne = nx = 6
    R, Re, dt, chi = 40.0, 100.0, 2e-3, 16
    ops = Q.Ops(ne, nx, R, Re, dt, "interleaved")
    u, v, p = wake_state(ops, ne, nx, chi, seed)
    q = (u, v, [c * (1.0 + 2.0 ** -50) for c in p])
    case = qtt.Case(ctx, ne, nx, R, Re, dt, chi, "interleaved", mom=TIGHT_MOM, poi=TIGHT_POI,
                    poisson_warm="extrapolated")
    case.set_state(*(qtt.MPS.from_cores(ctx, x) for x in (u, v, p)))
    o = step_opts(chi, qtt)
    o.poisson_warm = "extrapolated"
    pp, qp = None, None          # no previous pressure right after set_state
    for s in range(3):
        info = case.fractional_step(1, check=False)
        un, vn, pn, oi = S.step(ops, u, v, p, o, p_prev=pp)
        qn = S.step(ops, *q, o, p_prev=qp)[:3]
        pp, qp = p, q[2]
        u, v, p, q = un, vn, pn, qn
        same_solves(info[0], oi)
        for k, g, r, r2 in zip("uvp", case.get_state(), (u, v, p), q):
            spread = rel(tt.full(r2), tt.full(r))
            d = rel(qtt.qtt_decode(ctx, g), tt.full(r))
            assert d < max(TOL, 10.0 * spread), (s, seed, k, d, spread)


def rest_state(ne, nx, chi):
    """A flow at rest-like start: u = 1, v = 0, p = 0 held in the chi bond profile by N(0, 1e-8^2)
    padding (the exact rank-1 or zero block plus noise)."""
    def padded(value, seed):
        cores = inputs.random_cores(ne + nx, chi, seed, scale=1e-8)
        for k, c in enumerate(cores):
            c[0, :, 0] = value if k == 0 else (1.0 if value != 0.0 else 0.0)
        return cores
    return padded(1.0, 3), padded(0.0, 4), inputs.random_cores(ne + nx, chi, 5, scale=1e-8)


def test_truncated_steps_from_rest_match_oracle(ctx):
    """Ten truncated steps (5 + 6 bits, sequential order, chi = 8, Re = 20, dt = 1e-2) from the
    padded uniform start: the zero fields' trains have norms ~1e-80, so their products' Gram
    matrices test the eigensolver's scaling; each field equals the oracle's to 1e-10 or ten times
    the oracle's own spread under a 2^-50 change of its initial pressure; the pressure, the
    solution of an SPD system swept to a relative residual, also within kappa(A_p) times the sum
    of the two solves' residuals (the stop rule fixes p no closer than that)."""
    from paper_2507_05222_gb300 import qtt
    ne, nx, chi = 5, 6, 8
    R, Re, dt = 32.0, 20.0, 1e-2
    ops = Q.Ops(ne, nx, R, Re, dt, "sequential")
    lam = np.linalg.eigvalsh(tt.full_mpo(ops.Ap))
    kappa = lam[-1] / lam[0]
    u, v, p = rest_state(ne, nx, chi)
    q = (u, v, [c * (1.0 + 2.0 ** -50) for c in p])
    case = qtt.Case(ctx, ne, nx, R, Re, dt, chi, "sequential", mom=TIGHT_MOM, poi=TIGHT_POI)
    case.set_state(*(qtt.MPS.from_cores(ctx, x) for x in (u, v, p)))
    o = step_opts(chi, qtt)
    for s in range(10):
        info = case.fractional_step(1, check=False)
        u, v, p, oi = S.step(ops, u, v, p, o)
        q = S.step(ops, *q, o)[:3]
        assert info[0]["finite"] == 1
        kres = kappa * (info[0]["p"]["rel_residual"] + oi["p"]["rel_residual"])
        for k, g, r, r2 in zip("uvp", case.get_state(), (u, v, p), q):
            spread = rel(tt.full(r2), tt.full(r))
            d = rel(qtt.qtt_decode(ctx, g), tt.full(r))
            assert d < max(TOL, 10.0 * spread, kres if k == "p" else 0.0), (s, k, d, spread, kres)
