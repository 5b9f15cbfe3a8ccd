"""Batched stepping of independent cylinder cases (Sec. III.C per case; the rotating-wall
boundary condition of Sec. IV.B): cases of different grids, bond caps, Reynolds numbers and
rotation rates advanced together by fractional_step_batch, each graph replayed concurrently on
its own stream.  Every case must equal the oracle's L1 step and be bit-identical to the same
case stepped alone."""
import numpy as np
import pytest

from oracle import tt, qtt_ops as Q, step as S
from paper_2507_05222_gb300 import inputs

pytestmark = pytest.mark.gpu
TIGHT_MOM = (6, 1e-10, 300, 1e-10, 0.1)
TIGHT_POI = (12, 1e-10, 600, 1e-10, 0.1)
# (ordering, n_eta, n_xi, chi, Re, dt, rotation rate)
MIX = [("interleaved", 3, 3, 8, 100.0, 2e-3, 0.0),
       ("interleaved", 4, 4, 8, 60.0, 2e-3, 1.0),
       ("sequential", 3, 4, 8, 150.0, 1e-3, 0.5),
       ("interleaved", 4, 5, 16, 40.0, 2e-3, 2.0)]
R = 40.0


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


def start_state(ne, nx, chi, seed, ops):
    u0 = 1.0 + inputs.gaussian_field(ne, nx, seed, 1e-3)
    v0 = inputs.gaussian_field(ne, nx, seed + 1, 1e-3)
    u, v = ops.encode(u0, chi), ops.encode(v0, chi)
    p = S.padded([np.zeros((1, 2, 1))] * (ne + nx), chi, inputs.random_cores(ne + nx, chi, seed + 2, scale=1e-8))
    return u, v, p


def make_case(ctx, spec, state, mom=TIGHT_MOM, poi=TIGHT_POI):
    from paper_2507_05222_gb300 import qtt
    ordering, ne, nx, chi, Re, dt, rot = spec
    case = qtt.Case(ctx, ne, nx, R, Re, dt, chi, ordering, rot=rot, mom=mom, poi=poi)
    case.set_state(*[qtt.MPS.from_cores(ctx, x) for x in state])
    return case


def test_batch_matches_oracle_and_single_cases(ctx):
    from paper_2507_05222_gb300 import qtt
    nsteps = 2
    opsl = [Q.Ops(ne, nx, R, Re, dt, o, rot=rot) for (o, ne, nx, chi, Re, dt, rot) in MIX]
    states = [start_state(s[1], s[2], s[3], 10 * i, ops) for i, (s, ops) in enumerate(zip(MIX, opsl))]
    # each case alone, each created, stepped and freed in turn (graph arenas released in between)
    alone = []
    for spec, st in zip(MIX, states):
        case = make_case(ctx, spec, st)
        case.fractional_step(nsteps)
        alone.append([qtt.qtt_decode(ctx, g) for g in case.get_state()])
        del case
    cases = [make_case(ctx, spec, st) for spec, st in zip(MIX, states)]
    recs, status = qtt.fractional_step_batch(ctx, cases, nsteps, with_forces=True)
    assert status == [0] * len(MIX)
    for i, (spec, ops, st, case) in enumerate(zip(MIX, opsl, states, cases)):
        got = [qtt.qtt_decode(ctx, g) for g in case.get_state()]
        for a, b in zip(got, alone[i]):
            assert np.array_equal(a, b), i          # concurrency changes nothing
        # the oracle, and the oracle from a 2^-50 change of the initial pressure: a field may
        # differ from the oracle by 1e-10 or by ten times that spread, whichever is larger (the
        # truncated steps amplify rounding-level differences, mostly in the pressure)
        u, v, p = st
        q = (u, v, [c * (1.0 + 2.0 ** -50) for c in p])
        opts = S.StepOpts(chi=spec[3], fit_sweeps=1, mom=S.SolveOpts(*TIGHT_MOM), poi=S.SolveOpts(*TIGHT_POI))
        for s in range(nsteps):
            u, v, p, oi = S.step(ops, u, v, p, opts)
            q = S.step(ops, *q, opts)[:3]
            for k in "uvp":
                assert (recs[i][s][k]["sweeps"], recs[i][s][k]["status"]) == (oi[k]["sweeps"], oi[k]["status"])
        for k, g, r, r2 in zip("uvp", got, (u, v, p), q):
            spread = rel(tt.full(r2), tt.full(r))
            d = rel(g, tt.full(r))
            print(f"case {i} {k}: GPU - oracle {d:.2e}, oracle spread {spread:.2e}")
            assert d < max(1e-10, 10.0 * spread), (i, k, d, spread)
        assert all(np.isfinite([r["cd"], r["cl"]]).all() for r in recs[i])


def test_batch_reports_status_per_case(ctx):
    from paper_2507_05222_gb300 import qtt
    opsl = [Q.Ops(ne, nx, R, Re, dt, o, rot=rot) for (o, ne, nx, chi, Re, dt, rot) in MIX[:3]]
    states = [start_state(s[1], s[2], s[3], 10 * i, ops) for i, (s, ops) in enumerate(zip(MIX[:3], opsl))]
    # the middle case's Poisson solve gets one sweep for an unreachable tolerance
    cases = [make_case(ctx, MIX[0], states[0]),
             make_case(ctx, MIX[1], states[1], poi=(1, 1e-15, 50, 1e-2, 0.0)),
             make_case(ctx, MIX[2], states[2])]
    with pytest.raises(qtt.QttError) as e:
        qtt.fractional_step_batch(ctx, cases, 1)
    assert e.value.code == -4
    assert e.value.statuses == [0, -4, 0]
    assert "case 1" in str(e.value)
    assert e.value.records[1][0]["p"]["sweeps"] == 1


def test_batch_argument_errors(ctx):
    from paper_2507_05222_gb300 import qtt
    ops = Q.Ops(3, 3, R, 100.0, 2e-3, "interleaved")
    st = start_state(3, 3, 8, 0, ops)
    a, b = make_case(ctx, MIX[0], st), make_case(ctx, MIX[0], st)
    for bad in ([a, a], []):
        with pytest.raises(qtt.QttError) as e:
            qtt.fractional_step_batch(ctx, bad, 1)
        assert e.value.code == -1
    b.use_graph(False)
    with pytest.raises(qtt.QttError) as e:
        qtt.fractional_step_batch(ctx, [a, b], 1)
    assert e.value.code == -1


def test_autotuner_picks_and_products(ctx):
    """The GEMM autotuner times each new shape under every candidate engine and keeps the
    fastest; a tuned product is still the FP64 product (every engine is FP64-accurate)."""
    from paper_2507_05222_gb300 import qtt
    c2 = qtt.Context(0)
    c2.set_autotune(1)
    g = inputs.rng(5)
    shapes = [(96, 80, 64), (300, 70, 129), (128, 512, 96), (1024, 64, 576)]
    for m, n, k in shapes:
        A, B = g.standard_normal((m, k)), g.standard_normal((k, n))
        C = qtt.qtt_dgemm(c2, A, B, path=0)
        ref = A @ B
        assert np.linalg.norm(C - ref) <= 1e-14 * np.linalg.norm(np.abs(A) @ np.abs(B)), (m, n, k)
    table = c2.autotune_table()
    assert sorted((r["M"], r["N"], r["K"]) for r in table) == sorted(shapes)
    for r in table:
        assert r["engine"] in (0, 1) and 0 < r["best_ns"] <= r["default_ns"], r
    qtt.qtt_dgemm(c2, A, B, path=0)
    assert len(c2.autotune_table()) == len(shapes)     # a known shape is not tuned again
    c2.set_autotune(-1)
    assert c2.autotune_table() == []


def test_autotuned_batch_matches_oracle(ctx):
    """Cases stepped with the tuner on (shapes tuned while the step graphs are captured) still
    equal the oracle's step."""
    from paper_2507_05222_gb300 import qtt
    c2 = qtt.Context(0)
    c2.set_autotune(1)
    mix = [MIX[1], MIX[3]]
    opsl = [Q.Ops(ne, nx, R, Re, dt, o, rot=rot) for (o, ne, nx, chi, Re, dt, rot) in mix]
    states = [start_state(s[1], s[2], s[3], 7 + i, ops) for i, (s, ops) in enumerate(zip(mix, opsl))]
    cases = [make_case(c2, spec, st) for spec, st in zip(mix, states)]
    recs, status = qtt.fractional_step_batch(c2, cases, 1)
    assert status == [0, 0]
    assert len(c2.autotune_table()) > 0
    for spec, ops, st, case in zip(mix, opsl, states, cases):
        u, v, p = st
        q = (u, v, [c * (1.0 + 2.0 ** -50) for c in p])
        opts = S.StepOpts(chi=spec[3], fit_sweeps=1, mom=S.SolveOpts(*TIGHT_MOM), poi=S.SolveOpts(*TIGHT_POI))
        r = S.step(ops, u, v, p, opts)[:3]
        r2 = S.step(ops, *q, opts)[:3]
        for k, g, a, b in zip("uvp", case.get_state(), r, r2):
            spread = rel(tt.full(b), tt.full(a))
            d = rel(qtt.qtt_decode(c2, g), tt.full(a))
            assert d < max(1e-10, 10.0 * spread), (spec, k, d, spread)


def test_batch_with_extrapolated_warm_start(ctx):
    """Cases with the extrapolated Poisson warm start in a batch: their first step after
    set_state (no previous pressure) runs eagerly before the concurrent replays, the later ones
    from their graphs; every case equals the same case stepped alone, bit for bit."""
    from paper_2507_05222_gb300 import qtt
    mix = [MIX[0], MIX[3]]
    opsl = [Q.Ops(ne, nx, R, Re, dt, o, rot=rot) for (o, ne, nx, chi, Re, dt, rot) in mix]
    states = [start_state(s[1], s[2], s[3], 40 + i, ops) for i, (s, ops) in enumerate(zip(mix, opsl))]

    def make(spec, st, warm):
        ordering, ne, nx, chi, Re, dt, rot = spec
        case = qtt.Case(ctx, ne, nx, R, Re, dt, chi, ordering, rot=rot, mom=TIGHT_MOM, poi=TIGHT_POI,
                        poisson_warm=warm)
        case.set_state(*[qtt.MPS.from_cores(ctx, x) for x in st])
        return case

    alone = []
    for spec, st in zip(mix, states):
        case = make(spec, st, "extrapolated")
        case.fractional_step(3)
        alone.append([qtt.qtt_decode(ctx, g) for g in case.get_state()])
    cases = [make(mix[0], states[0], "extrapolated"), make(mix[1], states[1], "extrapolated")]
    recs, status = qtt.fractional_step_batch(ctx, cases, 3)
    assert status == [0, 0]
    for i, case in enumerate(cases):
        for a, b in zip((qtt.qtt_decode(ctx, g) for g in case.get_state()), alone[i]):
            assert np.array_equal(a, b), i
    # a second batch call continues from the graphs (the history is kept)
    recs2, status2 = qtt.fractional_step_batch(ctx, cases, 1)
    assert status2 == [0, 0]
