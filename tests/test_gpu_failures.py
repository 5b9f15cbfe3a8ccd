"""Failure detection through the C ABI (include/qtt.h error codes), made on the host or by a
bounded device wait that runs out -- nothing here faults, traps or hangs the GPU:

* a grid barrier of the cooperative CG solve whose wait limit is shortened to 1 ns runs out:
  the kernel leaves at once, the solve reports QTT_SOLVE_TIMEOUT and the call returns
  QTT_ERR_TIMEOUT (poisson_solve and fractional_step, the latter also without per-step records);
  the context stays usable;
* a NaN in a host input core gives QTT_ERR_NONFINITE from the step (its residual is NaN);
* an allocator hook that returns NULL gives QTT_ERR_ALLOC;
* a solve that runs out of sweeps returns QTT_ERR_NOT_CONVERGED with the last iterate (also in
  tests/test_gpu_ops.py::test_poisson_solve_statuses)."""
import numpy as np
import pytest

from oracle import tt, qtt_ops as Q, step as S
from paper_2507_05222_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qtt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2507_05222_gb300 import qtt as q
    return q


def small_case(qtt, ctx, chi=8, ne=4):
    ops = Q.Ops(ne, ne, 40.0, 100.0, 2e-3, "interleaved")
    u0 = 1.0 + inputs.gaussian_field(ne, ne, 1, 1e-3)
    v0 = inputs.gaussian_field(ne, ne, 2, 1e-3)
    u, v = ops.encode(u0, chi), ops.encode(v0, chi)
    p = S.padded([np.zeros((1, 2, 1))] * (2 * ne), chi, inputs.random_cores(2 * ne, chi, 3, scale=1e-8))
    case = qtt.Case(ctx, ne, ne, 40.0, 100.0, 2e-3, chi, "interleaved")
    return ops, case, (u, v, p)


def test_barrier_timeout_returns_timeout_and_context_survives(qtt):
    ctx = qtt.Context(0)
    ne = 4
    ops = Q.Ops(ne, ne, 40.0, 100.0, 2e-3, "interleaved")
    A = qtt.MPO.from_cores(ctx, ops.Ap)
    b = inputs.random_cores(2 * ne, 4, seed=80)
    x0 = inputs.random_cores(2 * ne, 8, seed=81, scale=0.1)
    ctx.set_cg_mode(2)                      # the cooperative FP64 CG kernel at every site
    ctx.set_wait_limit(1e-9)
    g = qtt.MPS.from_cores(ctx, x0)
    with pytest.raises(qtt.QttError) as e:
        qtt.poisson_solve(ctx, A, qtt.MPS.from_cores(ctx, b), g, 4, 1e-10, 100)
    assert e.value.code == -5 and "timed out" in str(e.value)
    ctx.set_wait_limit(2.0)
    g = qtt.MPS.from_cores(ctx, x0)
    info = qtt.poisson_solve(ctx, A, qtt.MPS.from_cores(ctx, b), g, 4, 1e-10, 100)
    ref, ir = tt.als(ops.Ap, [("vec", 1.0, b)], x0, 4, 100, 1e-2, 1e-10, 0.1)
    assert info["sweeps"] == ir["sweeps"] and info["status"] == ir["status"]
    assert np.linalg.norm(qtt.qtt_decode(ctx, g) - tt.full(ref)) <= 1e-10 * np.linalg.norm(tt.full(ref))
    # the step: with and without per-step records, captured graph and eager
    for graph in (True, False):
        ops, case, state = small_case(qtt, ctx)
        case.use_graph(graph)
        case.set_state(*(qtt.MPS.from_cores(ctx, x) for x in state))
        ctx.set_wait_limit(1e-9)
        case.use_graph(graph)               # re-capture with the short limit
        with pytest.raises(qtt.QttError) as e:
            qtt.fractional_step(ctx, case, 1, info=False)
        assert e.value.code == -5
        with pytest.raises(qtt.QttError) as e:
            case.fractional_step(1)
        assert e.value.code == -5 and any(r[k]["status"] == 4 for r in e.value.records for k in "uvp")
        ctx.set_wait_limit(2.0)
        case.use_graph(graph)
        case.set_state(*(qtt.MPS.from_cores(ctx, x) for x in state))
        info = case.fractional_step(1)
        assert info[0]["rc"] == 0 and info[0]["finite"] == 1
    ctx.set_cg_mode(0)


def test_nan_input_gives_nonfinite(qtt):
    ctx = qtt.Context(0)
    ops, case, (u, v, p) = small_case(qtt, ctx)
    bad = [c.copy() for c in u]
    bad[3][0, 1, 0] = np.nan
    case.set_state(*(qtt.MPS.from_cores(ctx, x) for x in (bad, v, p)))
    with pytest.raises(qtt.QttError) as e:
        case.fractional_step(1)
    assert e.value.code == -6
    r = e.value.records[0]
    assert r["finite"] == 0 or any(r[k]["status"] == 3 for k in "uvp")
    case.set_state(*(qtt.MPS.from_cores(ctx, x) for x in (u, v, p)))
    assert case.fractional_step(1)[0]["rc"] == 0


def test_allocation_failure_gives_alloc_error(qtt):
    import torch
    state = {"fail": False}

    def alloc(nbytes):
        if state["fail"]:
            return 0
        return torch.cuda.caching_allocator_alloc(nbytes, 0, torch.cuda.current_stream(0))

    def free(ptr):
        torch.cuda.caching_allocator_delete(ptr)

    ctx = qtt.Context(0, allocator=(alloc, free))
    x = inputs.random_cores(8, 4, seed=1)
    g = qtt.MPS.from_cores(ctx, x)                      # works while the hook allocates
    state["fail"] = True
    with pytest.raises(qtt.QttError) as e:           # 67 MB: more than the pool's first chunk holds
        qtt.MPS.from_cores(ctx, inputs.random_cores(3, 2048, seed=2, bonds=[1, 2048, 2048, 1]))
    assert e.value.code == -2
    state["fail"] = False
    ops, case, (u, v, p) = small_case(qtt, ctx)
    case.use_graph(False)
    case.set_state(*(qtt.MPS.from_cores(ctx, y) for y in (u, v, p)))
    state["fail"] = True
    try:
        with pytest.raises(qtt.QttError) as e:
            case.fractional_step(1)       # the step's worker pools take their first chunks here
        assert e.value.code == -2
    finally:
        state["fail"] = False
    ctx.sync()
    assert abs(qtt.mps_dot(ctx, g, g) - tt.dot(x, x)) <= 1e-12 * tt.dot(x, x)
