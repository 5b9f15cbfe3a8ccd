"""Reduced contraction precision (digit-split products keeping 3, 2 or 1 leading 8-bit digits
of each operand, exact accumulation), against FP64 definitions and the FP64 oracle.

Error model of one product C = A B with P digits: each operand entry is rounded to nearest at
8P bits relative to 2^e, where 2^e <= 4 max|row| (the row's or column's scale exponent), so its
error is at most 2^(e - 8P - 1) <= 2^(1 - 8P) max|row|; the dropped digit pairs (s + u > P + 1)
weigh at most as much again, so |C - A B|_ij <= 4 K 2^(1 - 8P) max|A_i:| max|B_:j|."""
import numpy as np
import pytest

from oracle import tt, qtt_ops as Q, step as S
from paper_2507_05222_gb300 import inputs

pytestmark = pytest.mark.gpu
DIGITS = {"fp32": 3, "tf32": 2, "bf16": 1}


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


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("m,n,k", [(64, 48, 32), (300, 70, 129), (17, 130, 1000)])
def test_reduced_product_error_bound(ctx, prec, m, n, k):
    from paper_2507_05222_gb300 import qtt
    g = inputs.rng(m + n + k)
    # rows and columns with a spread of magnitudes (the bound is relative to each row's max)
    A = g.standard_normal((m, k)) * np.exp2(g.integers(-20, 20, (m, 1)))
    B = g.standard_normal((k, n)) * np.exp2(g.integers(-20, 20, (1, n)))
    c2 = qtt.Context(0)
    c2.set_precision(prec)
    C = qtt.qtt_dgemm(c2, A, B, path=0)
    P = DIGITS[prec]
    bound = 4 * k * 2.0 ** (1 - 8 * P) * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :]
    err = np.abs(C - A @ B)
    assert (err <= bound).all(), float((err / bound).max())
    # and not FP64: the truncation is real (guards against the FP64 path being taken silently)
    assert np.abs(C - A @ B).max() > 0.0
    c2.set_precision("fp64")
    C64 = qtt.qtt_dgemm(c2, A, B, path=0)
    assert np.abs(C64 - A @ B).max() <= 1e-13 * (np.abs(A) @ np.abs(B)).max()


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_reduced_apply_and_fit_errors(ctx, prec):
    """MPO-MPS product with rounding and the Hadamard fit at reduced precision, against the
    FP64 oracle on a smooth 12-bit state.  The product's rounding works on Gram matrices of the
    environments, whose entries carry the contractions' relative error 2^-8P of the largest
    squared singular value; the eigenvectors of singular values below 2^-4P sigma_1 are then
    not resolved, which leaves an error of that size in the rounded product: bound 16 x
    2^-4P (measured ~7 x 2^-4P).  The fit's contractions at chi = 16 are small enough to run on
    the FP64 direct path, so its error stays at FP64 level."""
    from paper_2507_05222_gb300 import qtt
    ne = nx = 6
    ops = Q.Ops(ne, nx, 40.0, 200.0, 8e-4, "interleaved")
    f = inputs.wake_field(ne, nx, 3)
    u, v = ops.encode(f[0], 16), ops.encode(f[1], 16)
    gu, gv = qtt.MPS.from_cores(ctx, u), qtt.MPS.from_cores(ctx, v)
    P = DIGITS[prec]
    bound = 16.0 * 2.0 ** (-4 * P)
    ref = tt.full(tt.round_tt(tt.mpo_mps(ops.Dx, u), 16))
    y = qtt.mpo_apply_round(ctx, qtt.MPO.from_cores(ctx, ops.Dx), gu, 16, prec=prec)
    e1 = rel(qtt.qtt_decode(ctx, y), ref)
    ref = tt.full(tt.hadamard_round(u, v, 16, sweeps=2))
    h = qtt.mps_hadamard_round(ctx, gu, gv, 16, sweeps=2, prec=prec)
    e2 = rel(qtt.qtt_decode(ctx, h), ref)
    print(f"{prec}: apply error {e1:.2e}, Hadamard fit error {e2:.2e}, bound {bound:.1e}")
    assert e1 <= bound and e2 <= bound
    assert e1 > 2.0 ** (-8 * P - 8)      # the reduced path was taken


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_reduced_precision_step_against_fp64_oracle(ctx, prec):
    """One fractional step (12 bits, chi 16) with reduced-precision contractions against the
    FP64 oracle's step: every field within 2^(10 - 8P).  The momentum solve's environments
    carry the contractions' error 2^-8P and its operator |J| (I - dt/Re Lap) has a condition
    number of ~1e3 on this grid, so the solved field may move by up to ~2^10 times that; the
    Poisson solve and the divergence stay FP64.  (Measured: fp32 4e-6 / 2.5e-5 / 2.3e-6 in
    u / v / p, tf32 1e-4 / 7e-4 / 1.6e-4.)"""
    from paper_2507_05222_gb300 import qtt
    ne = nx = 6
    R, Re, dt, chi = 40.0, 100.0, 2e-3, 16
    ops = Q.Ops(ne, nx, R, Re, dt, "interleaved")
    f = inputs.wake_field(ne, nx, 5)
    u, v = ops.encode(f[0], chi), ops.encode(f[1], chi)
    p = S.padded([np.zeros((1, 2, 1))] * (ne + nx), chi, inputs.random_cores(ne + nx, chi, 7, scale=1e-8))
    c2 = qtt.Context(0)
    c2.set_precision(prec)
    mom, poi = (6, 1e-8, 300, 1e-6, 0.1), (12, 1e-10, 600, 1e-6, 0.1)
    case = qtt.Case(c2, ne, nx, R, Re, dt, chi, "interleaved", mom=mom, poi=poi)
    case.set_state(*(qtt.MPS.from_cores(c2, x) for x in (u, v, p)))
    info = case.fractional_step(1, check=False)
    un, vn, pn, oi = S.step(ops, u, v, p, S.StepOpts(chi=chi, fit_sweeps=1, mom=S.SolveOpts(*mom),
                                                        poi=S.SolveOpts(*poi)))
    bound = 2.0 ** (10 - 8 * DIGITS[prec])
    errs = [rel(qtt.qtt_decode(c2, g), tt.full(r)) for g, r in zip(case.get_state(), (un, vn, pn))]
    print(prec, "step errors u, v, p:", ["%.2e" % e for e in errs])
    assert max(errs) <= bound, errs
    assert info[0]["finite"] == 1
