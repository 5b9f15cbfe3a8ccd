"""GPU parity of the sketched rounding of mpo_apply_round (QTT_APPLY_SKETCH) against the FP64
oracle's TT-SVD of the exact product (Sec. II.A.2, then the rounding of Sec. II.A), through the
C ABI, at relative 1e-10 on reconstructed vectors.

Two regimes are covered.  Exact: when the sketch is as wide as the product's largest bond
w_k a_k (the width used whenever the QR of the sketch supports it), or as the right space of
every cut, it spans every cut's range, so the result is the TT-SVD up to rounding for any input,
random tensor trains included.  Decaying spectra: the fields of the step at 2^16 cells and
chi = 64 (sketch width 2 chi + 32 = 160 < w a = 512), where the sketch's range error falls
below 1e-13 and the Gram rounding's squared singular values leave ~1e-8 (shown beside it)."""
import numpy as np
import pytest

from oracle import tt, qtt_ops as Q, step as S
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


def smooth_field(ne, nx, seed, amp, modes):
    """Products of a cosine in eta and a sine in xi with amplitudes 2^(-k/2), seeded phases."""
    g = inputs.rng(seed)
    i = (np.arange(2 ** ne) + 0.5) / 2 ** ne
    j = np.arange(2 ** nx) / 2 ** nx
    f = np.zeros((2 ** ne, 2 ** nx))
    for k in range(1, modes + 1):
        ph, ps = g.uniform(0, 2 * np.pi, 2)
        f += 2.0 ** (-k / 2) * np.outer(np.cos(np.pi * k * i + ps), np.sin(2 * np.pi * k * j + ph))
    return amp * f


def check_product(ctx, M, x, chi, tol=TOL, disc_floor=1e-13):
    from paper_2507_05222_gb300 import qtt
    info = {}
    ref = tt.round_tt(tt.mpo_mps(M, x), chi, 0.0, info)
    full = tt.full(ref)
    gi = {}
    g = qtt.mpo_apply_round(ctx, qtt.MPO.from_cores(ctx, M), qtt.MPS.from_cores(ctx, x), chi, out_info=gi,
                            apply="sketch")
    assert g.bonds() == tt.bonds(ref)
    err = rel(qtt.qtt_decode(ctx, g), full)
    assert err < tol
    nrm = np.linalg.norm(full)
    # the discarded weight is the sum of the discarded Rayleigh quotients, each formed from the
    # explicit factor: known to ~1e-4 of itself where the cut falls among the smallest resolved
    # eigenvalues (measured 1.4e-4 for a discarded norm of 7.5e-9 ||y||), and to the FP64 floor
    # in absolute terms (disc_floor ||y||)
    assert abs(gi["discarded_norm"] - info["discarded_norm"]) <= 1e-3 * info["discarded_norm"] + disc_floor * nrm
    return err


@pytest.mark.parametrize("n,bx,w,chi", [(6, 4, 3, 5), (9, 7, 5, 9), (10, 16, 4, 12), (10, 32, 9, 64),
                                        (12, 24, 3, 16), (12, 40, 6, 40), (16, 16, 8, 16), (15, 24, 5, 24)])
def test_sketch_exact_regime_random(ctx, n, bx, w, chi):
    """Random tensor trains and operators (flat spectra, truncation active at most cuts) where
    the sketch spans every cut's right space: equal to the TT-SVD at 1e-10, bonds and discarded
    norm included."""
    x = inputs.random_cores(n, bx, seed=70 + n + bx)
    M = inputs.random_mpo_cores(n, w, seed=80 + n + w)
    check_product(ctx, M, x, chi)


@pytest.mark.parametrize("ne,nx,ordering,kind", [(8, 8, "interleaved", "wake"), (9, 8, "sequential", "smooth"),
                                                 (3, 4, "interleaved", "wake")])
def test_sketch_fd_products_match_tt_svd(ctx, ne, nx, ordering, kind):
    """D_x, D_z and the weighted Poisson operator on the step's kind of fields at chi = 64 (the
    middle cuts compressed by the sketch), against the oracle's TT-SVD at 1e-10; the Gram rounding
    of the same products is printed for comparison."""
    from paper_2507_05222_gb300 import qtt
    ops = Q.Ops(ne, nx, 40.0, 200.0, 8e-4, ordering)
    if kind == "wake":
        u0, v0 = inputs.wake_field(ne, nx, 3)
    else:
        u0, v0 = 1.0 + smooth_field(ne, nx, 11, 1e-2, 24), smooth_field(ne, nx, 12, 1e-2, 24)
    for f0 in (u0, v0):
        f = ops.encode(f0, 64)
        for M in (ops.Dx, ops.Dz, ops.Ap):
            # products of derivative operators cancel (||D|| ||f|| >> ||D f||): the oracle's own
            # QR resolves the discarded singular values only to ~1e-12 ||y|| here
            err = check_product(ctx, M, f, 64, disc_floor=1e-12)
            ref = tt.full(tt.round_tt(tt.mpo_mps(M, f), 64))
            g = qtt.mpo_apply_round(ctx, qtt.MPO.from_cores(ctx, M), qtt.MPS.from_cores(ctx, f), 64)
            print(f"sketch {err:.1e}  gram {rel(qtt.qtt_decode(ctx, g), ref):.1e}")


def test_sketch_step_matches_oracle(ctx):
    """A truncated fractional step (2^8 cells, chi = 8, local solves converged far below the
    stop rule) whose four MPO-MPS products use the sketched rounding equals the oracle's step
    (TT-SVD products) at 1e-10, with the same sweeps and stop decisions."""
    from paper_2507_05222_gb300 import qtt
    ne = nx = 4
    R, Re, dt, chi = 40.0, 100.0, 2e-3, 8
    tight_mom = (6, 1e-10, 400, 1e-10, 0.1)
    tight_poi = (12, 1e-10, 600, 1e-10, 0.1)
    ops = Q.Ops(ne, nx, R, Re, dt, "interleaved")
    u0 = 1.0 + inputs.gaussian_field(ne, nx, 1, 1e-3)
    v0 = inputs.gaussian_field(ne, nx, 2, 1e-3)
    u, v = ops.encode(u0, chi), ops.encode(v0, chi)
    p = S.padded([np.zeros((1, 2, 1))] * (ne + nx), chi, inputs.random_cores(ne + nx, chi, 3, scale=1e-8))
    case = qtt.Case(ctx, ne, nx, R, Re, dt, chi, "interleaved", mom=tight_mom, poi=tight_poi, apply="sketch")
    case.set_state(*(qtt.MPS.from_cores(ctx, x) for x in (u, v, p)))
    info = case.fractional_step(1, with_forces=False, check=False)
    o = S.StepOpts(chi=chi, fit_sweeps=1, mom=S.SolveOpts(*tight_mom), poi=S.SolveOpts(*tight_poi))
    un, vn, pn, oi = S.step(ops, u, v, p, o)
    for k in "uvp":
        assert (info[0][k]["sweeps"], info[0][k]["status"]) == (oi[k]["sweeps"], oi[k]["status"])
    for g, r in zip(case.get_state(), (un, vn, pn)):
        assert rel(qtt.qtt_decode(ctx, g), tt.full(r)) < TOL


def test_sketch_rejects_wide_cuts(ctx):
    """d chi > 256 exceeds the eigensolver of the cut matrices: QTT_ERR_UNSUPPORTED, and the
    case rejects the sketched products above chi = 128."""
    from paper_2507_05222_gb300 import qtt
    x = inputs.random_cores(8, 4, seed=1)
    M = inputs.random_mpo_cores(8, 2, seed=2)
    with pytest.raises(qtt.QttError) as e:
        qtt.mpo_apply_round(ctx, qtt.MPO.from_cores(ctx, M), qtt.MPS.from_cores(ctx, x), 160, apply="sketch")
    assert e.value.code == -7
    with pytest.raises(qtt.QttError) as e:
        qtt.Case(ctx, 4, 4, 40.0, 100.0, 2e-3, 160, "interleaved", apply="sketch")
    assert e.value.code == -1
