"""The dense Householder QR behind every gauge move of the fit and ALS sweeps (Sec. II.A.4),
one-CTA and cluster kernels, against LAPACK (numpy.linalg.qr uses the same reflector sign
convention, so Q and R agree entry by entry for well-conditioned input) and, for ill-
conditioned or rank-deficient input, against the defining properties A = QR, Q^T Q = I and
R upper triangular."""
import numpy as np
import pytest

from paper_2507_05222_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(128, 64), (130, 37), (64, 64), (256, 128), (40, 17), (16, 16), (200, 20), (96, 33), (12, 5), (5, 12)]


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2507_05222_gb300 import qtt
    return qtt.Context(0)


def cluster_ok(m, n):
    # the cluster kernel takes m >= n >= 16
    return m >= n >= 16


def one_cta_ok(m, n):
    # the one-CTA kernel keeps the whole matrix in shared memory (at most 220 KiB)
    return (m * n + m + min(m, n) + 32) * 8 <= 220 * 1024


def run(ctx, A, trans, path):
    from paper_2507_05222_gb300 import qtt
    if trans:
        Qt, R = qtt.qtt_qr(ctx, A.T.copy(), trans=True, path=path)
        return Qt.T, R
    return qtt.qtt_qr(ctx, A, trans=False, path=path)


def check_properties(A, Q, R, tol):
    kk = min(A.shape)
    scale = np.abs(A).max()
    assert np.abs(Q @ R - A).max() <= tol * scale
    assert np.abs(Q.T @ Q - np.eye(kk)).max() <= tol
    assert np.abs(np.tril(R, -1)).max() == 0.0


@pytest.mark.parametrize("m,n", SHAPES)
@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("path", [0, 1, 2])
def test_qr_matches_lapack(ctx, m, n, trans, path):
    if path == 2 and not cluster_ok(m, n):
        pytest.skip("cluster kernel needs m >= n >= 16")
    if path == 1 and not one_cta_ok(m, n):
        pytest.skip("matrix does not fit one CTA")
    g = inputs.rng(1000 * m + n)
    A = g.standard_normal((m, n))
    Q, R = run(ctx, A, trans, path)
    Qn, Rn = np.linalg.qr(A)
    # random Gaussian blocks are well conditioned (cond < 1e3 here): Q and R are determined to
    # ~cond * eps_64 relative accuracy
    assert np.abs(Q - Qn).max() <= 1e-12
    assert np.abs(R - Rn).max() <= 1e-12 * np.abs(A).max()
    check_properties(A, Q, R, 1e-13)


@pytest.mark.parametrize("m,n", [(128, 64), (256, 128), (64, 64)])
@pytest.mark.parametrize("trans", [False, True])
def test_qr_ill_conditioned_and_rank_deficient(ctx, m, n, trans):
    g = inputs.rng(7 * m + n)
    U, _ = np.linalg.qr(g.standard_normal((m, n)))
    V, _ = np.linalg.qr(g.standard_normal((n, n)))
    graded = (U * 10.0 ** (-np.linspace(0, 14, n))) @ V.T
    lowrank = g.standard_normal((m, n // 4)) @ g.standard_normal((n // 4, n))
    zero_cols = g.standard_normal((m, n))
    zero_cols[:, ::3] = 0.0
    for A in (graded, lowrank, zero_cols, np.zeros((m, n))):
        Qc, Rc = run(ctx, A, trans, 2)
        check_properties(A, Qc, Rc, 1e-13)
        if one_cta_ok(m, n):
            Q1, R1 = run(ctx, A, trans, 1)
            check_properties(A, Q1, R1, 1e-13)
        if not A.any():
            # sigma = 0 at every step: every reflector is the identity
            assert np.array_equal(Qc, np.eye(m, n)) and not Rc.any()


def test_qr_cluster_rejects_wide(ctx):
    from paper_2507_05222_gb300 import qtt
    with pytest.raises(qtt.QttError):
        qtt.qtt_qr(ctx, np.ones((8, 32)), path=2)


def test_householder_scalar_reciprocals(ctx):
    """The QR's Householder scalars use Newton-Raphson reciprocal and reciprocal square root
    instead of FP64 division and square root: within ~2 ulp of CUDA's correctly rounded 1/x and
    1/sqrt(x) over the whole normal range and near 1 (where column norms live)."""
    from paper_2507_05222_gb300 import qtt
    g = inputs.rng(4242)
    x = np.concatenate([10.0 ** g.uniform(-300, 300, 20000), g.uniform(0.5, 2.0, 20000),
                        1.0 + g.uniform(-1e-12, 1e-12, 1000), [1.0, 2.0, 4.0, 0.25, 1e-300, 1e300]])
    e_rcp, e_rsqrt = qtt.qtt_check_recip(ctx, x)
    assert e_rcp <= 4.5e-16 and e_rsqrt <= 4.5e-16
