"""The small symmetric eigensolver (FP32 Jacobi + FP64 refinement) against numpy on the
spectra the Gram roundings meet: one dominant value over a flat tail, exact zeros from
rank-deficient Gram matrices, clusters, and wide geometric decay; orders up to 160 (padded
shared-memory rows) and above (packed upper triangle, up to 256)."""
import numpy as np
import pytest

from paper_2507_05222_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2507_05222_gb300 import qtt
    return qtt.Context(0)


def spectrum(kind, n, g):
    if kind == "dominant_flat_tail":
        lam = np.concatenate([[256.0], 1.6e-5 * (1 + 0.3 * g.random(n - 1))])
    elif kind == "zeros":
        lam = np.concatenate([np.sort(g.random(n // 4))[::-1] * 10, 1.6e-5 * g.random(n // 4), np.zeros(n - 2 * (n // 4))])
    elif kind == "geometric":
        lam = 10.0 ** (-np.linspace(0, 15, n))
    elif kind.startswith("geometric"):
        # log-evenly spaced over a few decades: neighbours ~7-20 % apart at every scale, so
        # every refinement level has pairs just above its threshold with small absolute gaps
        lam = 10.0 ** (-np.linspace(0, int(kind[len("geometric"):]), n))
    elif kind == "cluster":
        lam = np.concatenate([np.ones(n // 2), 1 + 1e-9 * g.random(n // 4), 0.5 * np.ones(n - n // 2 - n // 4)])
    else:
        lam = g.standard_normal(n)
    return lam


@pytest.mark.parametrize("kind", ["dominant_flat_tail", "zeros", "geometric", "geometric4", "geometric8",
                                  "geometric12", "cluster", "random"])
@pytest.mark.parametrize("n", [16, 64, 128, 161, 256])
def test_sym_eig(ctx, kind, n):
    from paper_2507_05222_gb300 import qtt
    g = inputs.rng(n + len(kind))
    Qm, _ = np.linalg.qr(g.standard_normal((n, n)))
    lam = spectrum(kind, n, g)
    S = (Qm * lam) @ Qm.T
    S = 0.5 * (S + S.T)
    w, V = qtt.qtt_sym_eig(ctx, S)
    wr, Vr = np.linalg.eigh(S)
    wr, Vr = wr[::-1], Vr[:, ::-1]
    scale = np.abs(wr).max()
    # bounds from the arithmetic: FP64 products of length n accumulate ~n eps ||S||
    if kind == "cluster":
        sep = np.abs(wr - 1.0) > 1e-6               # outside the 1e-9-wide cluster at 1
        assert np.abs(w - wr)[sep].max() <= 1e-12 * scale
        assert abs(w[~sep].mean() - wr[~sep].mean()) <= 1e-12 * scale
    else:
        assert np.abs(w - wr).max() <= 1e-12 * scale
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-12
    if kind == "cluster":
        # eigenvectors inside a cluster of width 1e-9 are not individually determined; the
        # invariant subspace of the separated group (the quantity a truncation uses) is
        k = n // 2 + n // 4
        P, Pr = V[:, :k] @ V[:, :k].T, Vr[:, :k] @ Vr[:, :k].T
        assert np.abs(P - Pr).max() < 1e-12
    else:
        assert np.abs(S @ V - V * w).max() <= 1e-11 * scale


@pytest.mark.parametrize("kind", ["zeros", "dominant_flat_tail", "geometric", "geometric8"])
def test_sym_eig_many_seeds(ctx, kind):
    """Multi-level spectra (a dominant group, a group ~1e-6 below it, an exact null space) over
    many seeds: every level's refinement must leave X orthonormal whatever rounding the FP32
    start carries, so orthogonality, eigenvalues and residuals hold for each seed."""
    from paper_2507_05222_gb300 import qtt
    n = 128
    for seed in range(16):
        g = inputs.rng(5000 + 17 * seed + len(kind))
        Qm, _ = np.linalg.qr(g.standard_normal((n, n)))
        lam = spectrum(kind, n, g)
        S = (Qm * lam) @ Qm.T
        S = 0.5 * (S + S.T)
        w, V = qtt.qtt_sym_eig(ctx, S)
        wr = np.linalg.eigvalsh(S)[::-1]
        scale = np.abs(wr).max()
        assert np.abs(V.T @ V - np.eye(n)).max() < 1e-12, seed
        assert np.abs(w - wr).max() <= 1e-12 * scale, seed
        assert np.abs(S @ V - V * w).max() <= 1e-11 * scale, seed


@pytest.mark.parametrize("scale", [1e-200, 1e-100, 1e-40, 1e40, 1e150])
def test_sym_eig_extreme_scales(ctx, scale):
    """The solver works on S 2^-e (largest entry in [1, 2)): a matrix of any magnitude has the
    eigenvectors and the scaled eigenvalues of its unit-scale version.  Without the scaling a
    Gram matrix of a train with norm ~1e-96 (entries ~1e-192) vanished in the FP32 stage and the
    refinement diverged."""
    from paper_2507_05222_gb300 import qtt
    n = 64
    g = inputs.rng(77)
    Qm, _ = np.linalg.qr(g.standard_normal((n, n)))
    lam = spectrum("geometric8", n, g)
    S1 = (Qm * lam) @ Qm.T
    S1 = 0.5 * (S1 + S1.T)
    w1, V1 = qtt.qtt_sym_eig(ctx, S1)
    w, V = qtt.qtt_sym_eig(ctx, S1 * scale)
    assert np.all(np.isfinite(w)) and np.all(np.isfinite(V))
    assert np.abs(w / scale - w1).max() <= 1e-12 * np.abs(w1).max()
    assert np.abs(np.abs(V.T @ V1) - np.eye(n)).max() < 1e-6   # same eigenvectors up to sign


def test_sym_eig_zero_matrix(ctx):
    from paper_2507_05222_gb300 import qtt
    w, V = qtt.qtt_sym_eig(ctx, np.zeros((16, 16)))
    assert np.all(w == 0.0)
    assert np.abs(V.T @ V - np.eye(16)).max() < 1e-12
