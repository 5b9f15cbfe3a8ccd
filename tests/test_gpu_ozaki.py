"""FP64 products on the tensor cores by digit splitting (qtt_ozaki.cu).  Checked against an
extended-precision product, where the scheme must meet its own bound 2^-52 max_k|A_ik| sum_k|B_kj|
(dropped digit products and splitting remainders), and against NumPy's FP64 product within the
plain FP64 bound gamma_k |A||B| (NumPy's own rounding included): tile-ragged shapes, k beyond one
exact chunk (split k), rows and columns spanning many orders of magnitude, zero rows, and the
context's dispatch of large products."""
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


def bound(A, B):
    """The digit-split scheme's own error bound (dropped digit products and remainders)."""
    return 2.0 ** -52 * np.abs(A).max(axis=1, keepdims=True) * np.abs(B).sum(axis=0, keepdims=True)


def fp64_bound(A, B):
    """gamma_k |A||B|: how far a plain FP64 product (NumPy's reference included) may be off."""
    k = A.shape[1]
    return (k + 4) * 2.0 ** -53 * (np.abs(A) @ np.abs(B))


def exact(A, B):
    """The product in extended precision (x86 80-bit or aarch64 128-bit long double)."""
    return A.astype(np.longdouble) @ B.astype(np.longdouble)


@pytest.mark.parametrize("m,n,k", [(64, 32, 16), (130, 70, 64), (256, 128, 384), (1000, 48, 200), (17, 33, 17),
                                   (4096, 128, 64), (128, 64, 4096),
                                   # FP64 path: direct small contractions with 1, 8 and 32 lanes per
                                   # output, and split-K tiles finished by the last CTA of each tile
                                   (40, 30, 5), (16, 16, 1024), (3, 1000, 60), (16, 16, 4100), (33, 65, 2000)])
def test_ozaki_matches_fp64(ctx, m, n, k):
    from paper_2507_05222_gb300 import qtt
    g = inputs.rng(m * 7 + n * 3 + k)
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, n))
    C = qtt.qtt_dgemm(ctx, A, B, path=2)
    ref = A @ B
    assert np.all(np.abs(C - ref) <= fp64_bound(A, B) + 4 * bound(A, B))
    # the FP64 pipe path agrees too
    C1 = qtt.qtt_dgemm(ctx, A, B, path=1)
    assert np.all(np.abs(C1 - ref) <= 2 * fp64_bound(A, B))
    if m * n * k <= 2 ** 22:
        # against the extended-precision product the scheme meets its own (tighter) bound
        err = np.abs(C.astype(np.longdouble) - exact(A, B)).astype(np.float64)
        assert np.all(err <= 4 * bound(A, B))


def test_ozaki_graded_and_zero_rows(ctx):
    from paper_2507_05222_gb300 import qtt
    g = inputs.rng(99)
    m, n, k = 96, 40, 150
    A = g.standard_normal((m, k)) * 10.0 ** g.uniform(-12, 12, (m, 1))     # rows on different scales
    A[5] = 0.0
    A[7, :] = 0.0
    A[7, 3] = 1e-300
    B = g.standard_normal((k, n)) * 10.0 ** g.uniform(-6, 6, (1, n))       # columns on different scales
    C = qtt.qtt_dgemm(ctx, A, B, path=2)
    err = np.abs(C.astype(np.longdouble) - exact(A, B)).astype(np.float64)
    assert np.all(err <= 4 * bound(A, B) + 1e-300)
    assert not C[5].any()


def test_dispatch_of_large_products(ctx):
    """In mode 0 products of at least 2^23 multiply-adds take the tensor-core path, in mode 1
    the FP64 pipe; both agree with NumPy within the bounds."""
    from paper_2507_05222_gb300 import qtt
    g = inputs.rng(5)
    A = g.standard_normal((1024, 128))
    B = g.standard_normal((128, 256))
    ref = A @ B
    for mode in (0, 1):
        ctx.set_gemm_mode(mode)
        try:
            C = qtt.qtt_dgemm(ctx, A, B, path=0)
        finally:
            ctx.set_gemm_mode(0)
        assert np.all(np.abs(C - ref) <= 2 * fp64_bound(A, B) + 4 * bound(A, B))


@pytest.mark.parametrize("m,n,k", [(128, 32, 64), (130, 70, 64), (256, 128, 384), (1000, 48, 200), (17, 33, 17),
                                   (300, 31, 1000), (64, 4096, 128), (4096, 128, 64), (129, 257, 4100)])
def test_tcgen05_digit_products_equal_mma_sync(ctx, m, n, k):
    """The digit products on the fifth-generation tensor cores (tcgen05.mma on TMA-staged 128-byte
    swizzled tiles, seven tensor-memory accumulators, path 3) add the same exact integers as the
    warp-level mma.sync kernel (path 2): the results are bit-identical, on tile-ragged shapes, k
    spanning several 64-wide chunks and split k, and they meet the scheme's own bound."""
    from paper_2507_05222_gb300 import qtt
    g = inputs.rng(m * 7 + n * 3 + k)
    A = g.standard_normal((m, k)) * np.exp(g.uniform(-8, 8, (m, 1)))
    B = g.standard_normal((k, n)) * np.exp(g.uniform(-8, 8, (1, n)))
    c2 = qtt.qtt_dgemm(ctx, A, B, path=2)
    c3 = qtt.qtt_dgemm(ctx, A, B, path=3)
    assert np.array_equal(c2, c3)
    err = np.abs(c3 - exact(A, B)).astype(np.float64)
    assert np.all(err <= bound(A, B))


def test_tcgen05_step_equals_mma_sync_step(ctx):
    """A whole step at chi = 64 (12 bits) with every large product on the tcgen05 kernel equals the
    step with the mma.sync kernel bit for bit (same exact group sums, same kernels otherwise)."""
    from oracle import qtt_ops as Q, step as S
    from paper_2507_05222_gb300 import qtt
    ne = nx = 6
    chi = 64
    ops = Q.Ops(ne, nx, 40.0, 100.0, 2e-3, "interleaved")
    u0, v0 = inputs.wake_field(ne, nx, 3)
    u, v = ops.encode(u0, chi), ops.encode(v0, chi)
    p = S.padded([np.zeros((1, 2, 1))] * (ne + nx), chi, inputs.random_cores(ne + nx, chi, 5, scale=1e-8))
    out = []
    try:
        for mode in (2, 3):
            ctx.set_gemm_mode(mode)
            case = qtt.Case(ctx, ne, nx, 40.0, 100.0, 2e-3, chi, "interleaved")
            case.set_state(*(qtt.MPS.from_cores(ctx, x) for x in (u, v, p)))
            info = case.fractional_step(2, check=False)
            out.append(([qtt.qtt_decode(ctx, x) for x in case.get_state()], info))
    finally:
        ctx.set_gemm_mode(0)
    (a, ia), (b, ib) = out
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert [r["p"]["sweeps"] for r in ia] == [r["p"]["sweeps"] for r in ib]
