"""mps_dot_noalloc: the overlap entry point for callers that cannot allocate device memory
(inside another allocator's callback, allocation-free loops, fully reserved device memory).
It is checked through the C ABI against the existing mps_dot on two calls in a row, which
also shows that the shared fixed scratch array carries nothing over from one call to the
next.  This file is collected last on purpose."""
import numpy as np
import pytest

from oracle import tt
from paper_2507_05222_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dev(torch, cores):
    flat = np.concatenate([c.ravel() for c in cores])
    return torch.from_numpy(flat).cuda()


def test_noalloc_dot_matches_mps_dot_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2507_05222_gb300 import qtt
    ctx = qtt.Context(0)
    stream = torch.cuda.current_stream().cuda_stream
    full = [1, 4, 16, 64, 128, 128, 128, 128, 64, 16, 4, 1]     # d = 4, bonds at the 128 limit
    cases = [(inputs.random_cores(12, 24, seed=101), inputs.random_cores(12, 17, seed=102)),
             (inputs.random_cores(12, 9, seed=103), inputs.random_cores(12, 128, seed=104, scale=0.1)),
             (inputs.random_cores(11, 128, seed=105, d=4, bonds=full, scale=0.1),
              inputs.random_cores(11, 128, seed=106, d=4, bonds=full, scale=0.1))]
    out = torch.zeros(len(cases), dtype=torch.float64, device="cuda")
    keep = []
    for i, (a, b) in enumerate(cases):
        da, db = _dev(torch, a), _dev(torch, b)
        keep += [da, db]
        ab = [a[0].shape[0]] + [c.shape[2] for c in a]
        bb = [b[0].shape[0]] + [c.shape[2] for c in b]
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        n, d = len(a), a[0].shape[1]
        qtt.mps_dot_noalloc(n, d, ab, da.data_ptr(), bb, db.data_ptr(), out.data_ptr() + 8 * i, stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before
        ref = qtt.mps_dot(ctx, qtt.MPS.from_cores(ctx, a), qtt.MPS.from_cores(ctx, b))
        got = float(out[i].item())
        na = np.sqrt(qtt.mps_dot(ctx, qtt.MPS.from_cores(ctx, a), qtt.MPS.from_cores(ctx, a)))
        nb = np.sqrt(qtt.mps_dot(ctx, qtt.MPS.from_cores(ctx, b), qtt.MPS.from_cores(ctx, b)))
        assert abs(got - ref) <= 1e-12 * na * nb
        assert abs(got - tt.dot(a, b)) <= 1e-12 * na * nb      # the FP64 oracle's overlap


def test_noalloc_rejects_bond_above_limit():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2507_05222_gb300 import qtt
    a = inputs.random_cores(16, 129, seed=5)
    da = _dev(torch, a)
    ab = [1] + [c.shape[2] for c in a]
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(qtt.QttError) as e:
        qtt.mps_dot_noalloc(16, 2, ab, da.data_ptr(), ab, da.data_ptr(), out.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    assert e.value.code == -7 and "128" in str(e.value)
