"""The C-ABI library loads and exports every function include/qtt.h declares (CPU only: no
device call is made), and the host-only entry points behave."""
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    from paper_2507_05222_gb300 import build, qtt
    build.build()
    return qtt


def test_exports_every_declared_symbol(lib):
    names = lib.header_functions()
    assert len(names) >= 30
    h = lib.lib()
    assert [n for n in names if not hasattr(h, n)] == []
    assert set(names) == set(lib._SIGS)


def test_entry_points_named_after_the_method(lib):
    for n in ("qtt_encode", "mpo_apply_round", "mps_hadamard_round", "mps_axpby_round", "poisson_solve",
              "fractional_step"):
        assert n in lib.header_functions()


def test_null_handles_are_rejected_on_host(lib):
    h = lib.lib()
    assert h.qtt_mps_n(None) == 0
    assert h.qtt_mps_size(None) == 0
    assert h.qtt_mps_free(None) == 0
    rc = h.qtt_mps_bonds(None, None)
    assert rc == -1 and b"null" in h.qtt_last_error()


def test_strouhal_host_entry_point(lib):
    from oracle import fd
    t = np.arange(0, 60, 0.01)
    cl = 0.2 + 0.7 * np.sin(2 * np.pi * 0.1663 * t)
    st = lib.qtt_strouhal(t, cl)
    assert abs(st - 0.1663) < 1e-4
    assert abs(st - fd.strouhal(t, cl)) < 1e-4


def test_missing_library_fails_loudly(lib, monkeypatch, tmp_path):
    monkeypatch.setattr(lib, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(lib, "_lib", None)
    with pytest.raises(RuntimeError):
        lib.lib()
