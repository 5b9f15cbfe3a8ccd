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


def test_binding_structs_match_the_header_layout(lib, tmp_path):
    """Every struct the binding passes by value or pointer has the header's field names, offsets
    and size: a C program compiled against include/qtt.h prints sizeof and offsetof of each field
    the ctypes mirror names (a name the header lacks fails to compile; a field the binding lacks
    changes the size)."""
    import ctypes
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = [lib.qtt_trunc, lib.qtt_round_info, lib.qtt_solve_opts, lib.qtt_solve_info, lib.qtt_case_params,
               lib.qtt_step_info]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "qtt.h"', "int main(void) {"]
    expect = []
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("%zu\\n", sizeof({name}));')
        expect.append(ctypes.sizeof(st))
        for fname, _ in st._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({name}, {fname}));')
            expect.append(getattr(st, fname).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect
    # and the same member names in the same order (padding can hide a missing trailing field)
    import re
    header = open(os.path.join(root, "include", "qtt.h")).read()
    header = re.sub(r"/\*.*?\*/", "", header, flags=re.S)
    for st in structs:
        m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + st.__name__ + r"\s*;", header)
        assert m, st.__name__
        names = []
        for decl in m.group(1).split(";"):
            decl = decl.strip()
            if not decl:
                continue
            ty_and_first, *rest = [x.strip() for x in decl.split(",")]
            names.append(ty_and_first.split()[-1].lstrip("*"))
            names += [x.lstrip("*") for x in rest]
        assert names == [f for f, _ in st._fields_], st.__name__
