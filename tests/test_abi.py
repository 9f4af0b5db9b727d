"""CPU-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point declared in include/*.h; create fails cleanly
(status, not a crash) when there is no device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"LOBPCG_API[^;(]*?\b(lobpcg_\w+)\s*\(", src, flags=re.S))
    return names


def test_library_exports_every_declared_symbol():
    import paper_2109_00485_gb300 as pkg
    from paper_2109_00485_gb300 import _build
    _build.build()
    lib = ctypes.CDLL(_build.SO)
    names = declared_symbols()
    assert "lobpcg_spmm_sym" in names and "lobpcg_create" in names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    pkg.load()


def test_binding_has_every_entry_point():
    import paper_2109_00485_gb300 as pkg
    for n in declared_symbols():
        assert hasattr(pkg.Handle, n) or hasattr(pkg, n), f"binding lacks {n}"


def test_create_argument_errors_without_gpu():
    import numpy as np
    import paper_2109_00485_gb300 as pkg
    import synth
    A = synth.tile_matrix(100, 20, seed=1)
    with pytest.raises(pkg.LobpcgError) as ei:
        pkg.from_csr(A, k=0)          # rejected before any device call
    assert ei.value.status == 1
    with pytest.raises(pkg.LobpcgError) as ei:
        pkg.from_csr(A, k=4, nev=5)
    assert ei.value.status == 1
