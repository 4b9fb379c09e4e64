"""The C-ABI library builds, loads and exports every entry point include/dgk.h declares;
its host-only calls work without a GPU and its context calls fail cleanly (no crash)
when no GPU is present."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", hdr)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"\b(dgk_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    from paper_2208_05310_gb300 import build
    build.build()
    from paper_2208_05310_gb300 import dgk
    return dgk


def test_exports_every_declared_symbol(built):
    L = built.lib()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(built.EXPORTS) <= set(names)


def test_host_thermo_without_gpu(built, orc):
    rv, rl = built.maxwell(0.85)
    orv, orl = orc.maxwell(0.85)
    assert abs(rv - orv) < 1e-13 and abs(rl - orl) < 1e-13
    assert abs(built.sigma_vl(0.85) / orc.sigma_vl(0.85) - 1) < 1e-12
    with pytest.raises(built.DgkError):
        built.maxwell(1.2)


def test_status_strings(built):
    L = built.lib()
    for code in range(0, -9, -1):
        assert L.dgk_status_string(code)


def test_create_without_gpu_fails_cleanly(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    rc = built.lib().dgk_create(C.byref(h), 0, None)
    assert rc != 0 and not h.value
    assert built.lib().dgk_last_error()
