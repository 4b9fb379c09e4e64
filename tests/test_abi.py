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


def _static_call(built, dim, N, n, count, precision="fp64"):
    """dgk_rhs_static on host stand-in pointers: the call must refuse before any device
    work (the pointers are never dereferenced)."""
    p = built.make_params(precision=precision)
    m = built.make_box_mesh(dim, N, list(n) + [1] * (3 - len(n)), [0.0] * 3, [1.0] * 3, [1, 1, 1])
    buf = (C.c_double * 8)()
    ptr = C.cast(buf, C.c_void_p)
    return built.lib().dgk_rhs_static(C.byref(p), C.byref(m), ptr, ptr, count, None, None)


def test_static_rhs_refuses_bad_sizes_before_device_work(built):
    """Overflowing element counts, sums that wrap around 2^64, counts that do not match the
    mesh and a bad dimension are refused with DGK_ERR_ARG / DGK_ERR_UNSUPPORTED and a
    message; nothing touches the device (this runs without a GPU)."""
    L = built.lib()
    # 2^30 x 2^29 elements in 2D: the element count alone passes 2^32
    assert _static_call(built, 2, 5, [1 << 30, 1 << 29], 8) == -1
    assert b"static scratch" in L.dgk_last_error()
    # 3D, each factor < 2^31, product of the first two already >= 2^32
    assert _static_call(built, 3, 3, [1 << 20, 1 << 20, 2], 8) == -1
    # a small mesh whose count does not match nvar * nelem * np
    assert _static_call(built, 2, 3, [4, 4], 5 * 16 * 16 - 1) == -1
    assert b"count" in L.dgk_last_error()
    # dimension checked before anything indexes by it
    assert _static_call(built, 4, 3, [2, 2, 2], 8) == -6
    # a mesh that fits no 64 MiB scratch, with a matching count
    assert _static_call(built, 3, 5, [16, 16, 16], 6 * 4096 * 216) == -1
    assert b"static scratch" in L.dgk_last_error()


def test_static_rhs_wrapper_checks_tensor_sizes(built):
    """The Python wrapper computes nvar * nelem * np from the mesh and refuses arrays of
    another size before calling the library."""
    import numpy as np
    p = built.make_params()
    m = built.make_box_mesh(2, 3, [4, 4, 1], [0.0] * 3, [1.0] * 3, [1, 1, 1])
    with pytest.raises(built.DgkError, match="nvar"):
        built.rhs_static(p, m, np.zeros(5 * 16 * 16 - 1), np.zeros(5 * 16 * 16))
