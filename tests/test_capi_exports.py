"""The CUDA library builds for sm_103a, loads without a GPU and exports every
entry point that include/cavity.h declares (no compute calls here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if hdr.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", hdr)).read()
            names += re.findall(r"^CAVITY_API\s+[\w\s\*]*?\b(cavity_\w+)\s*\(", txt, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2006_02602_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = set(_declared())
    for required in ("cavity_create", "cavity_set_params", "cavity_step", "cavity_residual",
                     "cavity_nusselt", "cavity_get_fields", "cavity_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_mirrors_the_header(lib):
    import paper_2006_02602_gb300 as m
    declared = set(_declared())
    assert set(m.EXPORTED) == declared
    for name in declared:
        assert callable(getattr(m, name)), name


def test_host_only_calls_without_gpu(lib):
    import paper_2006_02602_gb300 as m
    L = m.load_library()
    p = m.cavity_params()
    assert L.cavity_default_params(ctypes.byref(p)) == 0
    assert p.Ra == 1e5 and p.gravity_axis == 2 and p.u_ref == pytest.approx((1e5 * 0.71) ** 0.5)
    assert L.cavity_default_params(None) == m.CAVITY_ERR_INVALID_ARG
    assert L.cavity_destroy(None) == 0
    assert L.cavity_strerror(m.CAVITY_ERR_NONFINITE).decode().startswith("non-finite")
    out = ctypes.c_void_p(123)
    assert L.cavity_create(None, ctypes.byref(out)) == m.CAVITY_ERR_INVALID_ARG
    assert out.value is None
    d = m.cavity_desc(1, 8, 8, 1, 1, 1, 0, 0, 0.0, 0, None)
    assert L.cavity_create(ctypes.byref(d), ctypes.byref(out)) == m.CAVITY_ERR_INVALID_ARG
    d = m.cavity_desc(8, 8, 8, 5, 1, 1, 0, 0, 0.0, 0, None)  # blocks thinner than 2 nodes
    assert L.cavity_create(ctypes.byref(d), ctypes.byref(out)) == m.CAVITY_ERR_INVALID_ARG
    assert L.cavity_step(None, 1) == m.CAVITY_ERR_INVALID_ARG
