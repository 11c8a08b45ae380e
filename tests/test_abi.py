"""CPU checks of the C ABI: the library builds, loads and exports every declared symbol,
and argument validation answers with status codes before any device work."""
import ctypes
import os
import re

import pytest

from paper_1204_1225_gb300 import build as khbuild
from paper_1204_1225_gb300 import kirchhoff as kh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "kirchhoff.h")).read()
    return sorted(set(re.findall(r"^KH_API\s+[\w\s\*]+?\b(kirchhoff_\w+)\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def L():
    khbuild.build()
    return kh.lib()


def test_header_declares_the_abi():
    syms = declared_symbols()
    for name in ("kirchhoff_create", "kirchhoff_migrate", "kirchhoff_demigrate", "kirchhoff_destroy"):
        assert name in syms
    assert set(syms) == set(kh.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    for name in declared_symbols():
        assert hasattr(L, name), name
    assert "sm_103a" in kh.kirchhoff_version()


def _desc(**kw):
    d = kh.kh_desc(2, 16, 1, 16, 0.0, 0.0, 0.0, 10.0, 10.0, 10.0, 4, 50.0, kh.KH_VEL_CONST, 2000.0,
                   0.0, 25.0, kh.KH_F16, kh.KH_W_ONE, 1000.0, 0.0, 64, 0.0, 0.004, kh.KH_F32)
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("field,value,status", [
    ("dim", 4, kh.KH_ERR_INVALID_ARG),
    ("nx", 0, kh.KH_ERR_INVALID_ARG),
    ("ny", 3, kh.KH_ERR_INVALID_ARG),          # dim 2 needs ny == 1
    ("dz", 0.0, kh.KH_ERR_INVALID_ARG),
    ("n_bins", 0, kh.KH_ERR_INVALID_ARG),
    ("n_bins", 257, kh.KH_ERR_INVALID_ARG),
    ("bin_width", -1.0, kh.KH_ERR_INVALID_ARG),
    ("v0", 0.0, kh.KH_ERR_INVALID_ARG),
    ("nt", 1, kh.KH_ERR_UNSUPPORTED),
    ("dt", 0.0, kh.KH_ERR_INVALID_ARG),
    ("weight", 7, kh.KH_ERR_INVALID_ARG),
    ("trace_dtype", 9, kh.KH_ERR_INVALID_ARG),
    ("nt", 1 << 20, kh.KH_ERR_UNSUPPORTED),    # too long for the shared-memory ring
])
def test_create_rejects_bad_descriptors(L, field, value, status):
    h = ctypes.c_void_p()
    rc = L.kirchhoff_create(ctypes.byref(_desc(**{field: value})), ctypes.byref(h))
    assert rc == status
    assert h.value is None
    assert L.kirchhoff_last_error()


def test_create_rejects_nonpositive_velocity_in_grid(L):
    h = ctypes.c_void_p()
    d = _desc(vel=kh.KH_VEL_LINEAR_Z, v0=1000.0, k=-10.0)   # v(150 m) = -500 m/s
    assert L.kirchhoff_create(ctypes.byref(d), ctypes.byref(h)) == kh.KH_ERR_UNSUPPORTED


def test_null_arguments(L):
    assert L.kirchhoff_create(None, None) == kh.KH_ERR_INVALID_ARG
    assert L.kirchhoff_migrate(None, 0, None, None, None, None, None, None, None) == kh.KH_ERR_INVALID_ARG
    assert L.kirchhoff_set_option(None, 1, 0) == kh.KH_ERR_INVALID_ARG
    assert L.kirchhoff_destroy(None) == kh.KH_OK
