"""The C-ABI library builds, loads and exports every entry point declared in
include/scfft.h; host-side argument validation works without a GPU."""

import ctypes
import os
import re

import pytest

import paper_1803_01346_gb300 as S
from paper_1803_01346_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return S.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "scfft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(scfft_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert set(declared_functions()) == set(S.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code in range(9):
        assert lib.scfft_status_string(code)
    assert lib.scfft_status_string(0) == b"ok"


def test_create_rejects_bad_arguments_on_host(lib):
    """Validation happens before any CUDA call, so this runs without a GPU."""
    out = ctypes.c_void_p()
    m = S._Material(20.0, 1.0, 1.0, 20.0, 1.0)
    o = S._Options(0, 2e-5, 100, 1.0, 2e-4, 1e-6)
    for g in (S._Grid(17, 16, 16, 1, 1, 1), S._Grid(16, 16, 256, 1, 1, 1), S._Grid(16, 16, 16, 0, 1, 1)):
        assert lib.scfft_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(o), None, ctypes.byref(out)) == 1
    g = S._Grid(16, 16, 16, 1, 1, 1)
    bad_m = S._Material(0.5, 1.0, 1.0, 20.0, 1.0)
    assert lib.scfft_create(ctypes.byref(g), ctypes.byref(bad_m), ctypes.byref(o), None, ctypes.byref(out)) == 1
    bad_o = S._Options(7, 2e-5, 100, 1.0, 2e-4, 1e-6)
    assert lib.scfft_create(ctypes.byref(g), ctypes.byref(m), ctypes.byref(bad_o), None, ctypes.byref(out)) == 1
    assert lib.scfft_rhs(None, 0.0, 0, None, None, None, None) == 1
    t, dt = ctypes.c_double(0.0), ctypes.c_double(1e-3)
    assert lib.scfft_step_host(None, ctypes.byref(t), ctypes.byref(dt), 1.0, None, None, None, None, None) == 1
    lib.scfft_destroy(None)


def test_every_entry_point_validates_before_any_cuda_call(lib):
    """A null context (or null arrays) gives SCFFT_EINVAL from every entry point without a
    GPU: each validates its arguments before it touches CUDA."""
    d = ctypes.c_double(0.0)
    sz = ctypes.c_size_t(0)
    calls = {
        "scfft_set_geometry": (None, None),
        "scfft_set_jc_map": (None, None),
        "scfft_set_field_path": (None, None),
        "scfft_precompute_kernel": (None,),
        "scfft_curl": (None, None, None),
        "scfft_phi": (None, None, None),
        "scfft_step": (None, ctypes.byref(d), ctypes.byref(d), 1.0, None, None, None),
        "scfft_checkpoint_save": (None, 0.0, 1e-3, None, None, None, ctypes.byref(sz)),
        "scfft_checkpoint_load": (None, None, 0, ctypes.byref(d), ctypes.byref(d), None, None),
        "scfft_integrate": (None, 0.0, 1.0, 1e-3, 0, None, None, None, None, None, 0, None),
        "scfft_rhs_vjp": (None, None, None, None, None, None, None),
        "scfft_adjoint_integrate": (None, 0.0, None, 1, None, None, None, None, None, None, 4),
        "scfft_batch_step": (None, 1, None, None, None, None, None, None),
        "scfft_sync": (None,),
        "scfft_inject_fault": (None, 0),
        "scfft_get_stats": (None, None),
        "scfft_profile": (None, 1),
        "scfft_profile_read": (None, None, None),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == 1, name
    g = S._Grid(16, 16, 16, 1.0, 1.0, 1.0)
    assert lib.scfft_curl_noalloc(ctypes.byref(g), 1.0, None, None, None) == 1
