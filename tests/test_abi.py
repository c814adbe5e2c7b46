"""The C-ABI library loads and exports every symbol include/moff.h declares;
argument checks that run before any CUDA call report MOFF_EINVAL (CPU only)."""
import ctypes

import numpy as np
import pytest

import paper_0812_3669_gb300 as moff


@pytest.fixture(scope="module")
def L():
    moff.build()
    return moff.lib()


def test_header_declares_the_boundary():
    syms = moff.header_symbols()
    for name in ["moff_plan_create", "moff_set_gains", "moff_submit", "moff_read_image",
                 "moff_submit_adc", "moff_set_fstage", "moff_plan_destroy", "moff_last_error"]:
        assert name in syms


def test_library_exports_every_declared_symbol(L):
    for name in moff.header_symbols():
        assert hasattr(L, name), name


def test_argument_errors_without_gpu(L):
    out = ctypes.c_void_p()
    pos = np.zeros((4, 2))
    taps = np.ones((4, 1, 3, 3, 2), dtype=np.float32)
    # NULL out pointer
    assert L.moff_plan_create(None, 4, pos.ctypes.data, 3, taps.ctypes.data, 32, 1, 1, 0, None) == -1
    assert "out" in moff.moff_last_error()
    bad = [
        (0, 3, 32, 1, 1, 0),        # no antennas
        (4, 2, 32, 1, 1, 0),        # even kernel
        (4, 3, 48, 1, 1, 0),        # grid not a supported power of two
        (4, 3, 32, 0, 1, 0),        # no channels
        (4, 3, 32, 1, 3, 0),        # three pols
        (4, 3, 32, 1, 1, 4),        # Jones with one pol
        (4, 3, 32, 24, 1, 2),       # F-stage with non power-of-two channels
        (4, 3, 32, 1, 1, 1 << 9),   # unknown flag
        (4, 3, 32, 1, 1, 1 << 7),   # unknown flag next to MOFF_PERSIST
        (4, 3, 32, 1, 1, (1 << 6) | 1),   # MOFF_PERSIST with MOFF_PREC_FP16TC
        (4, 3, 32, 1, 1, (1 << 6) | 8),   # MOFF_PERSIST with MOFF_SERVED
    ]
    for (A, K, N, C, P, fl) in bad:
        st = L.moff_plan_create(ctypes.byref(out), A, pos.ctypes.data, K, taps.ctypes.data, N, C, P, fl, None)
        assert st == -1, (A, K, N, C, P, fl)
        assert not out.value
        assert moff.moff_last_error() != ""
    assert L.moff_plan_destroy(None) == 0
    assert L.moff_submit(None, None, 1, 0) == -1
    assert L.moff_read_image(None, None, None, 0, 0, 0) == -1


def test_python_binding_raises_on_error(L):
    with pytest.raises(moff.MoffError) as e:
        moff.moff_plan_create(np.zeros((0, 2)), np.ones((0, 1, 3, 3), complex), 32, 1, 1)
    assert e.value.status == -1


def test_server_argument_errors_without_gpu(L):
    out = ctypes.c_void_p()
    assert L.moff_server_create(None, 1 << 20, 1) == -1
    assert L.moff_server_create(ctypes.byref(out), 0, 1) == -1          # no pool
    assert "hbm_budget_bytes" in moff.moff_last_error()
    assert L.moff_server_create(ctypes.byref(out), 1 << 20, 0) == -1    # no slots
    assert L.moff_server_create(ctypes.byref(out), 1 << 20, 65) == -1   # too many slots
    assert not out.value
    t = ctypes.c_longlong(7)
    assert L.moff_server_submit(None, None, None, 1, 0, ctypes.byref(t)) == -1
    st = ctypes.c_int()
    assert L.moff_server_poll(None, 1, ctypes.byref(st), None) == -1
    assert L.moff_server_wait(None, 0, 0) == -1
    assert L.moff_server_stats(None, None, None, None, None, 0) == -1
    assert L.moff_server_destroy(None) == 0
