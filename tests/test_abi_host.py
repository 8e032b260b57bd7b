"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/ntu.h declares, and rejects
invalid configurations before touching the device."""
import ctypes

import pytest

from paper_2107_06635_gb300 import build as B
from paper_2107_06635_gb300 import ntu


@pytest.fixture(scope="module")
def lib():
    return ntu.load()


def test_library_builds_for_sm103a(lib):
    import os
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(B.LIB) and B.up_to_date()


def test_every_declared_symbol_is_exported(lib):
    names = ntu.header_symbols()
    assert len(names) >= 19
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(ntu._SIGS), "binding and header disagree"


@pytest.mark.parametrize("field,value", [("D", 0), ("D", 9), ("d_phys", 1), ("r", 0), ("r", 5),
                                          ("precision", 7), ("tau_kmin", 9), ("max_batch", 0),
                                          ("wait_budget", -1)])
def test_init_rejects_bad_config(lib, field, value):
    cfg = ntu.Config(4, 2, 1, 2, 10, 0, 4, 15, 1)
    if field == "tau_kmin":
        cfg.tau_kmin, cfg.tau_kmax = 9, 5
    else:
        setattr(cfg, field, value)
    h = ctypes.c_void_p()
    st = lib.ntu_init(ctypes.byref(cfg), None, ctypes.byref(h))
    assert st == 1, lib.ntu_last_error(None)
    assert h.value is None
    assert lib.ntu_last_error(None)


def test_init_rejects_too_few_rows(lib):
    # D=1, d_p=2 gives a 2 x r gated matrix: r=4 would need 4 rows
    cfg = ntu.Config(1, 2, 1, 4, 10, 0, 4, 15, 1)
    h = ctypes.c_void_p()
    assert lib.ntu_init(ctypes.byref(cfg), None, ctypes.byref(h)) == 1


def test_init_rejects_bf16x3_beyond_one_k_tile(lib):
    # the fused t1-t2 holds one 64-wide K tile of Y: 2 d_p D <= 64; d_phys=4,
    # d_anc=2, D=8 gives 128 and must be refused before any device work
    cfg = ntu.Config(8, 4, 2, 2, 10, 2, 4, 8, 1)
    h = ctypes.c_void_p()
    assert lib.ntu_init(ctypes.byref(cfg), None, ctypes.byref(h)) == 6
    assert h.value is None
    assert b"2*d_phys*d_anc*D" in lib.ntu_last_error(None)


def test_null_arguments(lib):
    assert lib.ntu_init(None, None, None) == 1
    assert lib.ntu_destroy(None) == 0
    assert lib.ntu_sync(None) == 1
    assert lib.ntu_inject_wait_timeout(None, 1) == 1


def test_uneven_init_rejects_bad_kinds(lib):
    import ctypes as C
    D = (C.c_int * 2)(4, 4)
    r = (C.c_int * 2)(2, 2)
    cap = (C.c_int * 2)(1, 1)
    h = C.c_void_p()
    st = lib.ntu_uneven_init(2, 1, 10, 0, 4, 15, 2, C.cast(D, C.c_void_p), C.cast(r, C.c_void_p),
                             C.cast(cap, C.c_void_p), None, C.byref(h))
    assert st == 1 and h.value is None
    assert b"repeats" in lib.ntu_uneven_last_error(None)
    assert lib.ntu_uneven_init(2, 1, 10, 0, 4, 15, 0, None, None, None, None, C.byref(h)) == 1
    assert lib.ntu_uneven_destroy(None) == 0
    # every uneven call rejects a NULL handle without touching a device
    assert lib.ntu_uneven_stage(None, 0, None, None, None, None) == 1
    assert lib.ntu_uneven_run(None, 0) == 1
    assert lib.ntu_uneven_sync(None) == 1
    assert lib.ntu_uneven_fetch(None, 0, None, None, None, None) == 1
    assert lib.ntu_uneven_update_host(None, 0, None, None, None, None, None, None, None, 0) == 1
    assert lib.ntu_uneven_last_launch_count(None) == 0


def test_init_without_a_device_fails_cleanly(lib):
    """A valid configuration on a machine without a usable GPU: context
    creation reports a CUDA error (NTU_ECUDA = 3) with a message, returns no
    handle and leaves the library usable."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = ntu.Config(4, 2, 1, 2, 10, 2, 4, 8, 8)
    h = ctypes.c_void_p()
    assert lib.ntu_init(ctypes.byref(cfg), None, ctypes.byref(h)) == 3
    assert h.value is None
    assert lib.ntu_last_error(None)
    assert lib.ntu_init(None, None, None) == 1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the compiled library the binding raises
    instead of computing anything."""
    monkeypatch.setattr(ntu, "_LIB", None)
    monkeypatch.setattr(B, "LIB", str(tmp_path / "libntu_missing.so"))
    with pytest.raises(OSError):
        ntu.load(build=False)
    assert ntu._LIB is None
