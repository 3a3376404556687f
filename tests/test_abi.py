"""The C ABI without a GPU: the library builds, loads, exports every function
include/mp.h declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1305_6758_gb300.build import build

    build()
    import paper_1305_6758_gb300 as mp

    return mp.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*)\s+(mp_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mp_create", "mp_create_ex", "mp_run", "mp_estimates", "mp_destroy"):
        assert required in names


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_function():
    import paper_1305_6758_gb300 as mp

    extra = {"mp_run_noalloc"}  # called directly through ctypes by its test
    assert set(declared_functions()) - extra == set(mp.EXPORTS)


@pytest.mark.parametrize("args,needle", [
    ((5, 1.5, 1.0, 0.0, 16, 1, 1, 1), "even"),          # odd L
    ((4, 0.0, 1.0, 0.0, 16, 1, 1, 1), "T > 0"),         # T <= 0
    ((4, 1.5, 1.0, 0.0, 0, 1, 1, 1), "n_paths"),        # no paths
    ((4, 1.5, 1.0, 0.0, 16, -1, 1, 1), "n_therm"),      # negative sweeps
    ((4, 1.5, 1.0, 0.0, 16, 1, 0, 1), "n_meas"),        # no measurement sweep
    ((4, float("nan"), 1.0, 0.0, 16, 1, 1, 1), "T > 0"),
    ((4, 1.5, float("inf"), 0.0, 16, 1, 1, 1), "finite"),
    ((2048, 1.5, 1.0, 0.0, 16, 1, 1, 1), "1024"),       # absurd size
])
def test_invalid_arguments_rejected_on_the_host(lib, args, needle):
    h = ctypes.c_void_p()
    rc = lib.mp_create(*args, ctypes.byref(h))
    assert rc == -1  # MP_EINVAL
    assert h.value is None
    assert needle in lib.mp_last_error(None).decode()


def test_null_out_and_status_strings(lib):
    assert lib.mp_create(4, 1.5, 1.0, 0.0, 16, 1, 1, 1, None) == -1
    assert lib.mp_status_string(-6) == b"MP_ETIMEOUT"
    assert lib.mp_status_string(0) == b"MP_OK"
    lib.mp_destroy(None)  # NULL-safe
    assert lib.mp_run(None) == -1


def test_noalloc_rejects_oversized_batches_before_the_device(lib):
    import paper_1305_6758_gb300 as mp

    lib.mp_run_noalloc.argtypes = [ctypes.POINTER(mp.MPSystem), ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                   ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    big = (mp.MPSystem * 1)(mp.MPSystem(0, 4, 1.0, 1.0, 0.0, 20000))
    assert lib.mp_run_noalloc(big, 1, 0, 1, 1, 1, ctypes.c_void_p(16), None) == -1
