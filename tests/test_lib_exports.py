"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
symbol include/cov.h declares, and its host-only functions behave."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cov.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2511_11514_b300 import build_lib
    path = build_lib.build()
    return ctypes.CDLL(path)


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^COV_API\s+[\w\s\*]+?\b(cov_\w+)\(", txt, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("cov_field_svgd", "cov_field_sinkhorn", "cov_lqr_track", "cov_solve"):
        assert required in names
    assert len(names) >= 17


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_export_list_matches_header():
    from paper_2511_11514_b300 import binding
    assert sorted(binding.EXPORTS) == _declared()


def test_status_strings(lib):
    lib.cov_status_string.restype = ctypes.c_char_p
    assert lib.cov_status_string(0) == b"COV_OK"
    assert lib.cov_status_string(5) == b"COV_ERR_TIMEOUT"
    assert lib.cov_status_string(99) == b"COV_ERR_UNKNOWN"


def test_workspace_size_is_monotone_and_rejects_bad_sizes(lib):
    f = lib.cov_workspace_size
    f.restype = ctypes.c_size_t
    f.argtypes = [ctypes.c_int] * 5
    assert f(0, 10, 2, 0, 0) == 0
    assert f(10, 10, 7, 0, 0) == 0
    a = f(4096, 16384, 2, 4, 2)
    b = f(65536, 262144, 2, 3, 2)
    assert 0 < a < b
    assert f(4096, 0, 2, 4, 2) > 0


def test_context_creation_without_device_is_an_error_not_a_crash(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    lib.cov_ctx_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t]
    assert lib.cov_ctx_create(ctypes.byref(h), 0, 0) != 0
    assert not h.value


def test_null_context_calls_return_invalid_arg(lib):
    lib.cov_field_sinkhorn.restype = ctypes.c_int
    assert lib.cov_field_sinkhorn(None, None, 1, None, None, 1, 2, ctypes.c_float(0.1), 1, 0,
                                  None, None, None, None, None) == 1
    lib.cov_solve.restype = ctypes.c_int
    assert lib.cov_solve(None, None, 1, None, None, None) == 1
