"""The C-ABI library builds for sm_103a and exports every entry point that
include/thc.h declares (no GPU: nothing is computed here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "thc.h")
LIB = os.path.join(ROOT, "paper_2409_12708_gb300", "lib", "libthc.so")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    # top-level prototypes start in column 0: "<type words> name("
    names = re.findall(r"^(?:[A-Za-z_]\w*[\s*]+)+([A-Za-z_]\w*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2409_12708_gb300 import build as b
        b.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for n in ["thc_apply_H", "mps_inner", "mps_add_compress", "krylov_lanczos_ground",
              "krylov_expm_apply", "thc_layer_apply", "thc_compress", "thc_kinetic_factors",
              "thc_mps_free", "thc_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_build_info_and_error_string_without_gpu(lib):
    lib.thc_build_info.restype = ctypes.c_char_p
    lib.thc_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.thc_build_info()
    assert isinstance(lib.thc_last_error(), bytes)


def test_invalid_arguments_rejected_before_any_gpu_work(lib):
    # a null descriptor is THC_EINVAL and touches no device
    lib.thc_apply_H.restype = ctypes.c_int
    assert lib.thc_apply_H(None, None, None, None, None, None) == 1
    lib.thc_last_error.restype = ctypes.c_char_p
    assert b"null" in lib.thc_last_error()


def test_binding_names_match_header():
    from paper_2409_12708_gb300 import binding as B
    assert set(B.EXPORTED) == set(declared_functions())
