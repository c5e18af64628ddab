"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every function that include/cpdgn.h declares, validates shapes and sizes its
workspace without touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cpdgn.h")
LIB = os.path.join(ROOT, "paper_1205_2584_gb300", "lib", "libcpdgn.so")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_1205_2584_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|double\*|cp_status\*|void)\s+\**\s*(cp_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_abi():
    names = declared_functions()
    for required in ("cp_gram", "cp_mttkrp_all", "cp_dgn_core_build", "cp_dgn_solve", "cp_dgn_step",
                     "cp_fit", "cp_workspace_bytes", "cp_state_create", "cp_state_init"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_workspace_and_validation_host_only(lib):
    from paper_1205_2584_gb300 import cpdgn as cp
    s = cp.make_shape((200, 200, 200), 20, "f32")
    b0 = cp.workspace_bytes(s, cp.CP_CORE_F64, False)
    b1 = cp.workspace_bytes(s, cp.CP_CORE_MIXED, True)
    n = 3 * 20 * 20
    assert b1 >= n * n * 4 and b0 > 0
    assert cp.workspace_bytes(s, cp.CP_CORE_F64, True) >= n * n * 8
    for bad in [cp.make_shape((5,), 2, "f64"), cp.make_shape((5, 6), 0, "f64"),
                cp.make_shape((5, 6), 33, "f64"), cp.make_shape((5, 0, 3), 2, "f64")]:
        with pytest.raises(cp.CPError):
            cp.workspace_bytes(bad)
    # the two-plane bfloat16 form exists only for 3-way tensors with I_1 % 8 == 0
    assert cp.workspace_bytes(cp.make_shape((64, 30, 7), 5, "bf16x2")) > 0
    for bad in [cp.make_shape((60, 30, 7), 5, "bf16x2"), cp.make_shape((8, 8, 8, 8), 2, "bf16x2")]:
        with pytest.raises(cp.CPError):
            cp.workspace_bytes(bad)
    bad_dtype = cp.make_shape((8, 8, 8), 2, "f32")
    bad_dtype.y_dtype = 4
    with pytest.raises(cp.CPError):
        cp.workspace_bytes(bad_dtype)
    assert cp._lib.cp_tensor_split(None, 8, None, None) == 1
    out = ctypes.c_size_t(0)
    assert cp._lib.cp_workspace_bytes(ctypes.byref(s), 7, 0, ctypes.byref(out)) == 1
    # null pointers are rejected on the host before any device work
    assert cp._lib.cp_gram(ctypes.byref(s), None, None, None, None, None, 0, None) == 1
    assert cp._lib.cp_state_create(ctypes.byref(s), None, None, None, 0, None) == 1
