"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/fastmc.h declares.  No compute calls are made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fastmc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(fmc_[a-z_0-9]+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import paper_2007_03847_gb300 as fmc
    path = fmc.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ["fmc_create", "fmc_destroy", "fmc_last_error", "fmc_lhs_sample", "fmc_lhs_sample_split",
                 "fmc_kl_basis", "fmc_kle_reconstruct", "fmc_equilibrium", "fmc_simulate", "fmc_moments"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib.fmc_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t]
    lib.fmc_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    rc = lib.fmc_create(ctypes.byref(h), 0, 0)
    assert rc != 0 and not h.value
    assert lib.fmc_last_error(None)


def test_binding_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2007_03847_gb300 as fmc
    with pytest.raises(fmc.FastMCError):
        fmc.Context(0)
