"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that the headers under include/ declare (fastmc.h, the method's API;
fastmc_diag.h, diagnostics and test hooks).  No compute calls are made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fastmc.h")
HEADERS = [HEADER, os.path.join(ROOT, "include", "fastmc_diag.h")]


def declared_functions():
    text = "\n".join(open(h).read() for h in HEADERS)
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
                 "fmc_kl_basis", "fmc_kle_reconstruct", "fmc_equilibrium", "fmc_simulate", "fmc_moments",
                 "fmc_profile", "fmc_check_wait_path"]:
        assert must in names
    # the method's header declares no test hook
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    for hook in ["fmc_test_sincos", "fmc_check_wait_path", "fmc_profile", "fmc_last_fused_occupancy"]:
        assert hook + "(" not in text


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


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of fmc_scenario and fmc_result have the C layout (gcc
    compiles a probe of the header's sizeof/offsetof; no GPU needed)."""
    import shutil
    import subprocess

    import paper_2007_03847_gb300 as fmc
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    hdr = os.path.join(ROOT, "include")
    fields_s = [f for f, _ in fmc._Scenario._fields_]
    fields_r = [f for f, _ in fmc._Result._fields_]
    fields_i = [f for f, _ in fmc._Ito._fields_]
    fields_l = [f for f, _ in fmc.LaunchRule._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "fastmc.h"', 'int main(void) {',
           'printf("%zu %zu\\n", sizeof(fmc_scenario), sizeof(fmc_result));']
    src += [f'printf("s {f} %zu\\n", offsetof(fmc_scenario, {f}));' for f in fields_s]
    src += [f'printf("r {f} %zu\\n", offsetof(fmc_result, {f}));' for f in fields_r]
    src += [f'printf("i {f} %zu\\n", offsetof(fmc_ito, {f}));' for f in fields_i]
    src += [f'printf("l {f} %zu\\n", offsetof(fmc_launch_rule, {f}));' for f in fields_l]
    src += ['printf("i_size %zu 0\\n", sizeof(fmc_ito));']
    src += ['printf("l_size %zu 0\\n", sizeof(fmc_launch_rule));']
    src += ["return 0; }"]
    c = tmp_path / "probe.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", hdr, str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    size_s, size_r = map(int, out[0].split())
    assert size_s == ctypes.sizeof(fmc._Scenario)
    assert size_r == ctypes.sizeof(fmc._Result)
    for line in out[1:]:
        if not line:
            continue
        kind, name, off = line.split()
        if kind == "i_size":
            assert int(name) == ctypes.sizeof(fmc._Ito)
            continue
        if kind == "l_size":
            assert int(name) == ctypes.sizeof(fmc.LaunchRule)
            continue
        cls = {"s": fmc._Scenario, "r": fmc._Result, "i": fmc._Ito, "l": fmc.LaunchRule}[kind]
        assert getattr(cls, name).offset == int(off), (kind, name)


def test_scenario_marshalling_carries_the_options():
    """The binding's fmc_scenario carries every option of a synthetic scenario
    (pure marshalling, no library call)."""
    import fmc_synth as fs
    import paper_2007_03847_gb300 as fmc
    sc = fs.multimachine_case(n=4, d=2, K=7, T=0.5, dt=0.005, N=33, seed=9).replace(
        forcing=fs.FORCING_SMOOTH, basis=fs.BASIS_COSINE, integrator=fs.HEUN, sampling=fs.LHS_MIDPOINT,
        event_machine=2, event_time=0.1, event_dpm=-0.3, ito=[fs.ito_gamma(2.0, 4.0), None])
    st = fmc.ScenarioStruct(sc, precision="f32")
    s = st.s
    assert (s.n, s.d, s.K, s.N, s.seed) == (4, 2, 7, 33, 9)
    assert s.forcing == fmc.FORCING_SMOOTH and s.basis == fmc.BASIS_COSINE
    assert s.integrator == fmc.HEUN and s.sampling == fs.LHS_MIDPOINT
    assert s.event_machine == 2 and s.event_time == 0.1 and s.event_dpm == -0.3
    assert s.ito and st.ito[0].kind == fmc.ITO_SQRT and st.ito[1].kind == 0
    assert fmc.ScenarioStruct(sc.replace(forcing=fs.FORCING_INCREMENTS)).s.forcing == fmc.FORCING_INCREMENTS
