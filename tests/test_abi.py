"""Host-side checks of the C ABI: the library builds for sm_103a and exports every
entry point include/lowmach.h declares (no GPU needed, no compute call)."""

import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    with open(os.path.join(ROOT, "include", "lowmach.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sim_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2603_01727_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert "sim_create" in names and "sim_step" in names and "sim_poisson_solve" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib_path):
    from paper_2603_01727_gb300 import lowmach
    assert sorted(lowmach.exported_symbols()) == _declared()
    lowmach.load()


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of sim_params_t / sim_ibm_t agree with the C compiler's
    layout of the header (sizes and every field offset)."""
    import subprocess
    from paper_2603_01727_gb300 import lowmach
    fields_p = [f for f, _ in lowmach.SimParams._fields_]
    fields_b = [f for f, _ in lowmach.SimIbm._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "lowmach.h"', "int main(void) {",
           '  printf("%zu\\n", sizeof(sim_params_t));']
    src += [f'  printf("%zu\\n", offsetof(sim_params_t, {f}));' for f in fields_p]
    src += ['  printf("%zu\\n", sizeof(sim_ibm_t));']
    src += [f'  printf("%zu\\n", offsetof(sim_ibm_t, {f}));' for f in fields_b]
    src += ["  return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(lowmach.SimParams)] + [getattr(lowmach.SimParams, f).offset for f in fields_p]
    want += [ctypes.sizeof(lowmach.SimIbm)] + [getattr(lowmach.SimIbm, f).offset for f in fields_b]
    assert got == want


def test_invalid_parameters_rejected_without_gpu(lib_path):
    """Validation happens before any CUDA call."""
    import workloads as W
    from paper_2603_01727_gb300 import lowmach as L
    lib = L.load()
    prm, _, _ = W.slot_burner(32, 64)
    sz = ctypes.c_size_t()
    p = L.params_struct(prm)
    assert lib.sim_workspace_size(ctypes.byref(p), ctypes.byref(sz)) == L.SIM_OK
    for key, val in [("dt", 0.0), ("dim", 4), ("poisson_rtol", 2.0), ("precision", 7), ("precision", -1)]:
        bad = dict(prm)
        bad[key] = val
        assert lib.sim_workspace_size(ctypes.byref(L.params_struct(bad)), ctypes.byref(sz)) == L.SIM_EINVAL
    bad = dict(prm)
    bad["bc"] = [[0, 1], [1, 2], [0, 0]]          # periodic without a periodic partner
    assert lib.sim_workspace_size(ctypes.byref(L.params_struct(bad)), ctypes.byref(sz)) == L.SIM_EINVAL
    bad = dict(prm)
    bad["closed_system"] = 1                      # enclosed but with inflow/outflow
    assert lib.sim_workspace_size(ctypes.byref(L.params_struct(bad)), ctypes.byref(sz)) == L.SIM_EINVAL
    h = ctypes.c_void_p()
    assert lib.sim_create(ctypes.byref(p), None, 0, None, ctypes.byref(h)) == L.SIM_ENOMEM


def test_variant_parameters_validated_without_gpu(lib_path):
    """The semi-enclosed system, the transport law and the isothermal walls are
    checked by the host before any CUDA call."""
    import workloads as W
    from paper_2603_01727_gb300 import lowmach as L
    lib = L.load()
    sz = ctypes.c_size_t()

    def status(prm):
        return lib.sim_workspace_size(ctypes.byref(L.params_struct(prm)), ctypes.byref(sz))

    chamber, _, _ = W.filling_chamber(16)
    assert status(chamber) == L.SIM_OK                                   # inlet, no outlet
    slot, _, _ = W.slot_burner(32, 64)
    assert status(dict(slot, closed_system=2)) == L.SIM_EINVAL           # semi-enclosed with an outlet
    assert status(dict(slot, closed_system=3)) == L.SIM_EINVAL
    assert status(dict(chamber, closed_system=1)) == L.SIM_EINVAL        # enclosed with an inlet
    cavity, _, _ = W.heated_cavity(16)
    assert status(cavity) == L.SIM_OK                                    # isothermal walls, Sutherland
    assert status(dict(cavity, transport=2)) == L.SIM_EINVAL
    assert status(dict(cavity, sutherland_C=-0.1)) == L.SIM_EINVAL
    assert status(dict(cavity, bc=[[6, 6], [3, 3], [0, 0]])) == L.SIM_EINVAL   # unknown kind
    tc, _, _ = W.taylor_couette(32)
    assert status(tc) == L.SIM_OK
    # the tanh-stretched grids of Eq 4.18 exist in the oracle only: the binding
    # refuses them instead of running a uniform grid
    assert status(dict(cavity, stretch=[0.0, 0.0])) == L.SIM_OK
    with pytest.raises(ValueError, match="stretched"):
        L.params_struct(dict(cavity, stretch=[1.8, 1.8]))
