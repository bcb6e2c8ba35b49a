"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point that include/mcspect.h declares (no compute calls)."""
import ctypes
import os
import re
import subprocess

import numpy as np

from paper_2105_13324_gb300 import build as B
from paper_2105_13324_gb300 import mcspect

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^MC_API\s+(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", txt, flags=re.M))
    return names


def test_header_declares_the_binding_names():
    assert _declared() == set(mcspect.EXPORTED)


def test_library_exports_every_declared_symbol():
    path = B.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = _declared() - exported
    assert not missing, missing
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert getattr(lib, name) is not None


def test_structs_match_header_layout():
    # sizes/offsets the C compiler gives the header's structs
    src = r'''
    #include <stdio.h>
    #include <stddef.h>
    #include "mcspect.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu\n", sizeof(mc_phantom), sizeof(mc_geometry), sizeof(mc_system_info),
             sizeof(mc_history_record), offsetof(mc_geometry, precision), offsetof(mc_history_record, e_final_kev));
      return 0;
    }'''
    tmp = os.path.join(ROOT, "paper_2105_13324_gb300", "_build")
    os.makedirs(tmp, exist_ok=True)
    c = os.path.join(tmp, "layout_probe.c")
    exe = os.path.join(tmp, "layout_probe")
    with open(c, "w") as f:
        f.write(src)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(mcspect.MCPhantom), ctypes.sizeof(mcspect.MCGeometry), ctypes.sizeof(mcspect.MCSystemInfo),
            mcspect.RECORD_DTYPE.itemsize, mcspect.MCGeometry.precision.offset,
            mcspect.RECORD_DTYPE.fields["e_final_kev"][1]]
    assert got == want


def test_error_message_is_empty_before_any_call():
    lib = mcspect.load(B.build())
    assert lib.mc_last_error() == b""


def test_invalid_arguments_are_rejected_on_the_host():
    # argument checks run before any device call, so they work without a GPU
    lib = mcspect.load(B.build())
    h = ctypes.c_void_p()
    rc = lib.mc_build_system(None, None, 10, 1, None, ctypes.byref(h))
    assert rc == mcspect.MC_EINVAL and b"phantom" in lib.mc_last_error()
    rows = np.array([0, 5], np.int32)
    cols = np.array([0, 1], np.int32)
    rc = lib.mc_system_from_events(4, 4, rows.ctypes.data, cols.ctypes.data, 2, 0, 10, None, ctypes.byref(h))
    assert rc == mcspect.MC_EINVAL and b"out of range" in lib.mc_last_error()
    assert lib.mc_system_free(None) == mcspect.MC_OK


def test_tally_material_and_debug_arguments_are_rejected_on_the_host():
    # the checks of the tally flags, the material table and the debug hooks
    # run before any device call
    from paper_2105_13324_gb300 import phantoms as P
    lib = mcspect.load(B.build())
    w = P.workload("water32")
    h = ctypes.c_void_p()
    for kw, word in (({"forced": True, "forced_direction": True, "primary_only": True}, b"FORCED_DIRECTION"),
                     ({"forced_direction": True}, b"FORCED_DIRECTION")):
        inp = mcspect._Inputs(w.phantom, w.geometry, mcspect.MC_FP32, **kw)
        rc = lib.mc_plan_create(ctypes.byref(inp.ph), ctypes.byref(inp.geo), None, ctypes.byref(h))
        assert rc == mcspect.MC_EINVAL and word in lib.mc_last_error() and not h.value
    # a voxel whose material is not in the table
    bad = P.Phantom(w.phantom.material.copy(), w.phantom.rho, w.phantom.z_over_a, w.phantom.z_eff,
                    w.phantom.voxel_mm)
    bad.material[3, 4, 5] = len(w.phantom.rho)
    inp = mcspect._Inputs(bad, w.geometry, mcspect.MC_FP32)
    rc = lib.mc_plan_create(ctypes.byref(inp.ph), ctypes.byref(inp.geo), None, ctypes.byref(h))
    assert rc == mcspect.MC_EINVAL and b"outside the table" in lib.mc_last_error()
    # the distance-map hook: no phantom, no output buffer
    assert lib.mc_debug_distance_map(None, None) == mcspect.MC_EINVAL and b"phantom" in lib.mc_last_error()
    inp = mcspect._Inputs(w.phantom, w.geometry, mcspect.MC_FP32)
    assert lib.mc_debug_distance_map(ctypes.byref(inp.ph), None) == mcspect.MC_EINVAL
    assert b"NULL output" in lib.mc_last_error()
    # weighted events outside the matrix
    rows = np.array([0, 4], np.int32)
    cols = np.array([0, 1], np.int32)
    wq = np.array([1, 2], np.uint64)
    rc = lib.mc_system_from_weighted_events(4, 4, rows.ctypes.data, cols.ctypes.data, wq.ctypes.data, 2, 0, 10,
                                            None, ctypes.byref(h))
    assert rc == mcspect.MC_EINVAL and b"out of range" in lib.mc_last_error()
