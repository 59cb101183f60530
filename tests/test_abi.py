"""The C ABI library builds, loads and exports every entry point of include/rtu.h;
the Python ctypes structures match the C layout.  No GPU compute is called."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rtu.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rtu_[a-z_0-9]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2606_30620_b300 import build
    lib_path = build.build()
    assert os.path.exists(lib_path)
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert {"rtu_build_grid", "rtu_forward", "rtu_adjoint", "rtu_workspace_size"} <= set(names)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in rtu.h but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}$", out, flags=re.M), n


def test_binding_structs_match_the_c_layout(tmp_path):
    from paper_2606_30620_b300 import rtu
    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "rtu.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(rtu_system_desc), offsetof(rtu_system_desc, weights),
         offsetof(rtu_system_desc, pix),
         offsetof(rtu_system_desc, data), sizeof(rtu_eval), offsetof(rtu_eval, lens),
         offsetof(rtu_eval, g_ps), offsetof(rtu_eval, ray_hist), offsetof(rtu_eval, light),
         offsetof(rtu_eval, g_light), offsetof(rtu_eval, sel_hist), offsetof(rtu_eval, centres));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(rtu.SystemDesc), rtu.SystemDesc.weights.offset, rtu.SystemDesc.pix.offset,
            rtu.SystemDesc.data.offset,
            ctypes.sizeof(rtu.Eval), rtu.Eval.lens.offset, rtu.Eval.g_ps.offset, rtu.Eval.ray_hist.offset,
            rtu.Eval.light.offset, rtu.Eval.g_light.offset, rtu.Eval.sel_hist.offset, rtu.Eval.centres.offset]
    assert got == want


def _desc(**kw):
    from paper_2606_30620_b300 import rtu
    d = dict(n_img=64, s_super=2, n_src=32, psf_k=9, profile=0, sub_kind=0, n_sub=0, ps_family=0,
             precision=0, n_nodes=22, degree=21, n_slots=1, transform=0, n_light=0, pix=0.05,
             src_pitch=0.1, sigma=0.02,
             data=1 << 20, mask=1 << 21, psf=1 << 22, weights=None)
    d.update(kw)
    return rtu.SystemDesc(**d)


def test_workspace_size_validates_the_description():
    from paper_2606_30620_b300 import rtu
    lib = rtu._lib
    ok = lib.rtu_workspace_size(ctypes.byref(_desc()))
    assert ok > 0
    two = lib.rtu_workspace_size(ctypes.byref(_desc(n_slots=2)))
    assert two > ok
    for bad in (dict(n_src=50), dict(n_src=512), dict(psf_k=4), dict(n_nodes=30), dict(s_super=0),
                dict(precision=3), dict(sigma=0.0), dict(n_sub=17), dict(data=0), dict(transform=3),
                dict(transform=-1), dict(n_light=9), dict(n_light=-1),
                dict(transform=rtu.RTU_TRANSFORM_LINEAR, weights=1 << 23)):
        assert lib.rtu_workspace_size(ctypes.byref(_desc(**bad))) == 0, bad
    # the unsmoothed eCDF keeps every order statistic: a larger slot
    lin = lib.rtu_workspace_size(ctypes.byref(_desc(transform=rtu.RTU_TRANSFORM_LINEAR)))
    assert lin > ok
    rc = lib.rtu_system_create(ctypes.byref(_desc(transform=2, weights=1 << 23)), ctypes.c_void_p(1 << 20),
                               1 << 30, ctypes.byref(ctypes.c_void_p()))
    assert rc == -1 and "weights" in lib.rtu_last_error().decode()


def test_create_rejects_bad_workspace_without_touching_the_gpu():
    from paper_2606_30620_b300 import rtu
    lib = rtu._lib
    h = ctypes.c_void_p()
    rc = lib.rtu_system_create(ctypes.byref(_desc()), None, 0, ctypes.byref(h))
    assert rc == -3 and not h.value
    assert "workspace" in lib.rtu_last_error().decode()
    rc = lib.rtu_system_create(ctypes.byref(_desc()), ctypes.c_void_p(1 << 20 | 8), 1 << 30, ctypes.byref(h))
    assert rc == -3 and "aligned" in lib.rtu_last_error().decode()
    rc = lib.rtu_system_create(ctypes.byref(_desc(n_src=7)), ctypes.c_void_p(1 << 20), 1 << 30, ctypes.byref(h))
    assert rc == -1 and "n_src" in lib.rtu_last_error().decode()


def test_compute_calls_reject_empty_or_null_arguments():
    from paper_2606_30620_b300 import rtu
    lib = rtu._lib
    assert lib.rtu_forward(None, None, 0, None) == 0
    assert lib.rtu_forward(None, None, 2, None) == -1
    assert lib.rtu_version().decode().startswith("rtu-b300")
