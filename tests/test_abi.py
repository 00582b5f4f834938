"""C-ABI checks that need no GPU: the library builds and loads, exports every
entry point declared in include/*.h, and rejects invalid arguments before
touching CUDA."""
import ctypes
import glob
import os
import re

import pytest

import paper_2105_09671_gb300 as ac
from paper_2105_09671_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(ac_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declarations_are_exported():
    lib = ac.lib()
    declared = _declared()
    assert {"ac_create", "ac_step", "ac_energy", "ac_destroy"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    # the binding covers every declared entry point
    assert declared <= set(L.EXPORTED) | {"ac_last_error", "ac_version"}


def test_version():
    assert "sm_103a" in ac.ac_version()


def _desc(**kw):
    base = dict(ndim=2, dtype=ac.AC_F32, nx=64, ny=64, nz=1, pitch_x=64, h=1 / 64, eps=0.015,
                dt=0.1 / 64 / 64)
    base.update(kw)
    return ac.make_desc(**base)


def test_workspace_bytes():
    assert ac.ac_workspace_bytes(_desc()) == 64 * 64 * 4
    assert ac.ac_workspace_bytes(_desc(dtype=ac.AC_F64, pitch_x=66)) == 66 * 64 * 8
    assert ac.ac_workspace_bytes(_desc(ndim=3, nz=5, dtype=ac.AC_F16S, pitch_x=72)) == 72 * 64 * 5 * 2


@pytest.mark.parametrize("bad", [
    dict(ndim=4), dict(ndim=2, nz=3), dict(nx=0), dict(ny=-1), dict(pitch_x=63),
    dict(pitch_x=65),                       # 260 bytes: not a multiple of 16
    dict(dtype=7), dict(h=0.0), dict(eps=-1.0), dict(dt=float("nan")),
    dict(dt=1 / 64 / 64),                   # beyond h^2 / (2 ndim)
    dict(eps=1e-4),                         # dt > eps^2
    dict(nx=1 << 30, pitch_x=1 << 30),
])
def test_invalid_descriptors_rejected(bad):
    with pytest.raises(ac.AcError) as e:
        ac.ac_workspace_bytes(_desc(**bad))
    assert e.value.code == ac.AC_ERR_INVALID
    assert L.last_error()


def test_create_rejects_null_and_misaligned_pointers():
    lib = ac.lib()
    d = _desc()
    out = ctypes.c_void_p()
    assert lib.ac_create(ctypes.byref(d), None, None, None, ctypes.byref(out)) == ac.AC_ERR_INVALID
    assert lib.ac_create(ctypes.byref(d), ctypes.c_void_p(0x1008), ctypes.c_void_p(0x900000),
                         None, ctypes.byref(out)) == ac.AC_ERR_INVALID
    # overlapping phi and workspace
    assert lib.ac_create(ctypes.byref(d), ctypes.c_void_p(0x100000), ctypes.c_void_p(0x100100),
                         None, ctypes.byref(out)) == ac.AC_ERR_INVALID
    assert "overlap" in L.last_error()
    assert out.value is None


def test_null_context_calls_fail_cleanly():
    lib = ac.lib()
    assert lib.ac_step(None, 1) == ac.AC_ERR_INVALID
    assert lib.ac_set_schedule(None, 2, 1) == ac.AC_ERR_INVALID
    assert lib.ac_destroy(None) == ac.AC_OK
    x = ctypes.c_double()
    assert lib.ac_energy(None, ctypes.byref(x)) == ac.AC_ERR_INVALID


def test_struct_layouts_match_the_header(tmp_path):
    # sizeof / offsetof of every public struct, from a C compiler reading
    # include/ac.h, against the ctypes mirrors of the binding
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"ac_grid_desc": L.AcGridDesc, "ac_guard": L.AcGuard, "ac_train_config": L.AcTrainConfig,
               "ac_learned_report": L.AcLearnedReport, "ac_guard_calibration": L.AcGuardCalibration}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ac.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, f"{cname}.{fname}"
