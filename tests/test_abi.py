"""The C ABI library builds, loads and exports what include/*.h declares (no GPU).

Also checks that the ctypes mirrors of fms_options / fms_stats have the C
layout (sizes and field offsets from a gcc-compiled probe) and exercises the
host-only entry points (strerror, defaults, argument validation).
"""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "fms_libbuild", os.path.join(ROOT, "paper_2112_13891_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    path = b.build()
    return ctypes.CDLL(path)


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(fms_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "fms_cluster" in names and "fms_select_seeds" in names
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (fms_\w+)", out))
    assert set(names) <= exported


def test_struct_layout_matches_c(tmp_path):
    import paper_2112_13891_gb300 as fms
    fields = {"fms_options": fms.FmsOptions, "fms_stats": fms.FmsStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fms.h"', "int main(void){"]
    for cname, cls in fields.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", f"-I{ROOT}/include", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    for line in out.strip().splitlines():
        cname, f, v = line.split()
        cls = fields[cname]
        if f == "sizeof":
            assert ctypes.sizeof(cls) == int(v), (cname, v)
        else:
            assert getattr(cls, f).offset == int(v), (cname, f, v)


def test_host_entry_points(lib):
    lib.fms_strerror.restype = ctypes.c_char_p
    assert lib.fms_strerror(0) == b"ok"
    assert b"max_modes" in lib.fms_strerror(3)
    import paper_2112_13891_gb300 as fms
    o = fms.FmsOptions()
    lib.fms_options_default(ctypes.byref(o))
    assert o.n_initial == 128 and abs(o.L - 8.0) < 1e-7 and abs(o.gamma - 0.95) < 1e-7
    # argument validation happens before any device call
    lib.fms_cluster.restype = ctypes.c_int
    nm = ctypes.c_int32(0)
    rc = lib.fms_cluster(None, ctypes.c_int64(10), 3, ctypes.c_float(1.0), ctypes.c_float(0.0),
                         10, None, None, 0, ctypes.byref(nm), None, None, None,
                         ctypes.c_size_t(0), None, None)
    assert rc == fms.FMS_ERR_INVALID_ARG
    lib.fms_select_seeds.restype = ctypes.c_int
    rc = lib.fms_select_seeds(ctypes.c_int64(10), ctypes.c_uint64(0), ctypes.c_int64(5),
                              ctypes.c_int64(6), None, None)
    assert rc == fms.FMS_ERR_INVALID_ARG
    lib.fms_workspace_size.restype = ctypes.c_size_t
    assert lib.fms_workspace_size(ctypes.c_int64(0), 3, None) == 0
    assert lib.fms_workspace_size(ctypes.c_int64(100), 65, None) == 0
