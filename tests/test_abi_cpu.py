"""The C ABI library builds, loads and exports every function include/tacta.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

import paper_2304_12168_gb300 as tacta
from paper_2304_12168_gb300 import build as tbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tacta.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(tacta.LIB_PATH):
        tbuild.build()
    return tacta.load_library()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:tacta_status|void|const char\*|int32_t|double)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("cta_solve", "ta_solve", "ta_minnorm", "tacta_plan_create", "tacta_plan_destroy",
                 "tacta_last_error"):
        assert want in names
    assert set(names) == set(tacta.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_struct_layouts_match_header(lib):
    # defaults come from the library itself; a layout mismatch would scramble them
    o = tacta.tacta_options()
    lib.tacta_default_options(ctypes.byref(o))
    assert o.tol == 1e-10 and o.tol_normal == -1.0 and o.max_iter == 1000
    assert o.t_max == 5 and o.cycle == 0 and o.recompute_every == 40 and o.use_graph == 1
    assert o.poll_every == 64 and o.stream is None
    assert o.precision == 0 and o.nonneg == 0 and o.enhanced == 0 and o.fused_chain == 1
    assert o.wait_limit_log2 == 0
    assert o.rho_max == 0.0 and o.profile == 0
    assert lib.tacta_version() == 10000
    assert lib.tacta_last_error() == b""


def test_invalid_arguments_are_rejected_before_gpu_work(lib):
    # argument checks run on the host before any CUDA call, so they work without a GPU
    info = tacta.tacta_info()
    st = lib.cta_solve(None, None, None, None, None, None, 0, ctypes.byref(info))
    assert st == -1 and b"NULL" in lib.tacta_last_error()
    M = tacta.tacta_matrix(0, 5, 0, 1, 0, None, None, None)
    st = lib.cta_solve(ctypes.byref(M), None, None, None, None, None, 0, ctypes.byref(info))
    assert st == -1 and b"m >= 1" in lib.tacta_last_error()
    M = tacta.tacta_matrix(3, 5, 0, 7, 0, 1, None, None)
    st = lib.cta_solve(ctypes.byref(M), None, None, None, None, None, 0, ctypes.byref(info))
    assert st == -1 and b"format" in lib.tacta_last_error()


def test_product_path_refuses_to_run_without_library(tmp_path, monkeypatch):
    import importlib
    monkeypatch.setattr(tacta, "_lib_handle", None)
    with pytest.raises(RuntimeError, match="missing"):
        tacta.load_library(str(tmp_path / "libtacta.so"))
    importlib.reload(tacta)


def test_ctypes_layouts_match_the_c_header(tmp_path):
    """Compile a probe against include/tacta.h with gcc and compare sizes and offsets."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = {"tacta_matrix": tacta.tacta_matrix, "tacta_options": tacta.tacta_options,
               "tacta_info": tacta.tacta_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tacta.h"', "int main(void){"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} %zu\\n", sizeof({sname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{sname}.{f} %zu\\n", offsetof({sname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(l.split() for l in out if l.strip())
    for sname, cls in structs.items():
        assert int(got[sname]) == ctypes.sizeof(cls), sname
        for f, _ in cls._fields_:
            assert int(got[f"{sname}.{f}"]) == getattr(cls, f).offset, f"{sname}.{f}"


def test_batch_arguments_are_rejected_before_gpu_work(lib):
    """tacta_batch_create / tacta_batch_cta validate on the host before any CUDA call."""
    i32 = ctypes.c_int32
    out = ctypes.c_void_p()
    m = (i32 * 2)(3, 0)
    n = (i32 * 2)(4, 5)
    vals = (ctypes.c_double * 32)()
    st = lib.tacta_batch_create(2, m, n, ctypes.cast(vals, ctypes.c_void_p), 0, 1, None, ctypes.byref(out))
    assert st == -1 and b"system 1" in lib.tacta_batch_last_error() and not out.value
    m2 = (i32 * 1)(3)
    n2 = (i32 * 1)(4)
    st = lib.tacta_batch_create(1, m2, n2, ctypes.cast(vals, ctypes.c_void_p), 0, 7, None, ctypes.byref(out))
    assert st == -1 and b"storage" in lib.tacta_batch_last_error()
    st = lib.tacta_batch_create(-1, None, None, None, 0, 1, None, ctypes.byref(out))
    assert st == -1 and b"count" in lib.tacta_batch_last_error()
    st = lib.tacta_batch_cta(None, None, None, None, None, None, None)
    assert st == -1 and b"NULL" in lib.tacta_batch_last_error()
    t, p = ctypes.c_int32(), ctypes.c_int32()
    assert lib.tacta_batch_num_configs() >= 1
    assert lib.tacta_batch_config_shape(0, ctypes.byref(t), ctypes.byref(p)) == 0 and t.value > 0 and p.value > 0
    assert lib.tacta_batch_config_shape(99, ctypes.byref(t), ctypes.byref(p)) == -1
    assert lib.tacta_batch_set_wide(None, -1, 0, 0) == -1
    assert lib.tacta_batch_wide_plan(None, None, None, None, None, None) == -1
