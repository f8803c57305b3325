"""The C ABI: libem.so builds, loads and exports every entry point declared in
include/em.h, and the binding's ctypes structures match the header's layout
(checked against a C program compiled with gcc).  No GPU needed."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "em.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(em_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2204_12876_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("em_create", "em_update", "em_shift", "em_get_layers", "em_destroy", "em_update_multi",
                     "em_set_layers", "em_get_stats", "em_sync", "em_status_str"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (em_\w+)$", out, re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert getattr(lib, n)


def test_status_strings_without_gpu(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.em_status_str.restype = ctypes.c_char_p
    assert lib.em_status_str(0) == b"ok"
    assert lib.em_status_str(-1) == b"invalid argument"
    assert lib.em_status_str(-4) == b"timeout"


def test_struct_layout_matches_header(tmp_path, lib_path):
    from paper_2204_12876_gb300 import em
    src = tmp_path / "layout.c"
    structs = {"em_params": em._Params, "em_cloud": em._Cloud, "em_info": em._Info, "em_stats": em._Stats,
               "em_tuning": em._Tuning, "em_server_cfg": em._ServerCfg, "em_result": em._Result,
               "em_server_stats": em._ServerStats, "em_request": em._Request}
    consts = {"EM_OK": em.EM_OK, "EM_ERR_INVALID_ARG": em.EM_ERR_INVALID_ARG, "EM_ERR_OOM": em.EM_ERR_OOM,
              "EM_ERR_CUDA": em.EM_ERR_CUDA, "EM_ERR_TIMEOUT": em.EM_ERR_TIMEOUT,
              "EM_ERR_REJECTED": em.EM_ERR_REJECTED, "EM_ERR_BUSY": em.EM_ERR_BUSY,
              "EM_ERR_CAPACITY": em.EM_ERR_CAPACITY, "EM_SERVE_BATCHED": em.SERVE_BATCHED,
              "EM_SERVE_PLAIN": em.SERVE_PLAIN, "EM_SERVE_RECORD_BYTES": em.SERVE_RECORD_BYTES,
              "EM_BATCH_GRAPH": em.BATCH_GRAPH, "EM_NOALLOC_MAX_CELLS": em.NOALLOC_MAX_CELLS,
              "EM_NOALLOC_MAX_POINTS": em.NOALLOC_MAX_POINTS, "EM_NOALLOC_MAX_CLOUDS": em.NOALLOC_MAX_CLOUDS,
              "EM_F_NORMALS": em.F_NORMALS, "EM_F_SMOOTH": em.F_SMOOTH, "EM_F_INPAINT": em.F_INPAINT,
              "EM_F_MEDIAN": em.F_MEDIAN, "EM_F_GAUSS": em.F_GAUSS, "EM_F_UPPER": em.F_UPPER,
              "EM_F_TRACE": em.F_TRACE, "EM_LAYER_UPPER": em.LAYER_UPPER,
              "EM_LAYER_VARIANCE_NOW": em.LAYER_VARIANCE_NOW}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "em.h"', "int main(void) {"]
    for cname in consts:
        lines.append(f'printf("{cname} %lld\\n", (long long){cname});')
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.rsplit(" ", 1) for line in out if line)
    for cname, v in consts.items():
        assert int(got[cname]) == v, cname
    for cname, py in structs.items():
        assert int(got[f"{cname} size"]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)


def test_product_path_has_no_oracle_dependency():
    """The package never imports the oracle and never falls back to the CPU."""
    pkg = os.path.join(ROOT, "paper_2204_12876_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.replace("the oracle", ""), f


def test_noalloc_binding_checks_layers_before_the_call(lib_path):
    """em.update_noalloc refuses layers the library could not check (wrong
    dtype, element count, contiguity, not on a CUDA device) with ValueError
    before anything reaches the library."""
    torch = pytest.importorskip("torch")
    from paper_2204_12876_gb300 import em
    p = em.Params(width=10, height=8)
    pose = [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0]
    pts = torch.zeros((5, 3))
    ok_f = torch.zeros((8, 10))
    ok_i = torch.zeros((8, 10), dtype=torch.int32)
    bad = [
        (ok_f.double(), ok_f, ok_i, "float32"),            # dtype
        (ok_f, torch.zeros((8, 9)), ok_i, "80 elements"),   # element count
        (ok_f, ok_f, ok_f, "int32"),                       # t_last dtype
        (ok_f, torch.zeros((10, 8)).t(), ok_i, "contiguous"),
    ]
    for h, v, t, what in bad:
        with pytest.raises(ValueError, match=what):
            em.update_noalloc(p, h, v, t, [(pts, pose)], t_now=1)
    with pytest.raises(ValueError, match="nx"):                  # a normal layer of the wrong size
        em.update_noalloc(p, ok_f, ok_f, ok_i, [(pts, pose)], t_now=1,
                          normals=(torch.zeros(3), ok_f, ok_f))
    with pytest.raises(ValueError, match="CUDA"):                # host tensors
        em.update_noalloc(p, ok_f, ok_f, ok_i, [(pts, pose)], t_now=1)


def test_cloud_marshalling_without_gpu(lib_path):
    """The binding's cloud descriptor (em_cloud): pointer, count, stride and the
    row-major 3x4 pose as the library reads them; points that are not
    contiguous float32 and poses that are not 12 numbers are refused."""
    torch = pytest.importorskip("torch")
    np = pytest.importorskip("numpy")
    from paper_2204_12876_gb300 import em
    pts = torch.arange(12, dtype=torch.float32).reshape(4, 3)
    pose = np.arange(12, dtype=np.float64).reshape(3, 4) / 8.0  # converted to float32, row-major
    c = em._cloud_struct(pts, pose, False, any_device=True)
    assert c.points == pts.data_ptr() and c.n == 4 and c.stride == 3
    assert list(c.pose) == [v / 8.0 for v in range(12)]
    c4 = em._cloud_struct(torch.zeros((7, 4)), pose.reshape(12), False, any_device=True)
    assert c4.n == 7 and c4.stride == 4
    with pytest.raises(ValueError):
        em._cloud_struct(pts.double(), pose, False, any_device=True)
    with pytest.raises(ValueError):
        em._cloud_struct(torch.zeros((3, 4)).t(), pose, False, any_device=True)  # not contiguous
    with pytest.raises(ValueError):
        em._pose(np.zeros(11))
