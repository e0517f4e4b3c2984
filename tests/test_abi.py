"""The C-ABI library builds, loads and exports every function include/rbf.h declares;
the Python binding declares exactly those; host-side argument checks need no GPU."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rbf.h")


def _header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:rbf_status|int|const char\s*\*)\s+(rbf_\w+)\s*\(",
                                 text, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1806_07884_gb300 import build as b
    if not os.path.exists(b.LIB):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build librbf")
        b.build()
    return b.LIB


def test_header_declares_the_pipeline():
    names = _header_functions()
    for required in ("rbf_bin", "rbf_assemble", "rbf_solve", "rbf_eval"):
        assert required in names


def test_library_exports_every_header_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(libpath):
    from paper_1806_07884_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == _header_functions()
    lib = _lib.load(libpath)
    assert lib.rbf_max_candidates() >= 128


def test_status_codes_match_header():
    from paper_1806_07884_gb300 import _lib
    text = open(HEADER).read()
    for name, code in re.findall(r"(RBF_\w+)\s*=\s*(\d+)", text):
        if name in _lib.STATUS_NAMES.values():
            assert _lib.STATUS_NAMES[int(code)] == name


def test_missing_library_fails_loudly(tmp_path):
    from paper_1806_07884_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "librbf.so"))
    finally:
        _lib._lib = saved


def test_null_arguments_rejected_without_gpu(libpath):
    from paper_1806_07884_gb300 import _lib
    lib = _lib.load(libpath)
    box = (ctypes.c_double * 4)(0, 0, 1, 1)
    assert lib.rbf_bin(None, None, None, 1, None, None, None, 1, 0.1, box, None) == _lib.RBF_ERR_ARG
    assert lib.rbf_assemble(None, 1, 0, None) == _lib.RBF_ERR_ARG
    assert lib.rbf_destroy(None) == _lib.RBF_ERR_ARG
    out = ctypes.c_void_p()
    nullf = ctypes.cast(None, _lib.ALLOC_FN)
    nullfree = ctypes.cast(None, _lib.FREE_FN)
    assert lib.rbf_create(None, 0, nullf, nullfree, None) == _lib.RBF_ERR_ARG
    # bad device index: rejected without touching a GPU
    assert lib.rbf_create(ctypes.byref(out), 1 << 20, nullf, nullfree, None) != 0


def test_struct_layouts_match_the_binding(tmp_path):
    """Size and field offsets of every struct in include/rbf.h, as a C compiler lays them out,
    equal those of the ctypes mirrors the binding passes to the library."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1806_07884_gb300 import _lib
    mirrors = {"rbf_solve_info": _lib.SolveInfo, "rbf_tile": _lib.Tile, "rbf_tile_info": _lib.TileInfo,
               "rbf_layout_stats": _lib.LayoutStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rbf.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    r = subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            name, key, val = line.split()
            got[(name, key)] = int(val)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def _ctx_functions():
    """Header functions whose first parameter is the context."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*rbf_status\s+(rbf_\w+)\s*\(\s*(?:const\s+)?rbf_ctx\s*\*\s*ctx\b",
                                 text, flags=re.M)))


def test_every_context_call_rejects_a_null_context(libpath):
    """Every entry point that takes a context returns RBF_ERR_ARG for a null one (other
    pointers null, numbers zero) before touching a GPU."""
    from paper_1806_07884_gb300 import _lib
    lib = _lib.load(libpath)
    names = _ctx_functions()
    assert "rbf_solve_tiles" in names and "rbf_warm_start" in names and len(names) >= 20
    for name in names:
        args = []
        for t in _lib.SIGNATURES[name][1]:
            if t in (ctypes.c_double, ctypes.c_float):
                args.append(0.0)
            elif t in (ctypes.c_int, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32):
                args.append(0)
            else:
                args.append(None)
        assert getattr(lib, name)(*args) == _lib.RBF_ERR_ARG, name
    assert lib.rbf_last_error(None) is not None


def test_context_free_calls_reject_bad_arguments(libpath):
    from paper_1806_07884_gb300 import _lib
    lib = _lib.load(libpath)
    assert lib.rbf_selftest_sqrt(None, None, 5, None) == _lib.RBF_ERR_ARG
    assert lib.rbf_eval_noalloc(None, None, None, 1, 0.1, None, 1, None, None, 0, None, None) \
        == _lib.RBF_ERR_ARG
