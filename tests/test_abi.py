"""The C-ABI library builds, loads and exports every entry point that
include/mmcq.h declares; the Python binding declares the same names.  No
compute call is made (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(mmcq_\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def libpath():
    from paper_2410_00966_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for n in ["mmcq_create", "mmcq_set_cavity", "mmcq_step", "mmcq_get_m", "mmcq_get_cavity"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mmcq_\w+)", out))
    assert set(_declared()) <= exported


def test_binding_covers_the_abi(libpath):
    import paper_2410_00966_gb300 as pkg
    assert sorted(pkg.PROTOTYPES) == _declared()
    lib = pkg.load_library(libpath)
    assert lib.mmcq_last_error(None) == b"null handle"


def test_bad_arguments_are_rejected_without_a_gpu(libpath):
    import paper_2410_00966_gb300 as pkg
    lib = pkg.load_library(libpath)
    h = ctypes.c_void_p()
    g = pkg.mmcq_grid(0, 4, 4, 1e-9, 1e-9, 1e-9, 1)
    assert lib.mmcq_create(ctypes.byref(h), ctypes.byref(g), 8e5, 1e-11, 0.01, 0.0, None, None) == pkg.MMCQ_ERR_ARG
    g = pkg.mmcq_grid(4, 4, 4, -1e-9, 1e-9, 1e-9, 1)
    assert lib.mmcq_create(ctypes.byref(h), ctypes.byref(g), 8e5, 1e-11, 0.01, 0.0, None, None) == pkg.MMCQ_ERR_ARG
    assert not h.value
    assert lib.mmcq_step(None, 1, 1e-13) == pkg.MMCQ_ERR_ARG
    assert lib.mmcq_sync(None) == pkg.MMCQ_ERR_ARG


def test_missing_library_fails_loudly(tmp_path):
    import paper_2410_00966_gb300 as pkg
    with pytest.raises(ImportError):
        pkg.load_library(str(tmp_path / "nope.so"))


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    of the C struct of the same name, as a C compiler lays it out from
    include/mmcq.h (a field added on one side only fails here)."""
    import shutil
    import paper_2410_00966_gb300 as pkg
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [getattr(pkg, n) for n in ("mmcq_grid", "mmcq_opts", "mmcq_cavity", "mmcq_info",
                                         "mmcq_objective", "mmcq_tuning", "mmcq_kernel_stat")]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "mmcq.h"', 'int main(void) {']
    for S in structs:
        n = S.__name__
        lines.append(f'    printf("{n} size %zu\\n", sizeof({n}));')
        for f, _ in S._fields_:
            lines.append(f'    printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line.strip()}
    for S in structs:
        n = S.__name__
        assert got[(n, "size")] == ctypes.sizeof(S), n
        for f, _ in S._fields_:
            assert got[(n, f)] == getattr(S, f).offset, (n, f)
