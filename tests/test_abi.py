"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/drsf.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

import paper_2607_20211_gb300 as drsf

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "drsf.h")


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"DRSF_API\s+[\w\s\*]*?\b(drsf_\w+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("drsf_create", "drsf_apply", "drsf_parent", "drsf_labels", "drsf_stats", "drsf_destroy",
              "drsf_error_string", "drsf_set_allocator"):
        assert n in names


def test_library_exports_every_declared_symbol():
    path = drsf.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_error_strings():
    lib = drsf.library()
    for s in range(7):
        assert lib.drsf_error_string(s)


@pytest.mark.parametrize("c_name, py_struct", [("drsf_batch_stats", drsf.BatchStats),
                                               ("drsf_batched_class", drsf.BatchedClass),
                                               ("drsf_profile_t", drsf.Profile)])
def test_struct_layout_matches_the_header(tmp_path, c_name, py_struct):
    """The binding's ctypes structs have the header's size and field offsets
    (checked by a C program compiled against include/drsf.h)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in py_struct._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"drsf.h\"\nint main(void) {\n"
                   f"  printf(\"%zu\\n\", sizeof({c_name}));\n" +
                   "".join(f"  printf(\"%zu\\n\", offsetof({c_name}, {f}));\n" for f in fields) + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got[0] == ctypes.sizeof(py_struct)
    assert got[1:] == [getattr(py_struct, f).offset for f in fields]
