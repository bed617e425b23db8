"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

import paper_1908_05944_gb300 as ac
import importlib

cuda_build = importlib.import_module("paper_1908_05944_gb300.build")

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "alphac.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^AC_API\s+[\w\s\*]+?\b(ac_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return ac.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["ac_create", "ac_create_batch", "ac_build", "ac_get_simplices", "ac_filtration_values",
                     "ac_eval_filtration", "ac_backward", "ac_get_stats", "ac_destroy", "ac_error_string"]:
        assert required in names
    assert sorted(ac.EXPORTS) == names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    out = os.popen(f"nm -D --defined-only {ac.LIB_PATH}").read()
    exported = set(re.findall(r"\bT (ac_\w+)", out))
    assert set(_declared()) <= exported


def test_error_strings_without_gpu(lib):
    assert ac.error_string(0) == "ok"
    for code in range(-8, 0):
        assert ac.error_string(code) != "unknown error"
    assert ac.error_string(-99) == "unknown error"


def test_null_arguments_are_rejected_without_touching_the_gpu(lib):
    assert lib.ac_create(None, None, 0, 0.0, None, None) == ac.AC_ERR_INVALID_ARG
    out = ctypes.c_void_p()
    assert lib.ac_create(None, None, -1, 0.0, None, ctypes.byref(out)) == ac.AC_ERR_INVALID_ARG
    assert not out.value
    assert lib.ac_build(None, None) == ac.AC_ERR_INVALID_ARG
    p = ctypes.c_void_p()
    n = ctypes.c_int64()
    assert lib.ac_get_simplices(None, 0, -1, ctypes.byref(p), ctypes.byref(n)) == ac.AC_ERR_INVALID_ARG
    assert lib.ac_get_stats(None, None) == ac.AC_ERR_INVALID_ARG
    d = ctypes.c_double()
    assert lib.ac_fma_peak(0, 100, None, None, None) == ac.AC_ERR_INVALID_ARG
    assert lib.ac_fma_peak(1, 0, None, ctypes.byref(d), None) == ac.AC_ERR_INVALID_ARG
    lib.ac_destroy(None)
    assert b"NULL" in lib.ac_last_error_detail() or lib.ac_last_error_detail() != b""


def test_stats_struct_layout_matches_header():
    txt = open(HEADER).read()
    body = txt[txt.index("typedef struct {\n    int64_t n_atoms;"):]
    body = body[: body.index("} ac_stats;")]
    fields = re.findall(r"^\s+\w+\s+(\w+)(?:\[\d\])?;", body, flags=re.M)
    assert fields == [f for f, _ in ac.ac_stats._fields_]


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of ac_options, ac_stats and ac_chunked_stats have the C layout: sizes and
    field offsets printed by a program compiled from the header with the system C compiler."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"ac_options": ac.ac_options, "ac_stats": ac.ac_stats, "ac_chunked_stats": ac.ac_chunked_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "alphac.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, key, val = ln.split()
        got[(name, key)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


PLUMBING = {"ac_destroy", "ac_error_string", "ac_last_error_detail", "ac_chunked_free", "ac_get_stats",
            "ac_get_sizes", "ac_chunked_info", "ac_chunked_simplices"}


def test_every_entry_point_cites_its_passage_and_errors():
    """Each declaration of the method's calls cites the paper (a Section or Step), or says the paper
    has none, and states its error behaviour."""
    txt = open(HEADER).read()
    seen = set()
    for m in re.finditer(r"/\*((?:(?!\*/).)*)\*/\s*(AC_API[^;]*;)", txt, re.S):
        com, decl = m.group(1), m.group(2)
        name = re.search(r"\b(ac_\w+)\s*\(", decl).group(1)
        seen.add(name)
        if name in PLUMBING:
            continue
        assert re.search(r"Section|Step|paper has no counterpart|paper gives no", com), f"{name}: no citation"
        assert re.search(r"Errors?:|errors", com), f"{name}: no error behaviour"
    assert seen == set(_declared())
