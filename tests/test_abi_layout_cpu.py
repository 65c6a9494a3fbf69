"""CPU checks that the ctypes binding and include/hgf.h describe the same ABI.

A mismatch between the two (a field added to a struct on one side only, an argument missing from a
ctypes signature, an enumerator renumbered) would not fail at load time: ctypes would pass garbage
or read the wrong bytes. These tests compile a small C program against the header with the host C
compiler and compare, for every struct the binding mirrors, its size and each field's offset and
size; for every enumerator, its value; and for every declared function, its parameter and return
kinds (pointer, 32-bit int, 64-bit unsigned, double) against the ctypes signature."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hgf.h")


def header_source(strip_comments=True):
    src = open(HEADER).read()
    if strip_comments:
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
    return src


def binding_structs():
    from paper_1803_00005_gb300 import hgf
    return {name: getattr(hgf, name) for name in
            ("hgf_params", "hgf_cost_params", "hgf_tuning", "hgf_request", "hgf_job",
             "hgf_serve_stats_t")}


def enumerators():
    names = []
    for body in re.findall(r"typedef\s+enum\s*\{(.*?)\}", header_source(), flags=re.S):
        names += re.findall(r"\b(HGF_[A-Z0-9_]+)\b", body)
    return names


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hgf.h"', "int main(void) {"]
    for sname, cls in binding_structs().items():
        lines.append(f'  printf("size {sname} %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("field {sname} {fname} %zu %zu\\n", offsetof({sname}, {fname}),'
                         f' sizeof((({sname} *)0)->{fname}));')
    for e in enumerators():
        lines.append(f'  printf("enum {e} %d\\n", (int){e});')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    sizes, fields, enums = {}, {}, {}
    for line in out.splitlines():
        kind, *rest = line.split()
        if kind == "size":
            sizes[rest[0]] = int(rest[1])
        elif kind == "field":
            fields[(rest[0], rest[1])] = (int(rest[2]), int(rest[3]))
        else:
            enums[rest[0]] = int(rest[1])
    return sizes, fields, enums


def test_struct_layouts_match_header(c_layout):
    sizes, fields, _ = c_layout
    for sname, cls in binding_structs().items():
        assert ctypes.sizeof(cls) == sizes[sname], sname
        for fname, ftype in cls._fields_:
            off, size = fields[(sname, fname)]
            assert getattr(cls, fname).offset == off, (sname, fname)
            assert ctypes.sizeof(ftype) == size, (sname, fname)


def test_enumerators_match_header(c_layout):
    from paper_1803_00005_gb300 import hgf
    _, _, enums = c_layout
    assert len(enums) >= 20
    for name, value in enums.items():
        assert getattr(hgf, name) == value, name


def _c_kind(decl):
    """Kind of one C parameter or return type: 'ptr', 'i32', 'u64' or 'f64'."""
    decl = " ".join(decl.split())
    if "*" in decl:
        return "ptr"
    toks = decl.replace("const ", "").split()
    ty = " ".join(toks[:-1]) if len(toks) > 1 else toks[0]
    if ty in ("int", "int32_t", "hgf_status") or (ty.startswith("hgf_") and ty in ENUM_TYPES):
        return "i32"
    if ty in ("size_t", "uint64_t", "unsigned long long"):
        return "u64"
    if ty == "double":
        return "f64"
    raise AssertionError(f"unclassified C type in {decl!r}")


ENUM_TYPES = set(re.findall(r"typedef\s+enum\s*\{.*?\}\s*(hgf_[a-z_]+)\s*;", header_source(),
                            flags=re.S))


def _ctypes_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(t, type) and
                                                    issubclass(t, ctypes._Pointer)):
        return "ptr"
    if t is ctypes.c_int:
        return "i32"
    if t in (ctypes.c_uint64, ctypes.c_size_t, ctypes.c_ulonglong):
        return "u64"
    if t is ctypes.c_double:
        return "f64"
    raise AssertionError(f"unclassified ctypes type {t!r}")


def declared_functions():
    out = {}
    for ret, name, args in re.findall(r"([A-Za-z_][A-Za-z0-9_ ]*?\**)\s*\b(hgf_[a-z_0-9]+)\s*\("
                                      r"([^;{)]*)\)\s*;", header_source()):
        params = [a for a in (x.strip() for x in args.split(",")) if a and a != "void"]
        out[name] = (_c_kind(ret + " r"), [_c_kind(p) for p in params])
    return out


def test_function_signatures_match_header():
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    lib = hgf.lib()
    decl = declared_functions()
    assert sorted(decl) == sorted(hgf.EXPORTED)
    for name, (ret, params) in decl.items():
        f = getattr(lib, name)
        assert f.argtypes is not None, f"{name} has no ctypes signature"
        assert [_ctypes_kind(t) for t in f.argtypes] == params, name
        assert _ctypes_kind(f.restype) == ret, name
