"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hms.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hms_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("hms_context_create", "hms_problem_create", "hms_solve", "hms_residual",
              "hms_update_residual", "hms_relax", "hms_coarse_matrix", "hms_coarse_solve"):
        assert f in names


def test_library_exports_every_declared_symbol():
    from paper_1208_4093_gb300 import build, capi
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hms_[a-z0-9_]+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    # the binding wraps exactly the declared entry points and loads them
    assert sorted(capi.exported_symbols()) == declared_functions()
    lib = capi.lib()
    for f in declared_functions():
        assert getattr(lib, f) is not None


def test_library_is_built_for_sm_103a():
    from paper_1208_4093_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_no_cpu_fallback_in_binding():
    """The binding only marshals arguments: it never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1208_4093_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "oracle" not in re.sub(r'""".*?"""', "", src, flags=re.S), f


def header_struct_fields(name):
    """(C type, field) of a typedef struct in the header, in order."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = {m.group(2): m.group(1) for m in re.finditer(r"typedef struct \{([^{}]*)\}\s*(\w+)\s*;", text)}[name]
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"((?:const\s+)?\w+\s*\**)\s*(.*)", decl)
        ctype = m.group(1).replace(" ", "")
        for field in m.group(2).split(","):
            field = field.strip()
            star = field.startswith("*")
            out.append((ctype + ("*" if star else ""), field.lstrip("*").strip()))
    return out


@pytest.mark.parametrize("cname,pyname", [("hms_options", "Options"), ("hms_lattice_desc", "LatticeDesc")])
def test_binding_structs_match_the_header(cname, pyname):
    """The ctypes structs the binding passes by pointer have the header's
    fields, in its order and with its sizes (an appended option must reach
    both sides)."""
    import ctypes
    from paper_1208_4093_gb300 import capi
    want = header_struct_fields(cname)
    got = getattr(capi, pyname)._fields_
    assert [n for _, n in want] == [n for n, _ in got]
    size = {"int32_t": ctypes.c_int32, "uint32_t": ctypes.c_uint32, "double": ctypes.c_double}
    for (ctype, n), (_, pytype) in zip(want, got):
        c = ctypes.c_void_p if ctype.endswith("*") else size[ctype]
        assert ctypes.sizeof(c) == ctypes.sizeof(pytype), n
