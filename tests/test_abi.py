"""The C-ABI library builds, loads without a GPU and exports every function
that include/mrpt.h declares; the Python binding mirrors those names.  No
compute call is made here."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mrpt.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mrpt_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1509_06957_gb300 import build
    return build.build_library()


def test_header_declares_the_boundary():
    fns = declared_functions()
    for name in ("mrpt_build", "mrpt_query", "mrpt_free", "mrpt_last_error"):
        assert name in fns


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (mrpt_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_mirrors_abi(lib_path):
    import paper_1509_06957_gb300 as mr
    assert set(mr.ABI_SYMBOLS) == set(declared_functions())
    for name in ("mrpt_build", "mrpt_query", "mrpt_query_ex", "mrpt_free", "mrpt_last_error",
                 "mrpt_set_stream", "mrpt_sync", "mrpt_info", "mrpt_export"):
        assert callable(getattr(mr, name))
    lib = mr.load_library()
    assert mr.mrpt_last_error() == ""
    # argument checks run before any device work, so they work without a GPU
    h = ctypes.c_void_p()
    rc = lib.mrpt_build(None, 10, 4, 1, 1, 0.5, 0, ctypes.byref(h))
    assert rc == mr.MRPT_ERR_INVALID_ARG
    assert "invalid argument" in mr.mrpt_last_error()


def _py_imports(path):
    import ast
    tree = ast.parse(open(path).read())
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            mods.add(node.module.split(".")[0])
    return mods


def test_oracle_and_library_share_nothing():
    """The oracle and the CUDA library are independent: neither includes,
    imports or links the other."""
    pkg = os.path.join(ROOT, "paper_1509_06957_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                assert "oracle" not in _py_imports(path), path
            elif f.endswith((".cu", ".cuh", ".h")):
                incs = re.findall(r'#include\s+[<"]([^>"]+)', open(path).read())
                assert not any("oracle" in i for i in incs), path
    assert "paper_1509_06957_gb300" not in _py_imports(os.path.join(ROOT, "oracle", "__init__.py"))
    otext = open(os.path.join(ROOT, "oracle", "mrpt_oracle.c")).read()
    assert not any("mrpt.h" in i or "csrc" in i
                   for i in re.findall(r'#include\s+[<"]([^>"]+)', otext))


def test_every_entry_point_cites_its_passage():
    """Each declaration in include/mrpt.h is documented with the passage of
    the paper it implements (Sec., Algorithm or Table), or says that the
    paper has no counterpart.  Declarations that follow one another with no
    comment between them share the comment above the first."""
    text = open(HEADER).read()
    cite = re.compile(r"Sec\.|Algorithm|Table|no\s+(?:\*\s+)?counterpart")
    pos, documented, seen = 0, False, []
    for m in re.finditer(r"^(?:int|const char|int64_t)\s*\*?\s*(mrpt_\w+)\s*\(", text, flags=re.M):
        region = text[pos:m.start()]
        if "/*" in region:
            documented = bool(cite.search(region))
        assert documented, f"{m.group(1)}: no citation and no 'no counterpart' in its comment"
        seen.append(m.group(1))
        pos = m.end()
    assert set(seen) == set(declared_functions())


def _c_layout(tmp_path, structs, macros):
    """Compile a probe against include/mrpt.h with the host C compiler and
    read back sizeof/offsetof of each struct field and the macro values."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mrpt.h"', "int main(void) {"]
    for cname, fields in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    for mname in macros:
        lines.append(f'  printf("macro {mname} %lld\\n", (long long)({mname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for ln in out.splitlines():
        a, b, c = ln.split()
        got[(a, b)] = int(c)
    return got


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes mirrors of mrpt_build_opts, mrpt_query_opts and
    mrpt_index_info have the C structs' field names, offsets and sizes, and
    the binding's constants equal the header's macros: the C ABI passes these
    structs and codes by layout and value only."""
    import paper_1509_06957_gb300 as mr
    mirrors = {"mrpt_build_opts": mr.BuildOpts, "mrpt_query_opts": mr.QueryOpts,
               "mrpt_index_info": mr.IndexInfo}
    structs = {c: [f[0] for f in py._fields_] for c, py in mirrors.items()}
    macros = [n for n in dir(mr) if n.startswith("MRPT_") and isinstance(getattr(mr, n), int)]
    got = _c_layout(tmp_path, structs, macros)
    for cname, py in mirrors.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for f in structs[cname]:
            assert got[(cname, f)] == getattr(py, f).offset, f"{cname}.{f}"
    for n in macros:
        assert got[("macro", n)] == getattr(mr, n), n
