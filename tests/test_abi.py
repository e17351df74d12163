"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/dock.h declares; the binding declares the same set; the
product code never reaches the oracle.  No compute call is made here."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dock.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"^\s*(?:const\s+)?(?:int|void|char|int64_t)\s*\*?\s*(\w+)\s*\(", src, flags=re.M))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("load_grids", "load_ligand", "dock", "score_batch", "score_grad_batch", "dock_create"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2203_02096_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2203_02096_gb300 import capi
    assert set(capi.SIGNATURES) == _declared()


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2203_02096_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
                assert "liboracle" not in text and "oracle.c" not in text, f


def test_binding_structs_match_the_header(tmp_path):
    """dock_params and dock_allocator: the binding's ctypes layout (size and
    every field offset) is the C compiler's."""
    import subprocess
    from paper_2203_02096_gb300 import capi
    checks = [("dock_params", capi.DockParams), ("dock_allocator", capi.DockAllocator)]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dock.h"', "int main(void) {"]
    for cname, cls in checks:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for _, cls in checks:
        want.append(ctypes.sizeof(cls))
        want += [getattr(cls, f[0]).offset for f in cls._fields_]
    assert got == want
