"""The C-ABI library builds for sm_103a, loads, and exports every symbol
that include/chfsi.h declares (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1404_4161_gb300.build import build
    return build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "chfsi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chfsi_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ["chfsi_init", "chfsi_solve", "chfsi_solve_sequence", "chfsi_free",
                 "chfsi_filter", "chfsi_lanczos", "chfsi_orthonormalize",
                 "chfsi_rayleigh_ritz", "chfsi_residuals", "chfsi_degrees"]:
        assert need in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches(libpath):
    from paper_1404_4161_gb300 import _lib
    h = _lib.lib()
    for name in declared_functions():
        assert hasattr(h, name)
    assert set(_lib.exported_names()) == set(declared_functions())
    o = _lib.default_opts()
    assert (o.deg_max, o.deg_extra, o.lanczos_steps) == (36, 1, 20)
    assert _lib.lib().chfsi_strerror(_lib.ENOCONV) == b"not converged within max_loops"


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with the library missing, the binding raises instead
    of computing anything."""
    from paper_1404_4161_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB", str(tmp_path / "libchfsi_missing.so"))
    with pytest.raises(ImportError):
        _lib.lib()


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structs of the binding have the header's sizes and field
    offsets (compiled with the host C compiler, no GPU)."""
    import ctypes as C
    from paper_1404_4161_gb300 import _lib
    structs = {"chfsi_opts": _lib.Opts, "chfsi_stats": _lib.Stats,
               "chfsi_filter_item": _lib.FilterItem, "chfsi_problem": _lib.Problem}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "chfsi.h"', 'int main(void) {']
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)
