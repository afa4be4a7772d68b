"""The C-ABI library builds, loads and exports every symbol declared in
include/*.h (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(inc, fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(rve_\w+)\s*\(", src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2207_10657_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["rve_create", "rve_set_state", "rve_hessp", "rve_energy_grad", "rve_solve_step",
                     "rve_destroy", "rve_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_2207_10657_gb300 import binding
    assert set(_declared_functions()) <= set(binding.EXPORTED)
    binding.lib()


def test_default_opts_and_argument_errors(libpath):
    """Host-side paths that need no GPU: defaults and argument validation."""
    from paper_2207_10657_gb300 import binding as B
    o = B.rve_default_opts()
    assert o.restart_thr == 0.2 and o.precision == 32 and o.max_nr == 50 and o.hessian == 0 and o.passes == 0
    lib = B.lib()
    h = ctypes.c_void_p()
    dims = (ctypes.c_int * 3)(7, 8, 8)  # odd size is rejected before any CUDA call
    ph = (B.rve_phase * 1)(B.rve_phase(1.0, 0.3, 0, 0.0, 0.0))
    st = lib.rve_create(dims, 3, ctypes.c_void_p(16), ph, 1, None, None, ctypes.byref(h))
    assert st == -1 and not h.value
    assert "even" in lib.rve_last_error(None).decode()
    dims = (ctypes.c_int * 3)(8, 8, 14)  # prime factor 7
    assert lib.rve_create(dims, 3, ctypes.c_void_p(16), ph, 1, None, None, ctypes.byref(h)) == -1
    dims = (ctypes.c_int * 3)(8, 8, 8)
    bad = (B.rve_phase * 1)(B.rve_phase(1.0, 0.3, 1, 1e-3, 1e-4))  # kappaf < kappa0
    assert lib.rve_create(dims, 3, ctypes.c_void_p(16), bad, 1, None, None, ctypes.byref(h)) == -1
    assert lib.rve_create(dims, 4, ctypes.c_void_p(16), ph, 1, None, None, ctypes.byref(h)) == -1
    lib.rve_destroy(None)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of rve_phase, rve_solver_opts and rve_step_report
    have the C sizes and field offsets (a host C program compiled against
    include/rve.h prints them)."""
    import shutil
    import subprocess
    from paper_2207_10657_gb300 import binding as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = {"rve_phase": B.rve_phase, "rve_solver_opts": B.rve_solver_opts, "rve_step_report": B.rve_step_report,
              "rve_cg_report": B.rve_cg_report}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rve.h"', "int main(void) {"]
    for s, cls in fields.items():
        lines.append(f'  printf("{s} %zu\\n", sizeof({s}));')
        for name, _ in cls._fields_:
            lines.append(f'  printf("{s}.{name} %zu\\n", offsetof({s}, {name}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.split("\n") if l)
    for s, cls in fields.items():
        assert int(out[s]) == ctypes.sizeof(cls), s
        for name, _ in cls._fields_:
            assert int(out[f"{s}.{name}"]) == getattr(cls, name).offset, (s, name)
