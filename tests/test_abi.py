"""The C-ABI library builds, loads without a GPU and exports every function
declared in include/ck.h (no compute calls here)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ck_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ck_load_mechanism", "ck_free_mechanism", "ck_rhs", "ck_jacobian", "ck_integrate_ros4",
                 "ck_integrate_rkf45", "ck_lu_factor", "ck_lu_solve", "ck_count_work", "ck_status_str"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1608_05794_gb300.build import build
    lib = build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = sorted(_declared() - exported)
    assert not missing, missing
    dll = ctypes.CDLL(lib)
    for name in _declared():
        getattr(dll, name)


def test_binding_loads_and_reports_version():
    import paper_1608_05794_gb300.ck as ck
    assert "sm_103a" in ck.version()
    assert ck.library_path().endswith("libck.so")


def test_header_is_plain_c_and_a_c_program_links(tmp_path):
    # the boundary is a C ABI: the header compiles as C99, and a C program
    # links against the library and calls the entry points that need no GPU
    from paper_1608_05794_gb300.build import build
    lib = build()
    src = tmp_path / "use_ck.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "ck.h"
int main(void) {
  ck_solver_opts o;
  ck_default_opts(&o);
  if (!(o.rtol == 1e-9 && o.atol == 1e-12 && o.max_steps == 100000 && o.precision == 0 && o.jac == 0)) return 1;
  if (strcmp(ck_status_str(CK_OK), "ok") != 0) return 2;
  if (ck_lu_factor(1, 0, 0, 0, 0, 0) != CK_ERANGE) return 3;
  if (ck_load_mechanism(0, 0) != CK_EINVAL) return 4;
  printf("%s\n", ck_version());
  return 0;
}
""")
    exe = tmp_path / "use_ck"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), lib,
                    "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert "sm_103a" in out.stdout
