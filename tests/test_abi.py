"""The C-ABI library builds, loads, and exports every entry point the header declares.

No compute calls here (no GPU needed): symbol presence, struct layout of the
ctypes mirror against the C compiler's own layout, and status strings.
"""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "krr.h")


@pytest.fixture(scope="module")
def lib_path():
    from paper_1611_03220_gb300 import build
    return build()


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(krr_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_entry_points():
    names = _declared()
    for must in ("krr_rff_features", "krr_kernel_matvec", "krr_precond_setup", "krr_precond_apply",
                 "krr_pcg_solve", "krr_predict", "krr_create", "krr_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s+(krr_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for n in _declared():
        assert hasattr(lib, n)


def test_binding_covers_every_symbol(lib_path):
    from paper_1611_03220_gb300 import _krr
    assert set(_declared()) <= set(_krr.EXPORTED)


def test_status_strings_without_gpu(lib_path):
    from paper_1611_03220_gb300 import _krr
    for code in range(10):
        s = _krr._lib.krr_status_string(code).decode()
        assert s and s != "unknown status"
    o = _krr.default_opts()
    assert o.tol == 1e-6 and o.max_iter == 1000 and o.precond == 1 and o.use_graph == 1


def test_struct_layout_matches_c_compiler(lib_path):
    """The ctypes mirrors of krr_opts / krr_report / krr_problem have the C layout."""
    from paper_1611_03220_gb300 import _krr
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "krr.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(krr_opts), offsetof(krr_opts, inner_tol),
         offsetof(krr_opts, warm_start), offsetof(krr_opts, fuse_step), sizeof(krr_report),
         offsetof(krr_report, rel_res), offsetof(krr_report, ms_total));
  printf("%zu %zu\n", offsetof(krr_report, kappa), offsetof(krr_report, rel_res_rec));
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(krr_problem), offsetof(krr_problem, sigma),
         offsetof(krr_problem, s), offsetof(krr_problem, Y), offsetof(krr_problem, C),
         offsetof(krr_problem, ldc));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "l.c")
        exe = os.path.join(td, "l")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True,
                                               check=True).stdout.split()]
    O, R, P = _krr.krr_opts, _krr.krr_report, _krr.krr_problem
    assert vals == [ctypes.sizeof(O), O.inner_tol.offset, O.warm_start.offset,
                    O.fuse_step.offset, ctypes.sizeof(R), R.rel_res.offset,
                    R.ms_total.offset, R.kappa.offset, R.rel_res_rec.offset,
                    ctypes.sizeof(P), P.sigma.offset, P.s.offset, P.Y.offset, P.C.offset,
                    P.ldc.offset]
