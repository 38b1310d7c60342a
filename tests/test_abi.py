"""The C ABI library on the CPU: it loads without a GPU, exports exactly the
symbols include/q4c.h declares, and rejects bad arguments with the
documented status codes before touching the device."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2608_00773_gb300 as q
from paper_2608_00773_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2608_00773_gb300 import _build
    _build.build()
    return q.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "q4c.h")).read()
    return sorted(set(re.findall(r"Q4C_API\s+[\w\s\*]+?\b(\w+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("nao_tabulate", "grid_partition", "q4c_integrate", "q4c_density", "q4c_integrate_backward"):
        assert must in names
    assert sorted(B.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", q.LIB_PATH], capture_output=True, text=True).stdout
    exported = sorted(l.split()[-1] for l in out.splitlines() if " T " in l)
    assert exported == declared_symbols()
    for n in declared_symbols():
        assert getattr(lib, n) is not None


def test_library_targets_sm103a(lib):
    # the build flags name exactly one architecture
    from paper_2608_00773_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_codes_on_bad_arguments(lib):
    h = C.c_void_p()
    # NULL descriptor
    assert lib.nao_tabulate(None, C.byref(h)) == 1
    # bad radii: r_on > r_cut
    n_rad = np.array([1], np.int32); l = np.array([0], np.int32); a = np.array([1.0])
    d = B.BasisDesc(1, n_rad.ctypes.data, l.ctypes.data, a.ctypes.data, 5.0, 6.0, 1e-4, 200)
    assert lib.nao_tabulate(C.byref(d), C.byref(h)) == 1
    assert b"r_min < r_on < r_cut" in lib.q4c_last_error()
    # l > 4 is outside what the kernels expand
    l5 = np.array([5], np.int32)
    d = B.BasisDesc(1, n_rad.ctypes.data, l5.ctypes.data, a.ctypes.data, 6.0, 5.0, 1e-4, 200)
    assert lib.nao_tabulate(C.byref(d), C.byref(h)) == 5
    # too few knots, negative exponent
    d = B.BasisDesc(1, n_rad.ctypes.data, l.ctypes.data, a.ctypes.data, 6.0, 5.0, 1e-4, 3)
    assert lib.nao_tabulate(C.byref(d), C.byref(h)) == 1
    neg = np.array([-1.0])
    d = B.BasisDesc(1, n_rad.ctypes.data, l.ctypes.data, neg.ctypes.data, 6.0, 5.0, 1e-4, 200)
    assert lib.nao_tabulate(C.byref(d), C.byref(h)) == 1
    # compute calls with NULL handles
    m = B.Matrices(0, 0, 0, 0, 0, 0)
    assert lib.q4c_integrate(None, None, None, 0, C.byref(m), None) == 1
    assert lib.q4c_density(None, None, None, 0, None, None) == 1
    assert lib.q4c_integrate_backward(None, None, C.byref(m), 0, None, None) == 1
    assert lib.grid_partition(None, None, C.byref(h)) == 1
    info = B.GridInfo()
    assert lib.q4c_grid_get_info(None, C.byref(info)) == 1
    # knot-value tables without knots, kappa selection and spinor counts without handles
    assert lib.nao_tabulate_knots(C.byref(d), None, C.byref(h)) == 1
    assert lib.q4c_tables_set_kappa(None, None) == 1
    n = C.c_int64()
    assert lib.q4c_spinor_nnz(None, None, C.byref(n)) == 1


def test_no_device_fails_loudly(lib):
    """Without a GPU the first device allocation fails with Q4C_ECUDA/ENOMEM and
    a message; nothing falls back to the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(q.Q4CError) as e:
        q.nao_tabulate([1], [0], [1.0])
    assert e.value.status in (2, 3)


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/q4c.h compiles as C99 (-pedantic-errors) and a C program links
    against the library and gets EINVAL plus a message for a NULL descriptor;
    no device call."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2608_00773_gb300 import binding
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "abi.c"
    src.write_text(
        "#include <stdio.h>\n#include \"q4c.h\"\n"
        "int main(void) {\n"
        "  q4c_tables* t = NULL;\n"
        "  q4c_status st = nao_tabulate(NULL, &t);\n"
        "  const char* msg = q4c_last_error();\n"
        "  printf(\"%d %s\\n\", (int)st, msg);\n"
        "  return (st == Q4C_EINVAL && t == NULL && msg && msg[0]) ? 0 : 1;\n"
        "}\n")
    exe = tmp_path / "abi"
    libdir = os.path.dirname(binding.LIB_PATH)
    subprocess.run([gcc, "-std=c99", "-pedantic-errors", "-Wall", "-Werror", "-I", os.path.join(root, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-lq4c", "-Wl,-rpath," + libdir], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr

