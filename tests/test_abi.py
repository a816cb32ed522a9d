"""The C-ABI library builds, loads and exports every symbol include/iedd.h declares (no GPU).

Also checks the boundary's host-side argument validation, which returns before any device
work, and that the product path refuses to run without its CUDA library.
"""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "iedd.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_12574_gb300 import iedd
    return iedd.load_library()


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^IEDD_API\s+[\w\s\*]*?\b(\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ie_discretize", "ie_matvec", "dd_partition", "dd_factor", "dd_apply", "pcg_solve"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)


def test_binding_covers_header():
    from paper_2108_12574_gb300 import iedd
    assert sorted(iedd.EXPORTS) == _declared()


def test_version_and_no_error(lib):
    assert b"sm_103a" in lib.ie_version()
    assert lib.ie_last_error() == b""


def test_library_is_built_for_sm_103a(lib):
    # every compile and the link name one target, the sm_103a real architecture (checked on the
    # build commands, not by taking the binary apart)
    from paper_2108_12574_gb300 import build as B
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.samefile(lib._name, B.LIB)


def test_null_arguments_rejected_without_gpu(lib):
    from paper_2108_12574_gb300 import iedd
    # argument checks run before any CUDA call
    assert lib.ie_discretize(4, 8, 0.0, 0, 0, None) == iedd.IE_ERR_ARG
    assert lib.ie_matvec(None, None, None, 1, 1, 1, None) == iedd.IE_ERR_ARG
    assert b"NULL" in lib.ie_last_error()
    assert lib.dd_partition(None, 2, 1, 1, None) == iedd.IE_ERR_ARG
    assert lib.dd_apply(None, None, None, 1, 1, None) == iedd.IE_ERR_ARG
    assert lib.pcg_solve(None, None, None, None, 1, 1, None, None, None) == iedd.IE_ERR_ARG
    lib.ie_destroy(None)
    lib.dd_partition_destroy(None)
    lib.dd_factor_destroy(None)
    assert lib.ie_kernel_launches(0) >= 0


def test_rs_entry_points_reject_null_arguments_without_gpu(lib):
    from paper_2108_12574_gb300 import iedd
    assert lib.dd_factor_rs(None, None, None, None, None) == iedd.IE_ERR_ARG
    assert b"out is NULL" in lib.ie_last_error()
    out = ctypes.c_void_p(1234)
    assert lib.dd_factor_rs(None, None, None, ctypes.byref(out), None) == iedd.IE_ERR_ARG
    assert out.value is None  # *out is cleared before the other checks
    nc = ctypes.c_int(-1)
    assert lib.dd_rs_info(None, ctypes.byref(nc), None, None, None) == iedd.IE_ERR_ARG
    assert nc.value == -1 and b"not an RS factor" in lib.ie_last_error()
    assert lib.dd_rs_export(None, 0, 1, None, None, None, None, None) == iedd.IE_ERR_ARG
    assert lib.ie_fp64_fma_rate(0, None) == iedd.IE_ERR_ARG


def test_default_opts(lib):
    from paper_2108_12574_gb300 import iedd
    o = iedd.pcg_default_opts()
    assert o.tol == 1e-8 and o.max_it == 1000 and o.precision == iedd.IE_MIXED
    assert o.replace_every == 50 and o.check_every == 8 and o.verify == 1
    assert ctypes.sizeof(iedd.PcgReport) == 72


def test_missing_library_fails_loudly(tmp_path):
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2108_12574_gb300 import iedd\n"
            "iedd._LIB = None\n"
            "try:\n"
            "    iedd.load_library(%r)\n"
            "except ImportError as e:\n"
            "    print('IMPORTERROR', e)\n") % (ROOT, str(tmp_path / "nope.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert "IMPORTERROR" in r.stdout


def test_product_path_never_imports_oracle():
    pkg = os.path.join(ROOT, "paper_2108_12574_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "ie_oracle" not in text and "direct_sum" not in text, f


def test_autotune_switch_without_gpu():
    # the autotuner's switch and report touch no device: query, off, on, forget
    from paper_2108_12574_gb300 import iedd
    prev = iedd.ie_autotune(-1)
    assert iedd.ie_autotune(0) == prev
    assert iedd.ie_autotune(-1) is False
    assert iedd.ie_autotune(1) is False
    assert iedd.ie_autotune(-1) is True
    iedd.ie_autotune(2)
    assert iedd.ie_autotune_report() == ""
    iedd.ie_autotune(1 if prev else 0)


C_CALLER = r"""
#include <stdio.h>
#include <string.h>
#include "iedd.h"

int main(void) {
    pcg_opts o;
    pcg_report rep;
    ie_problem *p = NULL;
    memset(&rep, 0, sizeof rep);
    pcg_default_opts(&o);
    if (o.max_it != 1000 || o.replace_every != 50 || o.precision != IE_MIXED) return 2;
    if (strstr(ie_version(), "sm_103a") == NULL) return 3;
    /* host-side argument checks return before any device work */
    if (ie_discretize(5, 8, 0.0, IE_GRID_TEXT, 0, &p) != IE_ERR_ARG || p != NULL) return 4;
    if (pcg_solve(NULL, NULL, NULL, NULL, 1, 1, &o, &rep, NULL) != IE_ERR_ARG) return 5;
    if (dd_apply(NULL, NULL, NULL, 1, 1, NULL) != IE_ERR_ARG) return 6;
    if (ie_last_error()[0] == '\0') return 7;
    ie_destroy(NULL);
    dd_partition_destroy(NULL);
    dd_factor_destroy(NULL);
    ws_destroy(NULL);
    printf("ok %s\n", ie_version());
    return 0;
}
"""


def test_plain_c_caller_builds_links_and_runs(lib, tmp_path):
    # the header is plain C (C99, no C++ or CUDA types) and a C program links the library and
    # calls its host-side entry points; nothing here touches a GPU
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(lib._name)
    cuda_lib = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", str(src),
                        "-I", os.path.join(ROOT, "include"), "-L", libdir, "-liedd",
                        f"-Wl,-rpath,{libdir}", f"-Wl,-rpath-link,{cuda_lib}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, LD_LIBRARY_PATH=cuda_lib + os.pathsep + os.environ.get("LD_LIBRARY_PATH", ""))
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("ok ")
