"""ie_matvec_noalloc's argument checks on the host (no GPU): a C++ program compiled by g++
includes the CUDA-free header that decides every rejection and prints the verdict for a table
of cases, among them memory and streams of another device, which a one-GPU machine cannot make.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2108_12574_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "noalloc_args.h"
int main() {
    static double X[64], Y[64];
    struct Case { const char *name; NoallocArgs a; long long max_n; };
    const Case cases[] = {
        {"ok",              {2, 8, 0, 0.0, X, Y, 0, 0, 0, 0}, 100},
        {"ok_table_shift",  {2, 8, 1, 0.5, X, Y, 1, 1, 1, 1}, 100},
        {"bad_dim",         {4, 8, 0, 0.0, X, Y, 0, 0, 0, 0}, 100},
        {"bad_n",           {2, 1, 0, 0.0, X, Y, 0, 0, 0, 0}, 100},
        {"bad_grid",        {2, 8, 2, 0.0, X, Y, 0, 0, 0, 0}, 100},
        {"nan_shift",       {2, 8, 0, NAN, X, Y, 0, 0, 0, 0}, 100},
        {"too_large",       {3, 8, 0, 0.0, X, Y, 0, 0, 0, 0}, 100},
        {"null_x",          {2, 8, 0, 0.0, nullptr, Y, 0, 0, 0, 0}, 100},
        {"host_y",          {2, 8, 0, 0.0, X, Y, 0, 0, -1, 0}, 100},
        {"x_other_device",  {2, 8, 0, 0.0, X, Y, 0, 1, 0, 0}, 100},
        {"y_other_device",  {2, 8, 0, 0.0, X, Y, 1, 1, 0, 1}, 100},
        {"stream_other",    {2, 8, 0, 0.0, X, Y, 0, 0, 0, 1}, 100},
        {"overlap",         {2, 8, 0, 0.0, X, X + 3, 0, 0, 0, 0}, 100},
        {"adjacent",        {2, 4, 0, 0.0, X, X + 16, 0, 0, 0, 0}, 100},
    };
    for (const Case &c : cases) {
        long long N = -1;
        const char *why = "";
        int rc = noalloc_check_args(c.a, c.max_n, &N, &why);
        std::printf("%s %d %lld %s\n", c.name, rc, rc == 0 ? N : -1LL, rc == 0 ? "-" : why);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def verdicts(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("noalloc_args")
    src, exe = d / "check.cpp", d / "check"
    src.write_text(PROGRAM)
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    res = {}
    for line in out.splitlines():
        name, rc, N, why = line.split(" ", 3)
        res[name] = (int(rc), int(N), why)
    return res


def test_valid_calls_pass_with_their_size(verdicts):
    assert verdicts["ok"][:2] == (0, 64)
    assert verdicts["ok_table_shift"][:2] == (0, 64)
    assert verdicts["adjacent"][:2] == (0, 16)  # x and y touch but do not overlap


@pytest.mark.parametrize("name,word", [("bad_dim", "dim"), ("bad_n", "n must"), ("bad_grid", "grid"),
                                       ("nan_shift", "a_shift"), ("too_large", "exceeds"),
                                       ("null_x", "NULL"), ("host_y", "device memory"),
                                       ("x_other_device", "current device"), ("y_other_device", "current device"),
                                       ("stream_other", "another device"), ("overlap", "overlap")])
def test_rejections(verdicts, name, word):
    rc, _, why = verdicts[name]
    assert rc == -1 and word in why, (name, why)
