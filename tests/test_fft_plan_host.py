"""The FFT radix plan and the FP32 passes' per-pass twiddle layout (csrc/fft_plan.h), compiled
on the host: radices multiply to L, each pass's run of NS * R factors follows the previous one
without gap or overlap, every run starts at an even entry (16-byte aligned float2 pairs), the
table stays below 2 L entries, and last_radix names the final pass."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1408_4495_gb300", "csrc")
LENGTHS = [16, 32, 48, 64, 96, 128, 256, 512, 1024, 2048, 4096]

PROG = r"""
#include <cstdio>
#include "fft_plan.h"
int main() {
  const int Ls[] = {%s};
  for (int L : Ls) {
    std::printf("L %%d last %%d size %%d\n", L, ls::last_radix(L), ls::tw_table_size(L));
    for (int NS = 1; NS < L; NS *= ls::pass_radix(L, NS))
      std::printf("pass %%d %%d %%d\n", NS, ls::pass_radix(L, NS), NS > 1 ? ls::tw_pass_offset(L, NS) : -1);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def plan(tmp_path_factory):
    cxx = shutil.which(os.environ.get("CXX", "g++"))
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("fftplan")
    src, exe = d / "p.cpp", d / "p"
    src.write_text(PROG % ", ".join(map(str, LENGTHS)))
    subprocess.run([cxx, "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    plans, cur = {}, None
    for line in out.splitlines():
        f = line.split()
        if f[0] == "L":
            cur = plans.setdefault(int(f[1]), {"last": int(f[3]), "size": int(f[5]), "passes": []})
        else:
            cur["passes"].append(tuple(int(x) for x in f[1:]))
    return plans


@pytest.mark.parametrize("L", LENGTHS)
def test_radices_and_twiddle_runs(plan, L):
    p = plan[L]
    prod = 1
    for NS, R, _ in p["passes"]:
        assert NS == prod and R in (8, 4, 2, 3)
        prod *= R
    assert prod == L
    assert p["passes"][-1][1] == p["last"]
    # radix 8 while the remaining length allows it, then 4 or 2, then 3
    radices = [R for _, R, _ in p["passes"]]
    assert radices == sorted(radices, reverse=True) or radices[-1] == 3
    off = 0
    for NS, R, o in p["passes"][1:]:
        assert o == off and o % 2 == 0
        off += NS * R
    assert p["size"] == off < 2 * L
