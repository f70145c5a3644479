"""Host-side checks of the C-ABI library: it builds, loads, and exports every symbol that
include/ls.h declares (no compute call: these run without a GPU)."""

import ctypes
import os
import re

import pytest

from paper_1408_4495_gb300 import build as B
from paper_1408_4495_gb300 import ls as LS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "ls.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:ls_status|void|const char\*)\s+(ls_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_binding_exports():
    assert _declared() == sorted(LS.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_structs_match_header_sizes():
    # ls_grid: 8 ints; ls_info: int, int, double, int (padded to 24);
    # ls_nd_stats: 3 ints (+pad) + int64 + 6 doubles
    assert ctypes.sizeof(LS.LsGrid) == 32
    assert ctypes.sizeof(LS.LsInfo) == 24
    assert ctypes.sizeof(LS.LsNdStats) == 72


def test_struct_layout_matches_the_c_compiler(tmp_path):
    # sizeof / offsetof of every field as the C compiler lays out include/ls.h
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"ls_grid": LS.LsGrid, "ls_info": LS.LsInfo, "ls_nd_stats": LS.LsNdStats}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ls.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], check=True, capture_output=True,
                                                   text=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


def test_binding_refuses_without_library(tmp_path):
    saved = LS._lib
    LS._lib = None
    try:
        with pytest.raises(RuntimeError):
            LS.load(str(tmp_path / "missing.so"))
    finally:
        LS._lib = saved


def test_host_entry_points_from_a_c_program(tmp_path, lib):
    # the C-ABI used from C: a program compiled against include/ls.h and linked with libls
    # calls the host computations (no device needed) and reports status and values
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text(r"""
#include <stdio.h>
#include <stdlib.h>
#include "ls.h"
int main(void) {
  double k[2];
  if (ls_k0_weight(3, 6.283185307179586, 1.0 / 17.0, LS_K0_BALL, k) != LS_OK) return 1;
  printf("%.17g %.17g\n", k[0], k[1]);
  if (ls_k0_weight(4, 1.0, 0.1, LS_K0_BALL, k) != LS_EINVAL) return 2;
  const int n = 16;
  double* m = calloc((size_t)n * n, sizeof(double));
  unsigned char* mask = calloc((size_t)n * n, 1);
  m[8 * n + 8] = -0.2;
  if (ls_general_support(2, n, m, 2, mask) != LS_OK) return 3;
  int cnt = 0;
  for (int i = 0; i < n * n; ++i) cnt += mask[i] != 0;
  printf("%d\n", cnt);
  printf("%s\n", ls_last_error(NULL) ? "ok" : "null");
  free(m);
  free(mask);
  return 0;
}
""")
    exe = tmp_path / "use"
    libdir = os.path.dirname(B.LIB)
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lls",
                    "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    re_, im_ = (float(v) for v in out[0].split())
    ref = LS.k0_weight(3, 6.283185307179586, 1.0 / 17.0, LS.LS_K0_BALL)
    assert re_ == ref.real and im_ == ref.imag
    assert int(out[1]) == 7 * 7  # the point and its b + 1 = 3 layers
    assert out[2] == "ok"


def test_fault_injection_arms_and_disarms_on_the_host(lib):
    # arming touches no device; the injected failure itself is exercised by the GPU tests
    assert lib.ls_fault_alloc(ctypes.c_long(3)) == LS.LS_OK
    assert lib.ls_fault_alloc(ctypes.c_long(0)) == LS.LS_OK
    assert lib.ls_fault_alloc(ctypes.c_long(-1)) == LS.LS_EINVAL
    LS.fault_alloc(0)
    with pytest.raises(LS.LsError):
        LS.fault_alloc(-2)
